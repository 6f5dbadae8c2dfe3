// Kernels of one frame of the CBT bisection update for sm_103a.
//
// Frame = k_prep, k_classify, k_gate, k_scatter, k_alloc, k_free, k_fill,
// k_cbt [, k_vertices], each launched once for a whole batch of independent
// instances (a single instance is a batch of one). Item kernels walk global
// tiles of 1024 live indices; tile t belongs to the instance b with
// tile_base[b] <= t < tile_base[b+1], recomputed on the device each frame
// from the CBT roots (this replaces the paper's DispatchIndirect). The two
// prefix scans and the reduction are single-pass decoupled look-back scans
// over tiles handed out by an atomic ticket, so a tile only waits for tiles
// owned by running blocks; the first tile of each instance starts its own
#include "cbt_kernels.cuh"
#include "cbt_phases.cuh"

namespace cbtgpu {

// ------------------------------------------------------------------ prep

// Frame start: per-instance counters, the item-tile prefix over the batch
// (block 0), the look-back descriptors zeroed, and the camera-relative root
// tables. FP64 is used here only to subtract the eye from the root vertices.
__global__ void __launch_bounds__(kThreads) k_prep(BatchDev bt, int frame_start) {
    __shared__ uint32_t s_carry, s_scarry, s_live;
    __shared__ Pair s_warp[kThreads / 32 + 1];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    if (frame_start) {
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) s_carry = s_scarry = s_live = 0;
            __syncthreads();
            for (uint32_t b0 = 0; b0 < bt.B; b0 += kThreads) {
                const uint32_t b = b0 + threadIdx.x;
                uint32_t tiles = 0, stl = 0;
                if (b < bt.B) {
                    const Inst& I = bt.inst[b];
                    const uint32_t N = I.sums[1];
                    Globals* g = I.g;
                    g->N = N;
                    g->F = I.cap - N;
                    g->A = 0;
                    g->Mg = 0;
                    g->done = 0;
                    g->marks_clean = 0;  // this frame writes its changed list over the chain-mark words
                    g->freel_full = 0;   // and a free list of its allocations only
                    tiles = (N + kTileItems - 1u) / kTileItems;
                    g->ntiles = tiles;
                    stl = (N + kScanItems - 1u) / kScanItems;
                    g->nstiles = stl;
                    for (int k = 0; k < kStCount; ++k) g->stats[k] = 0;
                    g->stats[kStLiveBefore] = N;
                    g->stats[kStFreeBefore] = I.cap - N;
                    g->stats[kStFrame] = frame_of(bt, b).frame;
                    pc_generation(g, frame_of(bt, b));
                    if (bt.nout) bt.nout[b] = N;
                    atomicAdd(&s_live, N);
                }
                Pair tot;
                const Pair ex = block_scan(Pair{stl, tiles}, tot, s_warp);
                if (b < bt.B) {
                    bt.tile_base[b] = s_carry + ex.b;
                    bt.stile_base[b] = s_scarry + ex.a;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    s_carry += tot.b;
                    s_scarry += tot.a;
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                bt.tile_base[bt.B] = s_carry;
                bt.stile_base[bt.B] = s_scarry;
                bt.bg->total_tiles = s_carry;
                bt.bg->total_stiles = s_scarry;
                bt.bg->live_total = s_live;
                for (int k = 0; k < 8; ++k) bt.bg->tickets[k] = 0;
            }
        }
        const uint32_t nstat = 2u * bt.Titems + bt.Twords;
        for (uint32_t k = tid; k < nstat; k += nth) bt.status[k] = 0ull;
    }
    for (uint32_t e = tid; e < bt.Trel; e += nth) rel_entry(bt, e);
}

__global__ void __launch_bounds__(kThreads) k_walk(BatchDev bt) {
    __shared__ uint32_t s_b, s_n;
    __shared__ Inst s_I;
    __shared__ uint2 s_list[kTileItems];  // {live index | split << 31, slot}
    const uint32_t T = ld_volatile(&bt.bg->total_tiles);
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        uint32_t b, lt;
        if (threadIdx.x == 0) s_n = 0;
        tile_begin(bt, bt.tile_base, t, &s_b, &s_I, nullptr, nullptr, b, lt);
        const Inst& I = s_I;
        const FrameP& fp = frame_of(bt, b);
        const bool chain = fp.gate != 1;
        const uint32_t N = I.g->N;
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
            if (i >= N) continue;
            const uint32_t s = I.live[i];
            const uint32_t cmd = *cmd_ptr(I, s);
            const bool split = (cmd & kSplitWish) != 0u;
            const bool need = (split && chain) || ((cmd & kMergeWish) && !(cmd & kHeapOdd));
            if (need) s_list[atomicAdd(&s_n, 1u)] = make_uint2(i | (split ? 0x80000000u : 0u), s);
        }
        __syncthreads();
        const uint32_t n = s_n;
        for (uint32_t q = threadIdx.x; q < n; q += kThreads) {
            const uint2 e = s_list[q];
            const uint32_t i = e.x & 0x7FFFFFFFu, s = e.y;
            if (e.x & 0x80000000u) {
                I.scan[i] = chain_walk(I, s, depth_of(I.heap[s], I.ch), false);
            } else {
                Group g;
                if (find_group(I, s, g) && g.imin == 0) {
                    I.grp[i] = make_uint4(g.m[0], g.m[1], g.m[2], g.m[3]);
                    atomicOr(cmd_ptr(I, s), kGrpMin);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_classify(BatchDev bt) {
    __shared__ uint32_t s_b;
    __shared__ Inst s_I;
    __shared__ FrameP s_fp;
    __shared__ uint32_t s_cnt[kBlockStats];
    __shared__ __align__(16) uint32_t s_tab[kDecTabWords];
    load_dec6(s_tab);
    const uint32_t T = ld_volatile(&bt.bg->total_tiles);
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.tile_base, t, &s_b, &s_I, &s_fp, s_cnt, b, lt);
        const Inst& I = s_I;
        const FrameP& fp = s_fp;
        const uint32_t N = I.g->N;
        const uint64_t key = splitmix64(((uint64_t)fp.seed << 32) | (uint64_t)fp.frame);
        // issue the slot and heap-ID loads of the thread's items first
        uint32_t sl[kItemsPerThread];
        uint64_t hj[kItemsPerThread];
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
            sl[k] = i < N ? I.live[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
            hj[k] = i < N ? I.heap[sl[k]] : 0ull;
        }
#pragma unroll 1
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
            if (i < N) classify_item(I, fp, key, i, sl[k], hj[k], s_tab, s_cnt);
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitWishes);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ gate

// Scan of (merge cost at the group's smallest member, split chain cost) in
// ascending slot order per instance; merges are granted while their running
// total fits the free slots, then splits while (granted merges + their
// running total) fits (deterministic form of the allocation-counter test of
// Sec. 3.3). The smallest member (always an even heap ID) walks its group
// once and records the members for k_alloc and k_fill: m0, m1 are the
// children of the smaller parent, m2, m3 those of the larger one.
__global__ void __launch_bounds__(kScanThreads) k_gate(BatchDev bt) {
    __shared__ uint32_t s_tile, s_b, s_mg;
    __shared__ Pair s_warp[kScanThreads / 32 + 1];
    __shared__ Pair s_excl;
    __shared__ Inst s_I;
    __shared__ uint32_t s_cnt[kBlockStats];
    const uint32_t T = ld_volatile(&bt.bg->total_stiles);
    unsigned long long* status = bt.status;
    for (;;) {
        const uint32_t t = next_ticket(bt.bg, 0, &s_tile);
        if (t >= T) break;
        uint32_t b, lt;
        if (threadIdx.x == 0) s_mg = 0;
        tile_begin(bt, bt.stile_base, t, &s_b, &s_I, nullptr, s_cnt, b, lt);
        const Inst& I = s_I;
        const uint32_t gate = frame_of(bt, b).gate;
        const uint32_t N = I.g->N, F = I.g->F;
        const uint32_t base = lt * kScanItems + threadIdx.x * kScanPerThread;
        Pair v[kScanPerThread];
        Pair loc{0, 0};
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) {
            const uint32_t i = base + k;
            v[k] = Pair{0, 0};
            if (i < N) {
                const uint32_t s = I.live[i];
                const uint32_t cmd = *cmd_ptr(I, s);
                v[k] = Pair{merge_cost(I, i, cmd, gate), I.scan[i]};
                loc = padd(loc, v[k]);
            }
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        const Pair ex = tile_prefix(status, t, lt == 0, tot, I.g, &s_excl);
        Pair run = padd(ex, tex);
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) {
            const uint32_t i = base + k;
            run = padd(run, v[k]);
            if (i >= N) continue;
            const bool cand = v[k].a > 0;
            const bool granted = cand && run.a <= F;
            if (cand) atomicOr(cmd_ptr(I, I.live[i]), granted ? (kCand | kMergeGrant) : kCand);
            if (granted) atomicMax(&s_mg, run.a);
            I.scan[i] = run.b;
            count_stat(s_cnt, 0, cand);
            count_stat(s_cnt, 1, granted);
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStMergeCand, kStMergeGranted);
        if (threadIdx.x == 0 && s_mg) atomicMax(&I.g->Mg, s_mg);
        __syncthreads();
    }
}

// --------------------------------------------------------------- scatter

// Granted split requests mark their chains. The requests of a tile are first
// packed in shared memory so that whole warps walk chains.
__global__ void __launch_bounds__(kThreads) k_scatter(BatchDev bt) {
    __shared__ uint32_t s_b, s_n;
    __shared__ uint32_t s_list[kTileItems];
    __shared__ Inst s_I;
    __shared__ uint32_t s_cnt[kBlockStats];
    const uint32_t T = ld_volatile(&bt.bg->total_tiles);
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        uint32_t b, lt;
        if (threadIdx.x == 0) s_n = 0;
        tile_begin(bt, bt.tile_base, t, &s_b, &s_I, nullptr, s_cnt, b, lt);
        const Inst& I = s_I;
        const uint32_t N = I.g->N;
        const uint64_t F = I.g->F, Mg = ld_volatile(&I.g->Mg);
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
            bool granted = false;
            if (i < N) {
                const uint32_t s = I.live[i];
                if (*cmd_ptr(I, s) & kSplitWish) {
                    granted = Mg + (uint64_t)I.scan[i] <= F;
                    if (granted) s_list[atomicAdd(&s_n, 1u)] = s;
                }
            }
            count_stat(s_cnt, 0, granted);
        }
        __syncthreads();
        const uint32_t n = s_n;
        for (uint32_t k = threadIdx.x; k < n; k += kThreads) chain_walk(I, s_list[k], 0, true);
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitGranted);
        __syncthreads();
    }
}


// Fates and the exclusive scan of allocation counts in ascending slot order
// (ReserveBlocks): a split bisector takes 2-4 leaves, a valid merge group
// its parents at its smallest member, which also marks every member merged
// and gives each the free-list index of its parent.
__global__ void __launch_bounds__(kScanThreads) k_alloc(BatchDev bt) {
    __shared__ uint32_t s_tile, s_b;
    __shared__ Pair s_warp[kScanThreads / 32 + 1];
    __shared__ Pair s_excl;
    __shared__ Inst s_I;
    __shared__ uint32_t s_cnt[kBlockStats];
    const uint32_t T = ld_volatile(&bt.bg->total_stiles);
    unsigned long long* status = bt.status + bt.Titems;
    for (;;) {
        const uint32_t t = next_ticket(bt.bg, 1, &s_tile);
        if (t >= T) break;
        uint32_t b, lt;
        tile_begin(bt, bt.stile_base, t, &s_b, &s_I, nullptr, s_cnt, b, lt);
        const Inst& I = s_I;
        const uint32_t N = I.g->N;
        const uint32_t base = lt * kScanItems + threadIdx.x * kScanPerThread;
        // fate per item, 4 bits each: allocation count (0-4) and whether the
        // item is a merge at its smallest member
        uint32_t packed = 0;
        Pair loc{0, 0};
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) {
            const uint32_t i = base + k;
            if (i >= N) continue;
            const uint32_t f = alloc_fate(I, i, *cmd_ptr(I, I.live[i]));
            const uint32_t na = f & 7u;
            packed |= f << (4 * k);
            loc = padd(loc, Pair{na ? 1u : 0u, na});
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        const Pair ex = tile_prefix(status, t, lt == 0, tot, I.g, &s_excl);
        uint32_t run = ex.b + tex.b;
        uint32_t crun = ex.a + tex.a;
#pragma unroll
        for (int k = 0; k < kScanPerThread; ++k) {
            const uint32_t i = base + k;
            const uint32_t f = (packed >> (4 * k)) & 15u;
            const uint32_t na = f & 7u;
            if (i >= N || !na) continue;
            I.chg[crun++] = i;
            alloc_apply(I, i, f, run, s_cnt);
            run += na;
        }
        if (lt == I.g->nstiles - 1u && threadIdx.x == blockDim.x - 1) {
            I.g->A = run;
            I.g->C = crun;
            I.g->stats[kStAllocated] = run;
            if (run > I.g->F) set_err(I.g, kErrOverflow);
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitBis, kStMergeGroups, kStMergedBis);
        __syncthreads();
    }
}

// ------------------------------------------------------------- free list

// freel[k] = slot of the k-th zero bit of the frame-start bitfield, k < A
// (Alg. 8 for the first A ranks at once): each tile of words (one word per
// thread) finds its zero offset from the sum tree and emits its zeros.
__global__ void __launch_bounds__(kMaxTileWords) k_free(BatchDev bt) {
    __shared__ uint32_t s_b, s_carry;
    __shared__ uint32_t s_w[kMaxTileWords / 32 + 1];
    __shared__ Inst s_I;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (blockIdx.x == 0) {
        // tiles of the changed-bisector lists, for k_fill
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        for (uint32_t b0 = 0; b0 < bt.B; b0 += blockDim.x) {
            const uint32_t b = b0 + threadIdx.x;
            const uint32_t n = b < bt.B ? (ld_volatile(&bt.inst[b].g->C) + kThreads - 1u) / kThreads : 0u;
            uint32_t inc = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_w[warp] = inc;
            __syncthreads();
            if (warp == 0) {
                const uint32_t x = lane < nw ? s_w[lane] : 0u;
                uint32_t xi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
                    if (lane >= o) xi += y;
                }
                __syncwarp();
                if (lane < nw) s_w[lane] = xi - x;
                if (lane == nw - 1) s_w[nw] = xi;
            }
            __syncthreads();
            if (b < bt.B) bt.ctile_base[b] = s_carry + s_w[warp] + inc - n;
            __syncthreads();
            if (threadIdx.x == 0) s_carry += s_w[nw];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            bt.ctile_base[bt.B] = s_carry;
            bt.bg->total_ctiles = s_carry;
        }
        __syncthreads();
    }
    for (uint32_t t = blockIdx.x; t < bt.Twords; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.wtile_base, t, &s_b, &s_I, nullptr, nullptr, b, lt);
        const Inst& I = s_I;
        const uint32_t A = min(ld_volatile(&I.g->A), I.g->F);
        const uint32_t TW = min(I.W, bt.tw);
        const uint32_t nt = I.W / TW;
        uint32_t ones_before = 0;
        for (uint32_t n = nt + lt; n > 1; n >>= 1)
            if (n & 1u) ones_before += I.sums[n - 1];
        const uint64_t zeros_before = (uint64_t)lt * TW * 32u - ones_before;
        if (zeros_before < A) {  // block-uniform
            const uint32_t w = lt * TW + threadIdx.x;
            uint32_t z = 0;
            if (threadIdx.x < TW) {
                const uint32_t valid = I.cap < 32u ? (1u << I.cap) - 1u : 0xFFFFFFFFu;
                z = ~I.bits[w] & valid;
            }
            const uint32_t mine = __popc(z);
            uint32_t inc = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_w[warp] = inc;
            __syncthreads();
            if (warp == 0) {
                const uint32_t x = lane < nw ? s_w[lane] : 0u;
                uint32_t xi = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
                    if (lane >= o) xi += y;
                }
                __syncwarp();
                if (lane < nw) s_w[lane] = xi - x;
            }
            __syncthreads();
            uint64_t r = zeros_before + s_w[warp] + (inc - mine);
            while (z && r < A) {
                I.freel[r] = w * 32u + (uint32_t)(__ffs(z) - 1);
                ++r;
                z &= z - 1u;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_fill(BatchDev bt) {
    __shared__ uint32_t s_b;
    __shared__ Inst s_I;
    __shared__ uint32_t s_cnt[kBlockStats];
    const uint32_t T = ld_volatile(&bt.bg->total_ctiles);
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.ctile_base, t, &s_b, &s_I, nullptr, s_cnt, b, lt);
        const Inst& I = s_I;
        const uint32_t C = I.g->C;
        const uint32_t k = lt * kThreads + threadIdx.x;
        if (k < C) {
            const uint32_t i = I.chg[k];
            const uint32_t s = I.live[i];
            const uint2 c = I.cd[s];
            uint32_t relinked;
            if (c.x & kSplitMask) {
                clear_bit(I, s);
                relinked = fill_split(I, s, c.x, c.y, DestPlain{I.g->A});
            } else {
                const uint4 m = I.grp[i];
                const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (ms[q] != kNull && !bad_slot(I, ms[q], kErrLink)) clear_bit(I, ms[q]);
                relinked = fill_merge(I, c.y, m, DestPlain{I.g->A});
            }
            if (relinked) atomicAdd(&s_cnt[0], relinked);
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStRelinked);
        __syncthreads();
    }
}

// ------------------------------------------------------ reduce + compact

// SumReduction over the updated bitfield (Sec. 3.1): each tile of words (one
// word per thread) writes its part of the sum tree; the last tile of an
// instance to finish builds the levels above its tiles.
__global__ void __launch_bounds__(kMaxTileWords) k_cbt(BatchDev bt) {
    __shared__ uint32_t s_b, s_last;
    __shared__ uint32_t s_lvl[kMaxTileWords];
    __shared__ Inst s_I;
    for (uint32_t t = blockIdx.x; t < bt.Twords; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.wtile_base, t, &s_b, &s_I, nullptr, nullptr, b, lt);
        const Inst& I = s_I;
        const uint32_t W = I.W;
        const uint32_t TW = min(W, bt.tw);
        const uint32_t nt = W / TW;
        const uint32_t w = lt * TW + threadIdx.x;
        const bool mine = threadIdx.x < TW;
        const uint32_t pc = mine ? __popc(I.bits[w]) : 0u;
        if (mine) I.sums[W + w] = pc;
        s_lvl[threadIdx.x] = pc;
        __syncthreads();
        uint32_t lvl = 1;
        for (uint32_t cnt = TW >> 1; cnt >= 1u; cnt >>= 1, ++lvl) {
            uint32_t v = 0;
            if (threadIdx.x < cnt) v = s_lvl[2 * threadIdx.x] + s_lvl[2 * threadIdx.x + 1];
            __syncthreads();
            if (threadIdx.x < cnt) {
                s_lvl[threadIdx.x] = v;
                I.sums[((W + lt * TW) >> lvl) + threadIdx.x] = v;
            }
            __syncthreads();
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&I.g->done, 1u) == nt - 1u) ? 1u : 0u;
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (uint32_t n = nt >> 1; n >= 1u; n >>= 1) {
                for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
                    I.sums[n + k] = __ldcg(I.sums + 2u * (n + k)) + __ldcg(I.sums + 2u * (n + k) + 1u);
                __threadfence();
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                I.g->stats[kStLiveAfter] = __ldcg(I.sums + 1);
                I.g->done = 0;
            }
        }
        __syncthreads();
    }
}

// CachePointers' live list (Alg. 7 for every rank at once) from the finished
// sum tree: each tile of words finds its live-count offset by walking up the
// tree (adding left siblings), scans its popcounts and writes the slots of
// its set bits, staged in shared memory so that the stores are coalesced.
__global__ void __launch_bounds__(kMaxTileWords) k_compact(BatchDev bt) {
    __shared__ uint32_t s_b;
    __shared__ uint32_t s_w[kMaxTileWords / 32 + 1];
    __shared__ uint32_t s_live[kMaxTileWords * 32];
    __shared__ Inst s_I;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t t = blockIdx.x; t < bt.Twords; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.wtile_base, t, &s_b, &s_I, nullptr, nullptr, b, lt);
        const Inst& I = s_I;
        const uint32_t W = I.W;
        const uint32_t TW = min(W, bt.tw);
        const uint32_t nt = W / TW;
        uint32_t before = 0;
        for (uint32_t n = nt + lt; n > 1; n >>= 1)
            if (n & 1u) before += I.sums[n - 1];
        const uint32_t w = lt * TW + threadIdx.x;
        const uint32_t wv = threadIdx.x < TW ? I.bits[w] : 0u;
        const uint32_t pc = __popc(wv);
        uint32_t inc = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t x = lane < nw ? s_w[lane] : 0u;
            uint32_t xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
                if (lane >= o) xi += y;
            }
            __syncwarp();
            if (lane < nw) s_w[lane] = xi - x;
            if (lane == nw - 1) s_w[nw] = xi;
        }
        __syncthreads();
        uint32_t r = s_w[warp] + inc - pc;
        const uint32_t tot = s_w[nw];
        uint32_t m = wv;
        while (m) {
            s_live[r++] = w * 32u + (uint32_t)(__ffs(m) - 1);
            m &= m - 1u;
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < tot; k += blockDim.x) I.live[before + k] = s_live[k];
        __syncthreads();
    }
}

// ------------------------------------------------------------------ init

// Root bisectors (Sec. 3.3 "Initialization") and the root vertex table
// (Alg. 1, one FP64 centroid per face summed from its smallest halfedge).
__global__ void __launch_bounds__(kThreads) k_init(Inst I, const int32_t* twin, const int32_t* next,
                                                   const int32_t* prev, const double* hpos) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    for (uint32_t w = tid; w < I.W; w += nth) {
        const uint32_t lo = w * 32u;
        uint32_t m = 0;
        if (lo < I.H) m = (I.H - lo >= 32u) ? 0xFFFFFFFFu : ((1u << (I.H - lo)) - 1u);
        I.bits[w] = m;
    }
    for (uint32_t h = tid; h < I.H; h += nth) {
        I.heap[h] = (1ull << I.ch) + h;
        const uint32_t tw = twin[h] < 0 ? kNull : (uint32_t)twin[h];
        const uint32_t rv = (tw == kNull ? 3u : (uint32_t)kT) | ((uint32_t)kPe << 2) | ((uint32_t)kNe << 4);
        I.nb[h] = make_uint4(tw, (uint32_t)next[h], (uint32_t)prev[h], rv);
        // smallest halfedge index of h's face
        int32_t first = (int32_t)h, x = next[h];
        for (uint32_t guard = 0; x != (int32_t)h && guard < I.H; ++guard) {
            if (x < first) first = x;
            x = next[x];
        }
        double sx = 0.0, sy = 0.0, sz = 0.0;
        uint32_t n = 0;
        x = first;
        do {
            sx = __dadd_rn(sx, hpos[3 * x + 0]);
            sy = __dadd_rn(sy, hpos[3 * x + 1]);
            sz = __dadd_rn(sz, hpos[3 * x + 2]);
            ++n;
            x = next[x];
        } while (x != first && n <= I.H);
        const double dn = (double)n;
        double* R = I.root64 + 9u * h;
        const int32_t nh = next[h];
        for (int c = 0; c < 3; ++c) {
            R[c] = hpos[3 * h + c];
            R[3 + c] = hpos[3 * nh + c];
        }
        R[6] = __ddiv_rn(sx, dn);
        R[7] = __ddiv_rn(sy, dn);
        R[8] = __ddiv_rn(sz, dn);
    }
}

// -------------------------------------------------------------- exports

__global__ void __launch_bounds__(kThreads) k_leaves(Inst I, uint32_t* slots, uint64_t* heap,
                                                     uint32_t* links) {
    const uint32_t N = I.sums[1];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t s = I.live[i];
        if (slots) slots[i] = s;
        if (heap) heap[i] = I.heap[s];
        if (links) {
            const uint4 r = I.nb[s];
            links[3 * i + 0] = r.x;
            links[3 * i + 1] = r.y;
            links[3 * i + 2] = r.z;
        }
    }
}

// over static tiles of its pool capacity (tiles past the live count exit).
__global__ void __launch_bounds__(kThreads, 3) k_vertices(BatchDev bt) {
    __shared__ uint32_t s_b;
    __shared__ Inst s_I;
    __shared__ FrameP s_fp;
    __shared__ __align__(16) uint32_t s_tab[kDecTabWords];
    __shared__ __align__(16) float s_stage[kThreads / 32][288];  // per warp: 32 rows of 9 floats
    load_dec6(s_tab);
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t t = blockIdx.x; t < bt.Titems; t += gridDim.x) {
        uint32_t b, lt;
        tile_begin(bt, bt.vtile_base, t, &s_b, &s_I, &s_fp, nullptr, b, lt);
        const Inst& I = s_I;
        const FrameP& fp = s_fp;
        const uint32_t N = fp.vout ? min(I.sums[1], fp.vcap) : 0u;
        if (lt * kTileItems < N) {
            uint64_t hj[kItemsPerThread];
#pragma unroll
            for (int k = 0; k < kItemsPerThread; ++k) {
                const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
                hj[k] = i < N ? I.heap[I.live[i]] : 0ull;
            }
#pragma unroll 1
            for (int k = 0; k < kItemsPerThread; ++k) {  // warp-uniform: 32 consecutive rows per warp
                const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
                const uint32_t w0 = i - lane;
                if (w0 >= N) continue;
                float r[9];
                bool ok = true;
                if (i < N) ok = vertex_eval(I, fp, hj[k], s_tab, r);
                if (__all_sync(0xFFFFFFFFu, ok)) {
                    warp_rows_out(r, s_stage[threadIdx.x >> 5], fp.vout, w0, min(32u, N - w0));
                } else if (i < N && ok) {  // a row the decode refused stays unwritten
                    float* o = fp.vout + 9ull * i;
#pragma unroll
                    for (int q = 0; q < 9; ++q) o[q] = r[q];
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launch

void launch_prep(const BatchDev& bt, bool frame_start, int grid, cudaStream_t s) {
    k_prep<<<grid, kThreads, 0, s>>>(bt, frame_start ? 1 : 0);
}
void launch_classify(const BatchDev& bt, int grid, cudaStream_t s) { k_classify<<<grid, kThreads, 0, s>>>(bt); }
void launch_walk(const BatchDev& bt, int grid, cudaStream_t s) { k_walk<<<grid, kThreads, 0, s>>>(bt); }
void launch_gate(const BatchDev& bt, int grid, cudaStream_t s) { k_gate<<<grid, kScanThreads, 0, s>>>(bt); }
void launch_scatter(const BatchDev& bt, int grid, cudaStream_t s) { k_scatter<<<grid, kThreads, 0, s>>>(bt); }
void launch_alloc(const BatchDev& bt, int grid, cudaStream_t s) { k_alloc<<<grid, kScanThreads, 0, s>>>(bt); }
void launch_free(const BatchDev& bt, int grid, cudaStream_t s) { k_free<<<grid, bt.tw, 0, s>>>(bt); }
void launch_fill(const BatchDev& bt, int grid, cudaStream_t s) { k_fill<<<grid, kThreads, 0, s>>>(bt); }
void launch_cbt(const BatchDev& bt, int grid, cudaStream_t s) {
    k_cbt<<<grid, bt.tw, 0, s>>>(bt);
    k_compact<<<grid, bt.tw, 0, s>>>(bt);
}
void launch_vertices(const BatchDev& bt, int grid, cudaStream_t s) { k_vertices<<<grid, kThreads, 0, s>>>(bt); }
void launch_init(const Inst& I, const int32_t* twin, const int32_t* next, const int32_t* prev,
                 const double* hpos, int grid, cudaStream_t s) {
    k_init<<<grid, kThreads, 0, s>>>(I, twin, next, prev, hpos);
}
void launch_leaves(const Inst& I, uint32_t* slots, uint64_t* heap, uint32_t* links, int grid,
                   cudaStream_t s) {
    k_leaves<<<grid, kThreads, 0, s>>>(I, slots, heap, links);
}

}  // namespace cbtgpu
