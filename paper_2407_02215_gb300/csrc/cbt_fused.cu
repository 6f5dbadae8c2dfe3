// One frame of a batch in one launch (the Sec. 3.3 pipeline, Alg. 9): a
// persistent cooperative kernel, every block resident, whose phases are
// separated by grid-wide barriers instead of kernel boundaries.
//
//   P0 prep       frame counters, item-tile prefix, camera-relative roots
//   P1 classify   LOD wishes, then the chain and group walks of the same tile
//   P2 gate-sum   per-tile sums of (merge cost, split cost)
//   P3 gate       tile prefix from the sums, grants, chain marking
//   P4 alloc-sum  fates and per-tile sums of (changed, allocations); free list
//   P5 alloc      tile prefix, free-list indices of the new records
//   P6 fill       new records, neighbour links, bitfield
//   P7 reduce     sum tree (the last word tile of an instance builds the top)
//   P8 compact    live list, and the vertices of the new triangulation
//
// The two prefix sums of the per-step kernels (decoupled look-back) become
// reduce-then-scan here: tile sums, a barrier, then each tile adds the sums
// before it. State between phases lives in the slot arrays (command words,
// scan words); each block keeps its instance descriptor and frame
// parameters in shared memory across tiles and phases. Reads of data other
// blocks wrote in an earlier phase follow a barrier whose fences order them.
// Every wait is bounded: a barrier that runs out sets the batch's abort word,
// every later wait then returns at once, and the instances report kErrTimeout.
#include "cbt_kernels.cuh"
#include "cbt_phases.cuh"

namespace cbtgpu {

namespace {

constexpr int kFThreads = 256;
constexpr int kFPer = 4;  // items per thread and tile: kFThreads * kFPer == kTileItems
static_assert(kFThreads * kFPer == (int)kTileItems, "tile shape");
constexpr uint32_t kFBuf = 4096;  // shared scratch words (lists, tree top, live slots)
constexpr uint32_t kRelRange = 256;  // root-table entries per warp range in P0
constexpr uint32_t kMinIpt = 4, kMaxIpt = 8;  // items per thread of a scan tile
constexpr int kBarrierSpin = 1 << 22;
constexpr uint32_t kBarriers = 8;  // grid barriers per frame (one more for a single instance)

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier k (1-based) of the launch: a monotonic arrival counter
// that never resets; barrier k of a launch that started at count `epoch` is
// passed once the count reaches epoch + k * gridDim.x (wrap-safe compare).
// Arrival is a release reduction of the block's writes (ordered after the
// whole block by __syncthreads); the spin is an acquire load. The launch is
// cooperative, so every block is resident and every arrival comes.
__device__ void grid_wait(BatchGlobals* bg, uint32_t target, int limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_gpu(&bg->bar_count, 1u);
        int it = 0;
        while ((int)(ld_acquire_gpu(&bg->bar_count) - target) < 0) {
            if (ld_volatile(&bg->abort)) break;
            if (++it > limit) {
                atomicExch(&bg->abort, 1u);
                break;
            }
            __nanosleep(32);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void grid_sync(BatchGlobals* bg, uint32_t epoch, uint32_t k) {
    grid_wait(bg, epoch + k * gridDim.x, kBarrierSpin);
}

__device__ __forceinline__ void stamp(const BatchDev& bt, int k) {
    if (bt.timing && blockIdx.x == 0 && threadIdx.x == 0) bt.bg->t[k] = global_ns();
}

// Per-block context: the instance of the current tile (descriptor and frame
// parameters reloaded only when the instance changes) and the tile's place.
struct FCtx {
    Inst I;
    FrameP fp;
    uint32_t b;       // cached instance, kNull before the first tile
    uint32_t nb, lt;  // instance and local index of the current tile
    uint32_t tb, te;  // the instance's tiles in the current partition
    uint32_t N, F;    // frame-start live and free counts of the cached instance
};

// Block-uniform; ends with __syncthreads.
__device__ __forceinline__ void ctx_tile(const BatchDev& bt, const uint32_t* base, uint32_t t, uint32_t T,
                                         FCtx& c) {
    if (threadIdx.x == 0) {
        if (bt.B == 1) {  // base[0] = 0, base[1] = T
            c.nb = 0;
            c.lt = t;
            c.tb = 0;
            c.te = T;
        } else {
            const uint32_t b = find_inst(base, bt.B, t);
            c.nb = b;
            c.lt = t - base[b];
            c.tb = base[b];
            c.te = base[b + 1];
        }
    }
    __syncthreads();
    const uint32_t b = c.nb;
    if (b != c.b) {
        load_tile_ctx(bt, b, &c.I, &c.fp);
        __syncthreads();
        if (threadIdx.x == 0) {
            c.b = b;
            c.N = c.I.g->N;
            c.F = c.I.g->F;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ unsigned long long pack_pair(Pair p) {
    return ((unsigned long long)p.a << 32) | (unsigned long long)p.b;
}
__device__ __forceinline__ Pair unpack_pair(unsigned long long v) {
    return Pair{(uint32_t)(v >> 32), (uint32_t)v};
}

// Block sums of two Pairs (s_red: 4 * (blockDim / 32) words); every thread
// gets both totals.
__device__ __forceinline__ void block_sum2(Pair& x, Pair& y, uint32_t* s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    uint32_t v[4] = {x.a, x.b, y.a, y.b};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xFFFFFFFFu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q) s_red[4 * warp + q] = v[q];
    __syncthreads();
    uint32_t r[4] = {0, 0, 0, 0};
    for (int w = 0; w < nw; ++w)
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] += s_red[4 * w + q];
    __syncthreads();
    x = Pair{min(r[0], kSat), min(r[1], kSat)};
    y = Pair{min(r[2], kSat), min(r[3], kSat)};
}

// Sums of the tile aggregates of the current instance: before tile t, and
// over all its tiles.
__device__ __forceinline__ void tile_sums(const unsigned long long* agg, const FCtx& c, Pair& before, Pair& all,
                                          uint32_t* s_red) {
    const uint32_t t = c.tb + c.lt;
    before = Pair{0, 0};
    all = Pair{0, 0};
    for (uint32_t u = c.tb + threadIdx.x; u < c.te; u += blockDim.x) {
        const Pair v = unpack_pair(__ldcg(agg + u));
        all = padd(all, v);
        if (u < t) before = padd(before, v);
    }
    block_sum2(before, all, s_red);
}

// ------------------------------------------------------------------ phases

// P0: frame counters per instance; the item tiles (kTileItems live indices)
// and the scan tiles (kFThreads * ipt, one per block when the live total
// allows) laid out over the batch; the camera-relative root tables.
__device__ void phase_prep(const BatchDev& bt, Pair* s_warp, uint32_t* s_tmp) {
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) s_tmp[0] = s_tmp[1] = s_tmp[2] = 0;
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < bt.B; b += blockDim.x) atomicAdd(&s_tmp[2], bt.inst[b].sums[1]);
        __syncthreads();
        const uint32_t per_round = gridDim.x * kFThreads;
        const uint32_t ipt = min(kMaxIpt, max(kMinIpt, (s_tmp[2] + per_round - 1u) / per_round));
        const uint32_t S = ipt * kFThreads;
        for (uint32_t b0 = 0; b0 < bt.B; b0 += blockDim.x) {
            const uint32_t b = b0 + threadIdx.x;
            uint32_t tiles = 0, stiles = 0;
            if (b < bt.B) {
                const Inst& I = bt.inst[b];
                const uint32_t N = I.sums[1];
                Globals* g = I.g;
                g->N = N;
                g->F = I.cap - N;
                g->A = 0;
                g->Mg = 0;
                g->Stot = 0;
                g->C = 0;
                g->done = 0;
                tiles = (N + kTileItems - 1u) / kTileItems;
                stiles = (N + S - 1u) / S;
                g->ntiles = tiles;
                g->nstiles = stiles;
                for (int k = 0; k < kStCount; ++k) g->stats[k] = 0;
                g->stats[kStLiveBefore] = N;
                g->stats[kStFreeBefore] = I.cap - N;
                g->stats[kStFrame] = frame_of(bt, b).frame;
                pc_generation(g, frame_of(bt, b));
                if (bt.nout) bt.nout[b] = N;
            }
            Pair tot;
            const Pair ex = block_scan(Pair{stiles, tiles}, tot, s_warp);
            if (b < bt.B) {
                bt.tile_base[b] = s_tmp[0] + ex.b;
                bt.stile_base[b] = s_tmp[1] + ex.a;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_tmp[0] += tot.b;
                s_tmp[1] += tot.a;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            bt.tile_base[bt.B] = s_tmp[0];
            bt.stile_base[bt.B] = s_tmp[1];
            bt.bg->total_tiles = s_tmp[0];
            bt.bg->total_stiles = s_tmp[1];
            bt.bg->scan_ipt = ipt;
            bt.bg->live_total = s_tmp[2];
            bt.bg->t[kFramePhases] = 0;
        }
    }
    // block 0 sets up the instances; the others share the root tables in
    // warp ranges (a multiple of 32 entries, at most kRelRange, enough ranges
    // for every warp)
    if (gridDim.x == 1 || blockIdx.x > 0) {
        const uint32_t nb = gridDim.x > 1 ? gridDim.x - 1u : 1u, bb = gridDim.x > 1 ? blockIdx.x - 1u : 0u;
        const uint32_t nw = nb * (kFThreads / 32), wid = bb * (kFThreads / 32) + threadIdx.x / 32u;
        const uint32_t per = min(kRelRange, ((bt.Trel + nw - 1u) / nw + 31u) & ~31u);
        for (uint32_t e = wid * per; e < bt.Trel; e += nw * per) rel_range(bt, e, min(bt.Trel, e + per));
    }
}

// Walks of listed items on the frame-start state: the chain cost of a split
// wish (command form of Alg. 3, its members recorded in its grp word for the
// marking), the Alg. 4 group of a merge wish with an even heap ID (its
// smallest member records the members).
__device__ __forceinline__ void walk_list(const Inst& I, const uint2* s_list, uint32_t n) {
    for (uint32_t q = threadIdx.x; q < n; q += kFThreads) {
        const uint2 e = s_list[q];
        const uint32_t i = e.x & 0x7FFFFFFFu, s = e.y;
        if (e.x & 0x80000000u) {
            uint4 rec;
            I.scan[i] = chain_walk(I, s, depth_of(I.heap[s], I.ch), false, &rec);
            I.grp[i] = rec;
        } else {
            Group g;
            if (find_group(I, s, g) && g.imin == 0) {
                I.grp[i] = make_uint4(g.m[0], g.m[1], g.m[2], g.m[3]);
                atomicOr(cmd_ptr(I, s), kGrpMin);
            }
        }
    }
}

__device__ __forceinline__ void classify_one(const Inst& I, const FrameP& fp, uint64_t key, uint32_t i, uint32_t s,
                                             uint64_t j, const uint32_t* s_tab, uint32_t* s_cnt, bool chain,
                                             uint32_t* s_n, uint2* s_list) {
    const uint32_t cmd = classify_item(I, fp, key, i, s, j, s_tab, s_cnt, vc_form(fp) && fp.vout);
    const bool split = (cmd & kSplitWish) && chain;
    const bool group = (cmd & kMergeWish) && !(cmd & kHeapOdd);
    if (split || group) s_list[atomicAdd(s_n, 1u)] = make_uint2(i | (split ? 0x80000000u : 0u), s);
}

constexpr uint32_t kWalkCap = kFBuf / 2;  // uint2 entries of the walk list

// P1: wishes of every live bisector (Sec. 3.3 GenerateCommands with the R8
// LOD reading), then the walks of the listed items. A single instance
// strides its live list over the whole grid (balanced; the slot and heap ID
// of the next rounds are loaded while the current item is classified); a
// batch walks its item tiles.
__device__ void phase_classify(const BatchDev& bt, FCtx& c, uint32_t* s_tab, uint32_t* s_cnt, uint32_t* s_n,
                               uint2* s_list) {
    if (bt.B == 1) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.tile_base, 0, 1, c);
        const Inst& I = c.I;
        const FrameP& fp = c.fp;
        const uint32_t N = c.N;
        const bool chain = fp.gate != 1;
        const uint64_t key = splitmix64(((uint64_t)fp.seed << 32) | (uint64_t)fp.frame);
        const uint32_t stride = gridDim.x * kFThreads;
        uint32_t i = blockIdx.x * kFThreads + threadIdx.x;
        uint32_t sa = i < N ? I.live[i] : 0u;
        uint64_t ja = i < N ? I.heap[sa] : 0ull;
        uint32_t sb = i + stride < N ? I.live[i + stride] : 0u;
        for (uint32_t base = blockIdx.x * kFThreads; base < N; base += stride, i += stride) {
            const uint32_t sc = i + 2u * stride < N ? I.live[i + 2u * stride] : 0u;
            const uint64_t jb = i + stride < N ? I.heap[sb] : 0ull;
            if (i < N) classify_one(I, fp, key, i, sa, ja, s_tab, s_cnt, chain, s_n, s_list);
            sa = sb;
            ja = jb;
            sb = sc;
            __syncthreads();
            const uint32_t n = *s_n;
            __syncthreads();
            if (n > kWalkCap - kFThreads) {  // block-uniform
                walk_list(I, s_list, n);
                __syncthreads();
                if (threadIdx.x == 0) *s_n = 0;
                __syncthreads();
            }
        }
        __syncthreads();
        walk_list(I, s_list, *s_n);
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitWishes);
        __syncthreads();
        return;
    }
    const uint32_t T = bt.bg->total_tiles;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.tile_base, t, T, c);
        const Inst& I = c.I;
        const FrameP& fp = c.fp;
        const uint32_t N = c.N;
        const uint32_t lt = c.lt;
        const bool chain = fp.gate != 1;
        const uint64_t key = splitmix64(((uint64_t)fp.seed << 32) | (uint64_t)fp.frame);
        uint32_t sl[kFPer];
        uint64_t hj[kFPer];
#pragma unroll
        for (int k = 0; k < kFPer; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kFThreads + threadIdx.x;
            sl[k] = i < N ? I.live[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kFPer; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kFThreads + threadIdx.x;
            hj[k] = i < N ? I.heap[sl[k]] : 0ull;
        }
#pragma unroll 1
        for (int k = 0; k < kFPer; ++k) {
            const uint32_t i = lt * kTileItems + (uint32_t)k * kFThreads + threadIdx.x;
            if (i < N) classify_one(I, fp, key, i, sl[k], hj[k], s_tab, s_cnt, chain, s_n, s_list);
        }
        __syncthreads();
        walk_list(I, s_list, *s_n);
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitWishes);
        __syncthreads();
    }
}

// Scan tiles: tile lt of an instance covers live indices [lt S, (lt+1) S)
// with S = kFThreads * ipt; thread x holds the ipt consecutive indices from
// lt S + x ipt (the order of the prefix sums).
__device__ __forceinline__ uint32_t stile_first(const FCtx& c, uint32_t ipt) {
    return c.lt * kFThreads * ipt + threadIdx.x * ipt;
}

// P2: per item its split cost and, at a merge group's smallest member, the
// merge cost (kept in the top byte of its scan word for P3); per tile the
// sums. The group checks (group record, then the members' command words)
// run from a list, two dependent loads per listed item.
__device__ void phase_gate_sum(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_red, uint32_t* s_n,
                               uint32_t* s_list) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = c.I;
        const uint32_t N = c.N;
        const uint32_t i0 = stile_first(c, ipt);
        uint32_t sl[kMaxIpt];
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const bool in = k < ipt && i0 + k < N;
            sl[k] = in ? I.live[i0 + k] : kNull;
            loc.b += in ? I.scan[i0 + k] : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k)
            if (sl[k] != kNull && (*cmd_ptr(I, sl[k]) & kGrpMin)) s_list[atomicAdd(s_n, 1u)] = i0 + k;
        __syncthreads();
        const uint32_t n = *s_n;
        for (uint32_t q = threadIdx.x; q < n; q += kFThreads) {
            const uint32_t i = s_list[q];
            const uint32_t mc = merge_cost(I, i, kGrpMin, c.fp.gate);
            if (mc) I.scan[i] |= mc << 24;
            loc.a += mc;
            count_stat(s_cnt, 0, mc != 0u);
        }
        Pair dummy{0, 0};
        block_sum2(loc, dummy, s_red);
        if (threadIdx.x == 0) bt.status[t] = pack_pair(loc);
        stats_flush(s_cnt, I.g, kStMergeCand);
        __syncthreads();
    }
}

// Granted merge total Mg when the merge requests of the instance overflow F:
// the largest inclusive merge prefix that fits (merges are granted first, in
// slot order). Only taken when the instance's merge sum exceeds F.
__device__ uint32_t crossing_mg(const BatchDev& bt, const FCtx& c, uint32_t F, uint32_t ipt, Pair* s_warp,
                                uint32_t* s_tmp) {
    if (threadIdx.x == 0) {
        uint32_t acc = 0, u = c.tb;
        for (; u < c.te; ++u) {
            const uint32_t a = unpack_pair(__ldcg(bt.status + u)).a;
            if ((uint64_t)acc + a > F) break;
            acc += a;
        }
        s_tmp[0] = u - c.tb;
        s_tmp[1] = acc;
        s_tmp[2] = acc;
    }
    __syncthreads();
    const uint32_t lt = s_tmp[0], acc = s_tmp[1];
    const Inst& I = c.I;
    const uint32_t i0 = lt * kFThreads * ipt + threadIdx.x * ipt;
    uint32_t mc[kMaxIpt];
    uint32_t loc = 0;
#pragma unroll
    for (uint32_t k = 0; k < kMaxIpt; ++k) {
        mc[k] = (k < ipt && i0 + k < c.N) ? (__ldcg(I.scan + i0 + k) >> 24) : 0u;
        loc += mc[k];
    }
    Pair tot;
    const Pair ex = block_scan(Pair{0, loc}, tot, s_warp);
    uint32_t run = acc + ex.b, best = acc;
#pragma unroll
    for (uint32_t k = 0; k < kMaxIpt; ++k) {
        run += mc[k];
        if (mc[k] && run <= F) best = max(best, run);
    }
    atomicMax(&s_tmp[2], best);
    __syncthreads();
    const uint32_t r = s_tmp[2];
    __syncthreads();
    return r;
}

// P3: tile prefix of the (merge, split) costs from the tile sums; merges are
// granted while their running total fits F, splits while Mg plus theirs
// does (R6 reading); granted splits mark their chains (command form of
// Alg. 3).
__device__ void phase_gate(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_red, Pair* s_warp,
                           uint32_t* s_tmp, uint32_t* s_n, uint2* s_list) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = c.I;
        const uint32_t N = c.N, F = c.F;
        Pair before, all;
        tile_sums(bt.status, c, before, all, s_red);
        const uint32_t Mg = all.a <= F ? all.a : crossing_mg(bt, c, F, ipt, s_warp, s_tmp);
        if (c.lt == 0 && threadIdx.x == 0) {
            I.g->Mg = Mg;
            I.g->Stot = all.b;
        }
        const uint32_t i0 = stile_first(c, ipt);
        uint32_t sl[kMaxIpt], w[kMaxIpt];
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const bool in = k < ipt && i0 + k < N;
            sl[k] = in ? I.live[i0 + k] : kNull;
            w[k] = in ? I.scan[i0 + k] : 0u;
            loc = padd(loc, Pair{w[k] >> 24, w[k] & 0xFFFFFFu});
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        Pair run = padd(before, tex);
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t mc = w[k] >> 24, sc = w[k] & 0xFFFFFFu;
            run = padd(run, Pair{mc, sc});
            if (sl[k] == kNull) continue;
            const bool mgrant = mc > 0u && run.a <= F;
            if (mc) atomicOr(cmd_ptr(I, sl[k]), mgrant ? (kCand | kMergeGrant) : kCand);
            count_stat(s_cnt, 0, mgrant);
            // a split wish, and only a split wish, has a nonzero split cost
            const bool sgrant = sc > 0u && (uint64_t)Mg + (uint64_t)run.b <= F;
            if (sgrant) s_list[atomicAdd(s_n, 1u)] = make_uint2(i0 + k, sl[k]);
            count_stat(s_cnt, 1, sgrant);
        }
        __syncthreads();
        const uint32_t n = *s_n;
        const bool recorded = c.fp.gate != 1;  // the paper's gate charges 3d + 4 without a walk
        for (uint32_t q = threadIdx.x; q < n; q += kFThreads) {
            const uint2 e = s_list[q];
            const uint4 r = recorded ? I.grp[e.x] : make_uint4(kNull, kNull, kNull, kNull);
            if (r.x == kNull && r.w == kNull) {
                chain_walk(I, e.y, 0, true);
                continue;
            }
            atomicOr(cmd_ptr(I, e.y), kR);
            const uint32_t m[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (uint32_t q2 = 0; q2 < 4; ++q2)
                if (m[q2] >> 30) atomicOr(cmd_ptr(I, m[q2] & 0x3FFFFFFFu), chain_code_bits(m[q2] >> 30));
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStMergeGranted, kStSplitGranted);
        __syncthreads();
    }
}

// P4: the fate of every item after the chains are marked (kept in its scan
// word for P5) and per tile the sums of (changed, allocations); then the
// free list up to the frame's allocation bound (Alg. 8 for every rank at
// once, per word tile).
__device__ void phase_alloc_sum(const BatchDev& bt, FCtx& c, uint32_t* s_red, uint32_t* s_w, uint32_t* s_n,
                                uint32_t* s_list) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = c.I;
        const uint32_t N = c.N;
        const uint32_t i0 = stile_first(c, ipt);
        uint32_t sl[kMaxIpt], cm[kMaxIpt];
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) sl[k] = (k < ipt && i0 + k < N) ? I.live[i0 + k] : kNull;
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) cm[k] = sl[k] != kNull ? *cmd_ptr(I, sl[k]) : 0u;
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            if (sl[k] == kNull) continue;
            if (!(cm[k] & kSplitMask) && (cm[k] & kCand) && (cm[k] & kMergeGrant)) {
                s_list[atomicAdd(s_n, 1u)] = i0 + k;  // a granted merge: validated below
                continue;
            }
            const uint32_t f = leaves_of(cm[k] & kSplitMask);
            I.scan[i0 + k] = f;
            loc = padd(loc, Pair{f ? 1u : 0u, f});
        }
        __syncthreads();
        const uint32_t n = *s_n;
        for (uint32_t q = threadIdx.x; q < n; q += kFThreads) {
            const uint32_t i = s_list[q];
            const uint32_t f = alloc_fate(I, i, kCand | kMergeGrant);
            I.scan[i] = f;
            const uint32_t na = f & 7u;
            loc = padd(loc, Pair{na ? 1u : 0u, na});
        }
        Pair dummy{0, 0};
        block_sum2(loc, dummy, s_red);
        if (threadIdx.x == 0) bt.status[bt.Titems + t] = pack_pair(loc);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t wt = blockIdx.x; wt < bt.Twords; wt += gridDim.x) {
        ctx_tile(bt, bt.wtile_base, wt, bt.Twords, c);
        const Inst& I = c.I;
        const uint32_t lt = c.lt;
        const uint32_t bound = (uint32_t)min((uint64_t)c.F, (uint64_t)I.g->Mg + (uint64_t)I.g->Stot);
        const uint32_t TW = min(I.W, bt.tw);
        const uint32_t nt = I.W / TW;
        uint32_t ones_before = 0;
        for (uint32_t n = nt + lt; n > 1; n >>= 1)
            if (n & 1u) ones_before += I.sums[n - 1];
        const uint64_t zeros_before = (uint64_t)lt * TW * 32u - ones_before;
        if (zeros_before < bound) {  // block-uniform
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
            while (z && r < bound) {
                I.freel[r] = w * 32u + (uint32_t)(__ffs(z) - 1);
                ++r;
                z &= z - 1u;
            }
        }
        __syncthreads();
    }
}

// P5: allocation prefix of the tile from the tile sums (ReserveBlocks in
// ascending slot order, R7 reading); the new records' free-list indices and
// the compacted list of changed items.
__device__ void phase_alloc(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_red, Pair* s_warp) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        stats_reset(s_cnt);
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = c.I;
        const uint32_t N = c.N;
        Pair before, all;
        tile_sums(bt.status + bt.Titems, c, before, all, s_red);
        const uint32_t i0 = stile_first(c, ipt);
        uint32_t f[kMaxIpt], sl[kMaxIpt], cm[kMaxIpt];
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const bool in = k < ipt && i0 + k < N;
            f[k] = in ? I.scan[i0 + k] : 0u;
            sl[k] = in ? I.live[i0 + k] : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) cm[k] = (f[k] & 7u) ? *cmd_ptr(I, sl[k]) : 0u;
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t na = f[k] & 7u;
            loc = padd(loc, Pair{na ? 1u : 0u, na});
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        uint32_t run = before.b + tex.b, crun = before.a + tex.a;
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t na = f[k] & 7u;
            if (!na) continue;
            // the fill's record: everything it needs before its first gather
            I.chgr[crun++] = make_uint4(i0 + k, sl[k], cm[k], run);
            alloc_apply(I, i0 + k, f[k], run, s_cnt);
            run += na;
        }
        if (c.lt == c.te - c.tb - 1u && threadIdx.x == blockDim.x - 1) {
            const uint32_t bound = (uint32_t)min((uint64_t)c.F, (uint64_t)I.g->Mg + (uint64_t)I.g->Stot);
            I.g->A = run;
            I.g->C = crun;
            I.g->stats[kStAllocated] = run;
            if (run > bound) set_err(I.g, kErrOverflow);
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStSplitBis, kStMergeGroups, kStMergedBis);
        __syncthreads();
    }
}

// One changed bisector: live index i, slot s, command word and free-list
// index of its first new record (a split, or a merge group's smallest
// member, whose command word carries no split bits). Returns the number of
// unchanged neighbours relinked.
__device__ __forceinline__ uint32_t fill_item(const Inst& I, uint32_t i, uint32_t s, uint32_t cmd, uint32_t dest) {
    if (cmd & kSplitMask) {
        clear_bit(I, s);
        return fill_split(I, s, cmd, dest);
    }
    const uint4 m = I.grp[i];
    const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (ms[q] != kNull && !bad_slot(I, ms[q], kErrLink)) clear_bit(I, ms[q]);
    return fill_merge(I, dest, m);
}

// P6: FillNewBlocks + UpdateNeighbors + UpdateBitfield for the changed items,
// from the fill records. Changed items cluster in slot order and in a few
// instances of a batch, so the records of all instances are walked as one
// range, evenly over the grid: a single instance directly, a batch through
// the prefix of its instances' record counts (built by every block in
// shared memory; warps add their relink counts per instance).
__device__ void phase_fill(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_list, Pair* s_warp) {
    const uint32_t stride = gridDim.x * kFThreads;
    if (bt.B == 1) {
        stats_reset(s_cnt);
        ctx_tile(bt, bt.tile_base, 0, 1, c);  // instance 0 in shared memory
        const Inst& I = c.I;
        const uint32_t C = I.g->C;
        uint32_t relinked = 0;
        for (uint32_t q = blockIdx.x * kFThreads + threadIdx.x; q < C; q += stride) {
            const uint4 r = I.chgr[q];
            relinked += fill_item(I, r.x, r.y, r.z, r.w);
        }
        if (relinked) atomicAdd(&s_cnt[0], relinked);
        __syncthreads();
        stats_flush(s_cnt, I.g, kStRelinked);
        __syncthreads();
        return;
    }
    const int lane = threadIdx.x & 31;
    const uint32_t wfirst = blockIdx.x * kFThreads + (threadIdx.x & ~31u);
    for (uint32_t cb = 0; cb < bt.B; cb += kFBuf) {  // kFBuf instances at a time
        const uint32_t nb = min(kFBuf, bt.B - cb);
        uint32_t total = 0;
        __syncthreads();
        for (uint32_t b0 = 0; b0 < nb; b0 += kFThreads) {
            const uint32_t b = b0 + threadIdx.x;
            const uint32_t n = b < nb ? __ldcg(&bt.inst[cb + b].g->C) : 0u;
            Pair tot;
            const Pair ex = block_scan(Pair{n, 0u}, tot, s_warp);
            if (b < nb) s_list[b] = total + ex.a;
            total += tot.a;
        }
        __syncthreads();
        for (uint32_t q0 = wfirst; q0 < total; q0 += stride) {  // warp-uniform trips
            const uint32_t q = q0 + (uint32_t)lane;
            uint32_t b = kNull, relinked = 0;
            if (q < total) {
                const uint32_t lb = find_inst(s_list, nb, q);
                b = cb + lb;
                const Inst& I = bt.inst[b];
                const uint4 r = I.chgr[q - s_list[lb]];
                relinked = fill_item(I, r.x, r.y, r.z, r.w);
            }
            __syncwarp();
            const uint32_t same = __match_any_sync(0xFFFFFFFFu, b);
            const uint32_t sum = __reduce_add_sync(same, relinked);
            if (b != kNull && sum && lane == __ffs(same) - 1) atomicAdd(&bt.inst[b].g->stats[kStRelinked], sum);
        }
    }
}

// P7: SumReduction (Sec. 3.1) per word tile; the last tile of an instance to
// finish builds the levels above the tiles, in shared memory once a level
// has at most kFBuf / 2 nodes.
__device__ void phase_reduce(const BatchDev& bt, FCtx& c, uint32_t* s_buf, uint32_t* s_flag) {
    for (uint32_t wt = blockIdx.x; wt < bt.Twords; wt += gridDim.x) {
        ctx_tile(bt, bt.wtile_base, wt, bt.Twords, c);
        const Inst& I = c.I;
        const uint32_t lt = c.lt;
        const uint32_t W = I.W;
        const uint32_t TW = min(W, bt.tw);
        const uint32_t nt = W / TW;
        const uint32_t w = lt * TW + threadIdx.x;
        const bool mine = threadIdx.x < TW;
        const uint32_t pc = mine ? __popc(I.bits[w]) : 0u;
        if (mine) I.sums[W + w] = pc;
        s_buf[threadIdx.x] = pc;
        __syncthreads();
        uint32_t lvl = 1;
        for (uint32_t cnt = TW >> 1; cnt >= 1u; cnt >>= 1, ++lvl) {
            uint32_t v = 0;
            if (threadIdx.x < cnt) v = s_buf[2 * threadIdx.x] + s_buf[2 * threadIdx.x + 1];
            __syncthreads();
            if (threadIdx.x < cnt) {
                s_buf[threadIdx.x] = v;
                I.sums[((W + lt * TW) >> lvl) + threadIdx.x] = v;
            }
            __syncthreads();
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) *s_flag = (atomicAdd(&I.g->done, 1u) == nt - 1u) ? 1u : 0u;
        __syncthreads();
        if (*s_flag) {
            __threadfence();
            uint32_t n = nt;  // nodes [n, 2n) hold the tile roots
            for (; n > kFBuf / 2u; n >>= 1) {
                for (uint32_t k = threadIdx.x; k < n / 2u; k += blockDim.x)
                    I.sums[n / 2u + k] = __ldcg(I.sums + n + 2u * k) + __ldcg(I.sums + n + 2u * k + 1u);
                __syncthreads();
            }
            if (n > 1u) {
                for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) s_buf[n + k] = __ldcg(I.sums + n + k);
                __syncthreads();
                for (uint32_t m = n >> 1; m >= 1u; m >>= 1) {
                    for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
                        const uint32_t p = m + k;
                        const uint32_t v = s_buf[2u * p] + s_buf[2u * p + 1u];
                        s_buf[p] = v;
                        I.sums[p] = v;
                    }
                    __syncthreads();
                }
            }
            if (threadIdx.x == 0) {
                I.g->stats[kStLiveAfter] = __ldcg(I.sums + 1);
                I.g->done = 0;
            }
        }
        __syncthreads();
    }
}

// P8: CachePointers (Alg. 7 for every rank at once) per word tile, and, in a
// batch, the FP32 vertices of the tile's live bisectors when the frame
// exports them.
__device__ void phase_compact(const BatchDev& bt, FCtx& c, const uint32_t* s_tab, uint32_t* s_buf,
                              uint32_t* s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t wt = blockIdx.x; wt < bt.Twords; wt += gridDim.x) {
        ctx_tile(bt, bt.wtile_base, wt, bt.Twords, c);
        const Inst& I = c.I;
        const FrameP& fp = c.fp;
        const uint32_t lt = c.lt;
        const uint32_t W = I.W;
        const uint32_t TW = min(W, bt.tw);
        const uint32_t nt = W / TW;
        if (32u * TW > kFBuf) {  // block-uniform: a tile's positions must fit the staging buffer
            if (threadIdx.x == 0) set_err(I.g, kErrOverflow);
            continue;
        }
        uint32_t before = 0;
        for (uint32_t n = nt + lt; n > 1; n >>= 1)
            if (n & 1u) before += __ldcg(I.sums + n - 1);
        const uint32_t w = lt * TW + threadIdx.x;
        const uint32_t wv = threadIdx.x < TW ? __ldcg(I.bits + w) : 0u;
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
            s_buf[r++] = w * 32u + (uint32_t)(__ffs(m) - 1);
            m &= m - 1u;
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < tot; k += blockDim.x) I.live[before + k] = s_buf[k];
        if (fp.vout && bt.B > 1) {
            const uint32_t lim = fp.vcap;
            for (uint32_t k = threadIdx.x; k < tot; k += blockDim.x) {
                const uint32_t i = before + k;
                if (i < lim) vertex_item_cached(I, fp, i, s_buf[k], s_tab, fp.vout);
            }
        }
        __syncthreads();
    }
}

// Resident blocks per SM the register budget is sized for (the cooperative
// grid is that many blocks per SM).
#ifndef CBT_FRAME_MIN_BLOCKS
#define CBT_FRAME_MIN_BLOCKS 4
#endif

// P9 (single instance): the vertices of the new live list, strided over the
// whole grid (word tiles hold very different live counts). In the sphere and
// displaced forms the unchanged bisectors' vertices are copied from the
// cache P1 filled (each costs three FP64 projections or three noise sums to
// evaluate), and the new ones are listed and evaluated densely by the block
// (so that no warp idles beside one evaluating lane); otherwise the slot and
// heap ID of the next round are loaded while the current one is evaluated.
__device__ void phase_vertices(const BatchDev& bt, FCtx& c, const uint32_t* s_tab, uint32_t* s_list,
                               uint32_t* s_n) {
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    const Inst& I = c.I;
    const FrameP& fp = c.fp;
    if (!fp.vout) return;
    const uint32_t n = min(__ldcg(I.sums + 1), fp.vcap);
    const uint32_t stride = gridDim.x * kFThreads;
    if (vc_form(fp)) {
        auto evaluate = [&](uint32_t cnt) {
            for (uint32_t q = threadIdx.x; q < cnt; q += kFThreads) {
                const uint32_t i = s_list[q];
                vertex_item(I, fp, i, I.heap[I.live[i]], s_tab, fp.vout);
            }
        };
        if (threadIdx.x == 0) *s_n = 0;
        __syncthreads();
        // the cached rows of a warp's 32 consecutive rows leave through the
        // warp's staging area (the list of uncached rows uses the front of
        // s_list, the staging its back) with one coalesced store per word
        const uint32_t lane = threadIdx.x & 31u;
        float* stage = reinterpret_cast<float*>(s_list) + (kFBuf - 288u * (kFThreads / 32)) + 288u * (threadIdx.x >> 5);
        for (uint32_t base = blockIdx.x * kFThreads; base < n; base += stride) {
            const uint32_t i = base + threadIdx.x;
            bool cached = false;
            if (i < n) {
                const uint32_t s = I.live[i];
                if (*cmd_ptr(I, s) & kVcValid) {
                    const float* src = I.vc + 9ull * s;
#pragma unroll
                    for (int k = 0; k < 9; ++k) stage[9u * lane + (uint32_t)k] = src[k];
                    cached = true;
                } else {
                    s_list[atomicAdd(s_n, 1u)] = i;
                }
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, cached);
            __syncwarp();
            const uint32_t w0 = i - lane;
            float* dst = fp.vout + 9ull * w0;
            for (uint32_t w = lane; w < 288u; w += 32u)
                if ((m >> (w / 9u)) & 1u) dst[w] = stage[w];
            __syncwarp();
            __syncthreads();
            const uint32_t cnt = *s_n;
            if (cnt > kFBuf - 288u * (kFThreads / 32) - kFThreads) {  // block-uniform: keep clear of the staging
                evaluate(cnt);
                __syncthreads();
                if (threadIdx.x == 0) *s_n = 0;
                __syncthreads();
            }
        }
        evaluate(*s_n);
        return;
    }
    // warp-uniform rounds of 32 consecutive rows, staged per warp in s_list
    // (8 warps x 288 floats) and stored 16 bytes wide
    const uint32_t lane = threadIdx.x & 31u;
    float* stage = reinterpret_cast<float*>(s_list) + 288u * (threadIdx.x >> 5);
    uint32_t w0 = blockIdx.x * kFThreads + (threadIdx.x & ~31u);
    uint64_t j = w0 + lane < n ? I.heap[I.live[w0 + lane]] : 0ull;
    for (; w0 < n; w0 += stride) {
        const uint32_t i = w0 + lane;
        const uint64_t jn = i + stride < n ? I.heap[I.live[i + stride]] : 0ull;
        float r[9];
        bool ok = true;
        if (i < n) ok = vertex_eval(I, fp, j, s_tab, r);
        if (__all_sync(0xFFFFFFFFu, ok)) {
            warp_rows_out(r, stage, fp.vout, w0, min(32u, n - w0));
        } else if (i < n && ok) {  // a row the decode refused stays unwritten
            float* o = fp.vout + 9ull * i;
#pragma unroll
            for (int k = 0; k < 9; ++k) o[k] = r[k];
        }
        j = jn;
    }
}

__global__ void __launch_bounds__(kFThreads, CBT_FRAME_MIN_BLOCKS) k_frame(BatchDev bt) {
    __shared__ FCtx s_c;
    __shared__ uint32_t s_tab[64 * 9];
    __shared__ __align__(16) uint32_t s_buf[kFBuf];
    __shared__ Pair s_warp[kFThreads / 32 + 1];
    __shared__ uint32_t s_red[4 * (kFThreads / 32)];
    __shared__ uint32_t s_cnt[kBlockStats];
    __shared__ uint32_t s_w[kFThreads / 32 + 1];
    __shared__ uint32_t s_tmp[4];
    __shared__ uint32_t s_n;
    // every block reads the epoch before its first arrival; block 0 advances
    // it after the last barrier, when every block has read it
    const uint32_t epoch = ld_volatile(&bt.bg->bar_epoch);
    stamp(bt, 0);
    load_dec6(s_tab);
    if (threadIdx.x == 0) s_c.b = kNull;
    phase_prep(bt, s_warp, s_tmp);
    grid_sync(bt.bg, epoch, 1u);
    stamp(bt, 1);
    phase_classify(bt, s_c, s_tab, s_cnt, &s_n, reinterpret_cast<uint2*>(s_buf));
    grid_sync(bt.bg, epoch, 2u);
    stamp(bt, 2);
    phase_gate_sum(bt, s_c, s_cnt, s_red, &s_n, s_buf);
    grid_sync(bt.bg, epoch, 3u);
    stamp(bt, 3);
    phase_gate(bt, s_c, s_cnt, s_red, s_warp, s_tmp, &s_n, reinterpret_cast<uint2*>(s_buf));
    grid_sync(bt.bg, epoch, 4u);
    stamp(bt, 4);
    phase_alloc_sum(bt, s_c, s_red, s_w, &s_n, s_buf);
    grid_sync(bt.bg, epoch, 5u);
    stamp(bt, 5);
    phase_alloc(bt, s_c, s_cnt, s_red, s_warp);
    grid_sync(bt.bg, epoch, 6u);
    stamp(bt, 6);
    phase_fill(bt, s_c, s_cnt, s_buf, s_warp);
    grid_sync(bt.bg, epoch, 7u);
    stamp(bt, 7);
    phase_reduce(bt, s_c, s_buf, &s_tmp[0]);
    grid_sync(bt.bg, epoch, 8u);
    stamp(bt, 8);
    phase_compact(bt, s_c, s_tab, s_buf, s_w);
    if (bt.B == 1) {
        grid_sync(bt.bg, epoch, 9u);
        stamp(bt, 9);
        phase_vertices(bt, s_c, s_tab, s_buf, &s_n);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bt.timing) atomicMax(&bt.bg->t[kFramePhases], global_ns());
        if (blockIdx.x == 0) {
            bt.bg->bar_epoch = epoch + (bt.B == 1 ? kBarriers + 1u : kBarriers) * gridDim.x;
            if (ld_volatile(&bt.bg->abort))
                for (uint32_t b = 0; b < bt.B; ++b) set_err(bt.inst[b].g, kErrTimeout);
        }
    }
}

// Self-test of the bounded wait: one barrier that expects one more arrival
// than the grid has. Every wait runs out after `limit` polls, sets the abort
// word and returns; block 0 then moves the epoch past this launch's
// arrivals so that the counters stay consistent.
__global__ void __launch_bounds__(kFThreads) k_wait_selftest(BatchGlobals* bg, int limit) {
    const uint32_t epoch = ld_volatile(&bg->bar_epoch);
    grid_wait(bg, epoch + gridDim.x + 1u, limit);
    if (blockIdx.x == 0 && threadIdx.x == 0) bg->bar_epoch = epoch + gridDim.x;
}

}  // namespace

cudaError_t launch_wait_selftest(BatchGlobals* bg, int blocks, int limit, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(blocks));
    cfg.blockDim = dim3(kFThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_wait_selftest, bg, limit);
}

int frame_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_frame, kFThreads, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_frame(const BatchDev& bt, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(kFThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_frame, bt);
}

}  // namespace cbtgpu
