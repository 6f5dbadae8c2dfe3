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
                g->marks_clean = 0;
                g->freel_full = 0;
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
                               uint32_t* s_list, bool clear_marks = false) {
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
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            if (sl[k] == kNull) continue;
            // the single-instance frame's classify marked every chain; the
            // prefix gate starts from unmarked words
            const uint32_t cw = clear_marks ? atomicAnd(cmd_ptr(I, sl[k]), ~kSplitMask) : *cmd_ptr(I, sl[k]);
            if (cw & kGrpMin) s_list[atomicAdd(s_n, 1u)] = i0 + k;
        }
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
        mc[k] = (k < ipt && i0 + k < c.N) ? ((__ldcg(I.scan + i0 + k) >> 24) & kMergeCostMask) : 0u;
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
// kOne: the single-instance frame, whose descriptor is in the launch
// parameters (a copy in shared memory is reloaded after every store).
template <bool kOne = false>
__device__ void phase_gate(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_red, Pair* s_warp,
                           uint32_t* s_tmp, uint32_t* s_n, uint2* s_list, bool always_recorded = false) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = kOne ? bt.inst0 : c.I;
        const uint32_t N = c.N, F = c.F;
        const uint32_t i0 = stile_first(c, ipt);
        uint32_t sl[kMaxIpt], w[kMaxIpt];
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {  // loaded before the tile sums, which do not need them
            const bool in = k < ipt && i0 + k < N;
            sl[k] = in ? I.live[i0 + k] : kNull;
            w[k] = in ? I.scan[i0 + k] : 0u;
        }
        Pair before, all;
        tile_sums(bt.status, c, before, all, s_red);
        const uint32_t Mg = all.a <= F ? all.a : crossing_mg(bt, c, F, ipt, s_warp, s_tmp);
        if (c.lt == 0 && threadIdx.x == 0) {
            I.g->Mg = Mg;
            I.g->Stot = all.b;
        }
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) loc = padd(loc, Pair{(w[k] >> 24) & kMergeCostMask, w[k] & 0xFFFFFFu});
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        Pair run = padd(before, tex);
        uint32_t gmask = 0, nmg = 0;  // the thread's granted splits (by k), granted merges
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t mc = (w[k] >> 24) & kMergeCostMask, sc = w[k] & 0xFFFFFFu;
            run = padd(run, Pair{mc, sc});
            if (sl[k] == kNull) continue;
            const bool mgrant = mc > 0u && run.a <= F;
            if (mc) atomicOr(cmd_ptr(I, sl[k]), mgrant ? (kCand | kMergeGrant) : kCand);
            nmg += mgrant ? 1u : 0u;
            // a split wish, and only a split wish, has a nonzero split cost
            if (sc > 0u && (uint64_t)Mg + (uint64_t)run.b <= F) gmask |= 1u << k;
        }
        // the granted splits listed in thread order (bit 31 of the list's
        // live index: its chain continues past the recorded members), the
        // counts added once per warp
        Pair ntot;
        const Pair gex = block_scan(Pair{(uint32_t)__popc(gmask), nmg}, ntot, s_warp);
        uint32_t q = gex.a;
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k)
            if ((gmask >> k) & 1u) s_list[q++] = make_uint2((i0 + k) | (w[k] & kScanMore), sl[k]);
        if (threadIdx.x == 0) {
            s_cnt[0] += ntot.b;
            s_cnt[1] += ntot.a;
        }
        __syncthreads();
        const uint32_t n = ntot.a;
        // the paper's gate charges 3d + 4 without a walk (the single-instance
        // frame walks, and records, every chain that can be granted); the
        // records of four grants are loaded before their marks go out
        const bool recorded = always_recorded || c.fp.gate != 1;
        for (uint32_t q0 = threadIdx.x; q0 < n; q0 += 4u * kFThreads) {
            uint2 e[4];
            uint4 r[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t q = q0 + k * kFThreads;
                e[k] = q < n ? s_list[q] : make_uint2(0u, kNull);
                r[k] = (q < n && recorded) ? I.grp[e[k].x & ~kScanMore] : make_uint4(kNull, kNull, kNull, kNull);
            }
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                if (e[k].y == kNull) continue;
                if (r[k].x == kNull && r[k].w == kNull) {
                    chain_walk(I, e[k].y, 0, true);
                    continue;
                }
                atomicOr(cmd_ptr(I, e[k].y), kR);
                const uint32_t m[4] = {r[k].x, r[k].y, r[k].z, r[k].w};
#pragma unroll
                for (uint32_t q2 = 0; q2 < 4; ++q2)
                    if (m[q2] >> 30) atomicOr(cmd_ptr(I, m[q2] & 0x3FFFFFFFu), chain_code_bits(m[q2] >> 30));
                // a longer chain goes on from its fourth member (the walk
                // from there is the rest of the chain)
                if ((e[k].x & kScanMore) && (m[3] >> 30)) chain_walk(I, m[3] & 0x3FFFFFFFu, 0, true);
            }
        }
        __syncthreads();
        stats_flush(s_cnt, I.g, kStMergeGranted, kStSplitGranted);
        __syncthreads();
    }
}

__device__ void free_list(const BatchDev& bt, FCtx& c, uint32_t* s_w, bool all_granted,
                          const unsigned long long* tcounts = nullptr);

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
    free_list(bt, c, s_w, false);
}

// The free list (Alg. 8 for every rank at once) per word tile: the frame's
// first `bound` zero bits of the frame-start bitfield, bound = the free
// slots or, when smaller, the granted merge cost plus the requested split
// cost (all requests with `all_granted`), an upper bound of the
// allocations.
// With `tcounts` (single instance, word tiles of the frame's tile counts)
// the ones before a word tile are summed over the block from those counts
// instead of read down the sum tree one level at a time.
__device__ void free_list(const BatchDev& bt, FCtx& c, uint32_t* s_w, bool all_granted,
                          const unsigned long long* tcounts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t wt = blockIdx.x; wt < bt.Twords; wt += gridDim.x) {
        ctx_tile(bt, bt.wtile_base, wt, bt.Twords, c);
        const Inst& I = c.I;
        const uint32_t lt = c.lt;
        const uint64_t req = all_granted ? __ldcg(&I.g->rq_merge) + __ldcg(&I.g->rq_split)
                                         : (uint64_t)I.g->Mg + (uint64_t)I.g->Stot;
        const uint32_t bound = (uint32_t)min((uint64_t)c.F, req);
        const uint32_t TW = min(I.W, bt.tw);
        const uint32_t nt = I.W / TW;
        uint32_t ones_before = 0;
        if (tcounts) {
            uint32_t part = 0;
            for (uint32_t t = threadIdx.x; t < lt; t += blockDim.x) part += (uint32_t)(__ldcg(tcounts + t) >> 32);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            if (lane == 0) s_w[warp] = part;
            __syncthreads();
            for (int q = 0; q < nw; ++q) ones_before += s_w[q];
            __syncthreads();
        } else {
            for (uint32_t n = nt + lt; n > 1; n >>= 1)
                if (n & 1u) ones_before += I.sums[n - 1];
        }
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
            uint32_t* const freel = I.freel;  // in a register across the stores
            while (z && r < bound) {
                freel[r] = w * 32u + (uint32_t)(__ffs(z) - 1);
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
template <typename DM>
__device__ __forceinline__ uint32_t fill_item_dm(const Inst& I, uint32_t i, uint32_t s, uint32_t cmd, uint32_t dest,
                                                 const DM& dm) {
    if (cmd & kSplitMask) {
        dm.clear(I, s);
        return fill_split(I, s, cmd, dest, dm);
    }
    const uint4 m = I.grp[i];
    const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (ms[q] != kNull && !bad_slot(I, ms[q], kErrLink)) dm.clear(I, ms[q]);
    return fill_merge(I, dest, m, dm);
}
__device__ __forceinline__ uint32_t fill_item(const Inst& I, uint32_t i, uint32_t s, uint32_t cmd, uint32_t dest) {
    return fill_item_dm(I, i, s, cmd, dest, DestPlain{I.g->A});
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
__device__ void vertices_of(const Inst& I, const FrameP& fp, const uint32_t* s_tab, uint32_t* s_list,
                            uint32_t* s_n) {
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
    // warp-uniform rounds of 32 consecutive rows (warp-major over the grid,
    // so that rows of costly regions spread over the SMs), staged per warp in
    // s_list (8 warps x 288 floats) and stored 16 bytes wide
    const uint32_t lane = threadIdx.x & 31u;
    float* stage = reinterpret_cast<float*>(s_list) + 288u * (threadIdx.x >> 5);
    uint32_t w0 = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u;
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
__device__ void phase_vertices(const BatchDev& bt, FCtx& c, const uint32_t* s_tab, uint32_t* s_list,
                               uint32_t* s_n) {
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    vertices_of(c.I, c.fp, s_tab, s_list, s_n);
}

__global__ void __launch_bounds__(kFThreads, CBT_FRAME_MIN_BLOCKS) k_frame(BatchDev bt) {
    __shared__ FCtx s_c;
    __shared__ __align__(16) uint32_t s_tab[kDecTabWords];
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

// ===================================================== one instance, fewer phases
//
// k_frame1: the frame of a single instance (a batch of one), with the same
// results as k_frame in seven phases, or six when the frame's requests all
// fit the free slots or nothing is exported:
//   P0 prep      frame counters; the camera-relative roots; the word-tile
//                counts copied; the chain-mark words of the live slots and
//                the tile counters cleared (the marks only when the last
//                frame was not this kernel, which leaves them clear)
//   P1 classify  wishes (Sec. 3.3 GenerateCommands), in 32-item chunks dealt
//                warp-major over the grid; the items that need a walk
//                appended to the frame's walk list; per scan tile the split
//                wishes' lower-bound costs
//   P2 walks     the walk list spread evenly over the grid. A split wish's
//                chain (command form of Alg. 3) is walked, recorded and
//                marked (into the chain-mark words) unless the split wishes
//                before its scan tile and itself already cost more than the
//                free slots at their lower bounds, so that the gate denies
//                it whatever its cost. A merge wish with an even heap ID
//                walks its Alg. 4 group while it can be a merge candidate
//                with this wish its smallest member, which then records it
//                with its merge cost. Per scan tile the (merge, split) cost
//                sums, per frame their totals.
//   P3 gate      (when the totals exceed the free slots F) grants in the
//                order of the R6 reading and chain marking into the command
//                words; otherwise every request is granted and the chain-mark
//                words hold the marks
//   P4 alloc     fates, their tile-local allocation prefix (a destination
//                word holds the tile and the offset within it), the fill
//                records per tile, the bits cleared per word tile; the free
//                list only when the last frame was not this kernel
//   P5 fill      the tiles' record and allocation offsets in shared memory;
//                new records, links and bits
//   P6 final     every word tile's new count (frame-start count, clears, and
//                its share of the first A zero bits), hence the sum tree;
//                per 16-word part of a word tile (one warp), its rows of the
//                new live list and, from its zero bits, of the next frame's
//                free list (every zero bit in slot order)
//   P7 vertices  the export of the new list (FP32, fixed point, FP64
//                evaluated; sphere and displaced forms copied from the cache
//                of P1), 32 rows per warp, warp-major
// The instance descriptor and the frame parameters are read from the launch
// parameters (a copy in shared memory would be reloaded after every store
// through a generic pointer).

constexpr uint32_t kLocBits = 13, kLocMask = (1u << kLocBits) - 1u;  // offset of a new record within its tile
constexpr uint32_t kMaxTiles1 = kFBuf / 2;  // scan tiles and word tiles the shared tables hold

// Exclusive prefix sums of n <= kMaxTiles1 pairs over the block: thread x
// takes the consecutive entries [x k, x k + k), k = ceil(n / threads), loads
// them all at once (load(i) -> Pair), and after one block scan hands each
// entry's exclusive prefix to store(i, Pair); returns the total.
template <typename Load, typename Store>
__device__ __forceinline__ Pair block_table(uint32_t n, Load load, Store store, Pair* s_warp) {
    constexpr uint32_t kPer = kMaxTiles1 / kFThreads;
    const uint32_t per = (n + kFThreads - 1u) / kFThreads;
    const uint32_t i0 = threadIdx.x * per;
    Pair v[kPer];
    Pair loc{0, 0};
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        v[k] = (k < per && i0 + k < n) ? load(i0 + k) : Pair{0, 0};
        loc = padd(loc, v[k]);
    }
    Pair tot;
    Pair run = block_scan(loc, tot, s_warp);
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        if (k < per && i0 + k < n) store(i0 + k, run);
        run = padd(run, v[k]);
    }
    __syncthreads();
    return tot;
}

// A destination word (tile << kLocBits | offset) resolved through the
// tiles' allocation offsets in shared memory.
struct DestTiles {
    const uint32_t* apre;
    uint32_t A;
    __device__ __forceinline__ uint32_t operator()(uint32_t d) const {
        return apre[min(d >> kLocBits, kMaxTiles1 - 1u)] + (d & kLocMask);
    }
    __device__ __forceinline__ void set(const Inst& I, uint32_t s) const { set_bit(I, s); }
    __device__ __forceinline__ void clear(const Inst& I, uint32_t s) const { clear_bit(I, s); }
};

// Word-tile counts of the single-instance frame, one 64-bit word per word
// tile (2^tbits slots, its sum-tree node at nt + t): the node's frame-start
// value in the high half, the bits the frame clears in it in the low half.
// The bits it sets there follow from the allocation count A alone: the new
// records take the first A zero bits of the frame-start bitfield (Alg. 8).
__device__ __forceinline__ unsigned long long* tile_counts(const BatchDev& bt) {
    return bt.status + 2u * bt.Titems;
}
// Per scan tile: the split wishes' lower-bound costs (P1), then the
// allocation sums (P4).
__device__ __forceinline__ unsigned long long* wish_counts(const BatchDev& bt) { return bt.status + bt.Titems; }
// The chain marks of P2 (one word per slot; the per-step frame's list of
// changed items uses the same array).
__device__ __forceinline__ uint32_t* chain_marks(const Inst& I) { return I.chg; }
// The frame's walk list, in the fill records' array (written only in P4):
// per entry {live index | split flag << 31, slot, heap ID low, high}.
__device__ __forceinline__ uint4* walk_list_of(const Inst& I) { return I.chgr; }
constexpr uint32_t kWalkCap1 = kFBuf / 4;  // uint4 entries of the block's list
// The x word of a walk entry: the live index, bit 31 for a split wish, bit
// 30 for a split wish under a root whose halfedge has a Twin, so that it has
// one too (its chain then costs at least 4: itself and the Twin's pair,
// Alg. 3); else the chain can cost 2.
constexpr uint32_t kWalkSplit = 0x80000000u, kWalkInterior = 0x40000000u, kWalkIndex = 0x3FFFFFFFu;

// Alg. 4 group of s1 (heap ID j1, a merge wish) on the frame-start state,
// walked only while s1 can be its smallest member and every member wishes
// to merge: true when both hold, with the members (m[0] = s1, m[1] its
// sibling, m[2] the bisector across the outer half of the refinement edge,
// m[3] its sibling) and the parents' count.
static __device__ bool group_if_mergeable(const Inst& I, uint32_t s1, uint64_t j1, Group& g) {
    if (depth_of(j1, I.ch) < 1) return false;
    const uint4 r1 = I.nb[s1];
    const bool bit = j1 & 1ull;
    const uint32_t s2 = bit ? r1.z : r1.y;
    const uint32_t s3 = bit ? r1.y : r1.z;
    if (s2 == kNull || bad_slot(I, s2, kErrLink)) return false;
    if (s3 != kNull && bad_slot(I, s3, kErrLink)) return false;
    const uint64_t j2 = I.heap[s2];
    const uint32_t c2 = *cmd_ptr(I, s2);
    uint64_t j3 = 0ull;
    uint4 r3 = make_uint4(kNull, kNull, kNull, 0u);
    uint32_t c3 = 0u;
    if (s3 != kNull) {
        j3 = I.heap[s3];
        r3 = I.nb[s3];
        c3 = *cmd_ptr(I, s3);
    }
    if ((j2 >> 1) != (j1 >> 1) || j2 < j1 || !(c2 & kMergeWish)) return false;
    g.m[0] = s1;
    g.m[1] = s2;
    g.m[2] = g.m[3] = kNull;
    g.n = 2;
    g.np = 1;
    g.imin = 0;
    if (s3 != kNull) {
        // the other pair's smaller member is its even one
        if (bitlen64(j3) != bitlen64(j1) || (j3 >> 1) == (j1 >> 1) || (j3 & ~1ull) < j1 || !(c3 & kMergeWish))
            return false;
        const uint32_t s4 = bit ? r3.y : r3.z;
        if (s4 == kNull || bad_slot(I, s4, kErrLink)) return false;
        const uint64_t j4 = I.heap[s4];
        const uint32_t c4 = *cmd_ptr(I, s4);
        if ((j4 >> 1) != (j3 >> 1) || !(c4 & kMergeWish)) return false;
        g.m[2] = s3;
        g.m[3] = s4;
        g.n = 4;
        g.np = 2;
    }
    return true;
}

__device__ __forceinline__ uint32_t scan_ipt1(uint32_t N) {
    const uint32_t per_round = gridDim.x * kFThreads;
    return min(kMaxIpt, max(kMinIpt, (N + per_round - 1u) / per_round));
}

// P0 (single instance). The frame counters are set by block 0; every block
// reads the live count itself. The chain-mark words of the live slots are
// cleared unless the last frame (this kernel) left them 0.
__device__ void phase_prep1(const BatchDev& bt, uint32_t tbits) {
    const Inst& I = bt.inst0;
    const FrameP& fp = bt.fp0;
    const uint32_t N = __ldcg(I.sums + 1);
    const uint32_t nt = I.cap >> tbits;
    const uint32_t ipt = scan_ipt1(N), S = ipt * kFThreads, T = (N + S - 1u) / S;
    const uint32_t gt = blockIdx.x * kFThreads + threadIdx.x, stride = gridDim.x * kFThreads;
    unsigned long long* tc = tile_counts(bt);
    for (uint32_t t = gt; t < nt; t += stride) tc[t] = (unsigned long long)__ldcg(I.sums + nt + t) << 32;
    for (uint32_t t = gt; t < T; t += stride) {
        bt.status[t] = 0ull;
        wish_counts(bt)[t] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Globals* g = I.g;
        g->N = N;
        g->F = I.cap - N;
        g->A = 0;
        g->Mg = 0;
        g->Stot = 0;
        g->C = 0;
        g->done = 0;
        g->ntiles = (N + kTileItems - 1u) / kTileItems;
        g->nstiles = T;
        for (int k = 0; k < kStCount; ++k) g->stats[k] = 0;
        g->stats[kStLiveBefore] = N;
        g->stats[kStFreeBefore] = I.cap - N;
        g->stats[kStFrame] = fp.frame;
        g->rq_merge = 0;
        g->rq_split = 0;
        g->nwalk = 0;
        pc_generation(g, fp);
        if (bt.nout) bt.nout[0] = N;
        bt.tile_base[0] = 0;
        bt.tile_base[1] = g->ntiles;
        bt.stile_base[0] = 0;
        bt.stile_base[1] = T;
        bt.bg->total_tiles = g->ntiles;
        bt.bg->total_stiles = T;
        bt.bg->scan_ipt = ipt;
        bt.bg->live_total = N;
        bt.bg->t[kFramePhases] = 0;
    }
    const uint32_t nw = gridDim.x * (kFThreads / 32), wid = blockIdx.x * (kFThreads / 32) + threadIdx.x / 32u;
    const uint32_t per = min(kRelRange, ((bt.Trel + nw - 1u) / nw + 31u) & ~31u);
    for (uint32_t e = wid * per; e < bt.Trel; e += nw * per) rel_range(bt, e, min(bt.Trel, e + per));
    uint32_t* marks = chain_marks(I);
    if (__ldcg(&I.g->marks_clean)) return;  // the last frame left them 0
    for (uint32_t i0 = gt; i0 < N; i0 += 4u * stride) {
        uint32_t sl[4];
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) sl[k] = i0 + k * stride < N ? __ldcg(I.live + i0 + k * stride) : kNull;
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k)
            if (sl[k] != kNull) marks[sl[k]] = 0u;
    }
}

// P1 (single instance): the live list strided over the whole grid, the slot
// and heap ID of the next rounds loaded while the current item is classified.
// Walk entries (live index | split flag << 31, slot, heap ID) are listed per
// warp and flushed to the frame's walk list; split wishes are counted per
// scan tile (warp-aggregated, consecutive live indices share a tile).
// A warp's walk buffer (kWarpWalks entries of the block's shared list) out
// to the frame's walk list: one atomic for the range, then a coalesced copy.
constexpr uint32_t kWarpWalks = kWalkCap1 / (kFThreads / 32);
__device__ __forceinline__ void warp_walks_out(const Inst& I, const uint4* s_wl, uint32_t n) {
    if (n == 0u) return;  // warp-uniform
    uint32_t base = 0;
    if ((threadIdx.x & 31u) == 0u) base = atomicAdd(&I.g->nwalk, n);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    uint4* wl = walk_list_of(I);
    for (uint32_t q = threadIdx.x & 31u; q < n; q += 32u) wl[base + q] = s_wl[q];
    __syncwarp();
}

__device__ void phase_classify1(const BatchDev& bt, FCtx& c, uint32_t* s_tab, uint32_t* s_cnt, uint4* s_list) {
    stats_reset(s_cnt);
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    const Inst& I = bt.inst0;
    const FrameP& fp = bt.fp0;
    const uint32_t N = c.N;
    const uint32_t S = kFThreads * bt.bg->scan_ipt;
    unsigned long long* wc = wish_counts(bt);
    const uint64_t key = splitmix64(((uint64_t)fp.seed << 32) | (uint64_t)fp.frame);
    const bool cache = vc_form(fp) && fp.vout;
    const uint32_t lane = threadIdx.x & 31u;
    uint4* s_wl = s_list + kWarpWalks * (threadIdx.x >> 5);  // the warp's walk buffer
    uint32_t nwl = 0;                                           // its entries (warp-uniform)
    // 32-item chunks, warp-major (chunk c to warp c mod (warps of the grid),
    // warps numbered across the blocks first), so that the costly parts of
    // the list (in slot order, i.e. clustered in space) spread over the SMs;
    // the warps run independently (no block barrier in the loop)
    const uint32_t stride = gridDim.x * kFThreads;
    uint32_t i = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u + lane;
    uint32_t sa = i < N ? I.live[i] : 0u;
    uint64_t ja = i < N ? I.heap[sa] : 0ull;
    uint32_t sb = i + stride < N ? I.live[i + stride] : 0u;
    for (; i - lane < N; i += stride) {  // warp-uniform
        const uint32_t sc = i + 2u * stride < N ? I.live[i + 2u * stride] : 0u;
        const uint64_t jb = i + stride < N ? I.heap[sb] : 0ull;
        bool split = false, walk = false, interior = false;
        if (i < N) {
            const uint32_t cmd = classify_item(I, fp, key, i, sa, ja, s_tab, s_cnt, cache);
            split = (cmd & kSplitWish) != 0u;
            walk = split || ((cmd & kMergeWish) && !(cmd & kHeapOdd));
            // every bisector under a root whose halfedge has a Twin has one
            // (its refinement edge is inside the root triangle, on an edge
            // to the face's centroid, or on that halfedge)
            const int d = depth_of(ja, I.ch);
            const uint32_t h = d >= 0 ? (uint32_t)((ja >> d) - (1ull << I.ch)) : kNull;
            interior = split && h < I.H && !((__ldg(I.rbnd + (h >> 5)) >> (h & 31u)) & 1u);
        }
        const unsigned wm = __ballot_sync(0xFFFFFFFFu, walk);
        if (walk)
            s_wl[nwl + __popc(wm & ((1u << lane) - 1u))] =
                make_uint4(i | (split ? kWalkSplit : 0u) | (interior ? kWalkInterior : 0u), sa, (uint32_t)ja,
                           (uint32_t)(ja >> 32));
        nwl += __popc(wm);
        {  // the split wishes' lower-bound costs per scan tile
            const uint32_t t = i / S;
            const unsigned m = __match_any_sync(0xFFFFFFFFu, i < N ? t : kNull);
            const uint32_t lb = __reduce_add_sync(m, split ? (interior ? 4u : 2u) : 0u);
            if (lb && lane == (uint32_t)(__ffs(m) - 1)) atomicAdd(&wc[t], (unsigned long long)lb);
        }
        sa = sb;
        ja = jb;
        sb = sc;
        __syncwarp();
        if (nwl > kWarpWalks - 32u) {  // warp-uniform: room for the next round
            warp_walks_out(I, s_wl, nwl);
            nwl = 0;
        }
    }
    __syncwarp();
    warp_walks_out(I, s_wl, nwl);
    __syncthreads();
    stats_flush(s_cnt, I.g, kStSplitWishes);
    __syncthreads();
}

// P2 (single instance): the frame's walk list over the whole grid. s_wpre
// (shared) gets the split wishes' lower-bound costs before each scan tile
// (4 with a Twin, else 2). A block first takes
// its share of the entries and settles the splits past the bound below; the
// walks left are queued and spread evenly over the block's threads. Per
// entry:
//   - a split wish: unless those costs plus its own bound exceed F, its
//     chain is walked on the frame-start links, checked, its first members
//     recorded in grp[i] and marked in the chain-mark words; its scan word
//     the chain's allocation count (or 3d + 4 under the paper's gate, set by
//     classify); past that bound the gate denies it whatever its cost, and
//     its bound stands in;
//   - a merge wish with an even heap ID: its Alg. 4 group, walked while the
//     wish can be its smallest member and every member wishes to merge (a
//     merge candidate); then it records the members and kGrpMin, and the
//     merge cost (parents, or 2 under the paper's gate) in the top byte of
//     its scan word. A group that is no candidate can never merge.
// The costs go to their scan tile's (merge, split) sums in status[t] and to
// the frame's totals.
__device__ void phase_walks1(const BatchDev& bt, FCtx& c, uint32_t* s_cnt, uint32_t* s_buf, Pair* s_warp,
                             uint32_t* s_tmp, uint32_t* s_n1) {
    stats_reset(s_cnt);
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    const Inst& I = bt.inst0;
    const FrameP& fp = bt.fp0;
    const uint32_t T = bt.bg->total_stiles, S = kFThreads * bt.bg->scan_ipt;
    if (threadIdx.x == 0) s_tmp[0] = s_tmp[1] = s_tmp[2] = 0;
    if (T > kMaxTiles1) {  // the host keeps pools within the tables
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(I.g, kErrOverflow);
        __syncthreads();
        return;
    }
    uint32_t* s_wpre = s_buf;
    const unsigned long long* wc = wish_counts(bt);
    const uint32_t n = __ldcg(&I.g->nwalk), F = c.F;
    const uint4* wl = walk_list_of(I);
    // a warp takes 32 consecutive entries per round (neighbouring entries
    // walk neighbouring records, which its L1 then holds), warp-major over
    // the grid so that every SM gets its share of a short list; a thread
    // loads the entries of four rounds together, the first four before the
    // table of split wishes below is built
    const uint32_t stride = gridDim.x * kFThreads;
    const uint32_t mine = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u + (threadIdx.x & 31u);
    uint32_t qq[4];
    uint4 e[4];
    auto fetch = [&](uint32_t c0) {
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            const uint32_t q = c0 + k * stride + mine;
            qq[k] = q < n ? q : kNull;
            e[k] = qq[k] != kNull ? wl[qq[k]] : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    fetch(0u);
    block_table(T, [&](uint32_t t) { return Pair{(uint32_t)__ldcg(wc + t), 0u}; },
                [&](uint32_t t, Pair ex) { s_wpre[t] = ex.a; }, s_warp);
    uint32_t* marks = chain_marks(I);
    uint32_t* s_q = s_buf + kMaxTiles1;  // list indices of the block's walks to do
    constexpr uint32_t kQCap = kFBuf - kMaxTiles1;
    // a split's cost and a group's merge cost, added to their scan tile's
    // sums (one atomic per tile present among the active lanes)
    auto account = [&](uint32_t t, uint32_t mc, uint32_t sc) {
        const unsigned act = __activemask();
        const unsigned m = __match_any_sync(act, t);
        const uint32_t smc = __reduce_add_sync(m, mc), ssc = __reduce_add_sync(m, sc);
        if (t != kNull && (threadIdx.x & 31u) == (uint32_t)(__ffs(m) - 1) && (smc | ssc))
            atomicAdd(&bt.status[min(t, T - 1u)], ((unsigned long long)smc << 32) | ssc);
        if (mc) atomicAdd(&s_tmp[0], mc);
        if (sc) atomicAdd(&s_tmp[1], sc);
        count_stat(s_cnt, 0, mc != 0u);
    };
    // the queued walks over the block's threads, each taking the next one
    // when its last is done (chain lengths differ; s_tmp[2] counts them out)
    auto walk_queue = [&](uint32_t cnt) {
        for (uint32_t k = atomicAdd(&s_tmp[2], 1u); k < cnt; k = atomicAdd(&s_tmp[2], 1u)) {
            const uint32_t q = s_q[k];
            const uint4 e = wl[q];
            const uint32_t i = e.x & kWalkIndex, s = e.y;
            const uint64_t j = (uint64_t)e.z | ((uint64_t)e.w << 32);
            uint32_t mc = 0, sc = 0;
            if (e.x & kWalkSplit) {
                const int d = depth_of(j, I.ch);
                uint4 rec;
                bool more;
                const uint32_t cost = chain_walk(I, s, d, true, &rec, true, marks, &more);
                I.grp[i] = rec;
                sc = fp.gate == 1 ? 3u * (uint32_t)d + 4u : cost;
                I.scan[i] = sc | (more ? kScanMore : 0u);
            } else {
                Group g;
                if (group_if_mergeable(I, s, j, g)) {
                    I.grp[i] = make_uint4(g.m[0], g.m[1], g.m[2], g.m[3]);
                    atomicOr(cmd_ptr(I, s), kGrpMin);
                    mc = fp.gate == 1 ? 2u : (uint32_t)g.np;
                    I.scan[i] = mc << 24;
                }
            }
            account(i / S, mc, sc);
        }
    };
    if (threadIdx.x == 0) *s_n1 = 0;
    __syncthreads();
    for (uint32_t c0 = 0; c0 + blockIdx.x * 32u < n; c0 += 4u * stride) {  // block-uniform
        if (c0) fetch(c0);
#pragma unroll
        for (uint32_t k = 0; k < 4; ++k) {
            if (qq[k] == kNull) continue;
            const uint32_t i = e[k].x & kWalkIndex;
            const uint32_t t = i / S;
            // a split is denied whatever its cost when the lower bounds of
            // the split wishes before its scan tile and of its own exceed F
            const bool skip =
                (e[k].x & kWalkSplit) && (unsigned long long)s_wpre[min(t, T - 1u)] +
                                                 ((e[k].x & kWalkInterior) ? 4ull : 2ull) > (unsigned long long)F;
            if (skip) {
                // its bound stands in for its cost: every split after it in
                // the gate's order is then denied on these costs as on the
                // true ones, and the requested total still exceeds F
                const uint64_t j = (uint64_t)e[k].z | ((uint64_t)e[k].w << 32);
                const uint32_t sc = fp.gate == 1 ? 3u * (uint32_t)depth_of(j, I.ch) + 4u
                                                 : ((e[k].x & kWalkInterior) ? 4u : 2u);
                if (fp.gate != 1) I.scan[i] = sc;
                account(t, 0u, sc);
            } else {
                s_q[atomicAdd(s_n1, 1u)] = qq[k];
            }
        }
        __syncthreads();
        const uint32_t cnt = *s_n1;
        __syncthreads();
        if (cnt > kQCap - 4u * kFThreads) {  // block-uniform
            walk_queue(cnt);
            __syncthreads();
            if (threadIdx.x == 0) *s_n1 = s_tmp[2] = 0;
            __syncthreads();
        }
    }
    walk_queue(*s_n1);
    __syncthreads();
    stats_flush(s_cnt, I.g, kStMergeCand);
    if (threadIdx.x == 0) {
        if (s_tmp[0]) atomicAdd(&I.g->rq_merge, (unsigned long long)s_tmp[0]);
        if (s_tmp[1]) atomicAdd(&I.g->rq_split, (unsigned long long)s_tmp[1]);
    }
    __syncthreads();
}

// Fate of live index i that charges its group (kGrpMin) when every request
// is granted: the group's parent count (1 or 2) and bit 3 when every member
// wishes to merge and none is marked by a chain (marks in the command words
// or, with `marks`, in those words).
__device__ __forceinline__ uint32_t fate_group_granted(const Inst& I, uint32_t i, const uint32_t* marks) {
    const uint4 m = I.grp[i];
    const uint32_t ms[3] = {m.y, m.z, m.w};
    uint32_t c[3];
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const bool b = ms[q] != kNull && bad_slot(I, ms[q], kErrLink);
        bad = bad || b;
        c[q] = (ms[q] != kNull && !b) ? (*cmd_ptr(I, ms[q]) | marks[ms[q]]) : kMergeWish;
    }
    const bool all = !bad && (c[0] & c[1] & c[2] & kMergeWish);
    const bool ok = all && !((c[0] | c[1] | c[2]) & kSplitMask);
    return ok ? ((m.z == kNull ? 1u : 2u) | 8u) : 0u;
}

// P4 (single instance): per scan tile the fate of every item (allocation
// count, bit 3 for a merging group), the tile-local exclusive prefix of
// (changed, allocations), the fill records in the tile's region of chgr
// (tile t at t S), destination words (t << kLocBits | offset) and merged
// marks; the tile's totals go to status[Titems + t] for the fill. When every
// request was granted, the chain marks are ORed into the command words (the
// fill reads them there). Then the free list. Group validations run from a
// list (dependent loads), their fates returned through shared memory.
__device__ void phase_alloc1(const BatchDev& bt, FCtx& c, bool all_granted, bool carried, uint32_t tbits,
                             uint32_t* s_cnt, Pair* s_warp, uint32_t* s_w, uint32_t* s_n, uint32_t* s_buf) {
    const uint32_t T = bt.bg->total_stiles, ipt = bt.bg->scan_ipt;
    const uint32_t S = kFThreads * ipt;
    uint32_t* s_list = s_buf;          // local item indices to validate
    uint32_t* s_fate = s_buf + kFBuf / 2;  // their fates, by local item index
    __shared__ uint32_t s_first;
    if (T > kMaxTiles1 || S > kFBuf / 2) {  // the host keeps pools within the tables
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(bt.inst0.g, kErrOverflow);
        return;
    }
    if (all_granted && blockIdx.x == 0 && threadIdx.x == 0) {
        Globals* g = bt.inst0.g;
        g->stats[kStSplitGranted] = __ldcg(&g->stats[kStSplitWishes]);
        g->stats[kStMergeGranted] = __ldcg(&g->stats[kStMergeCand]);
    }
    for (uint32_t t = blockIdx.x; t < T; t += gridDim.x) {
        if (threadIdx.x == 0) *s_n = 0;
        stats_reset(s_cnt);
        ctx_tile(bt, bt.stile_base, t, T, c);
        const Inst& I = bt.inst0;
        const uint32_t N = c.N;
        const uint32_t* marks = chain_marks(I);
        const uint32_t ts = c.lt * S;  // the tile's first live index
        const uint32_t e0 = threadIdx.x * ipt, i0 = ts + e0;
        uint32_t sl[kMaxIpt], cm[kMaxIpt], f[kMaxIpt];
        {  // slots and command words loaded coalesced (item ts + k 256 + tid)
           // through shared memory, then taken ipt consecutive per thread
            uint32_t* s_sl = s_buf;
            uint32_t* s_cm = s_buf + kFBuf / 2;
            uint32_t a[kMaxIpt];
#pragma unroll
            for (uint32_t k = 0; k < kMaxIpt; ++k) {
                const uint32_t e = k * kFThreads + threadIdx.x;
                a[k] = (k < ipt && ts + e < N) ? I.live[ts + e] : kNull;
            }
#pragma unroll
            for (uint32_t k = 0; k < kMaxIpt; ++k) {
                if (k >= ipt) continue;
                uint32_t m = a[k] != kNull ? *cmd_ptr(I, a[k]) : 0u;
                if (all_granted && a[k] != kNull) {
                    const uint32_t mk = marks[a[k]];
                    if (mk) {
                        m |= mk;
                        atomicOr(cmd_ptr(I, a[k]), mk);
                    }
                }
                s_sl[k * kFThreads + threadIdx.x] = a[k];
                s_cm[k * kFThreads + threadIdx.x] = m;
            }
            __syncthreads();
#pragma unroll
            for (uint32_t k = 0; k < kMaxIpt; ++k) {
                sl[k] = k < ipt ? s_sl[e0 + k] : kNull;
                cm[k] = k < ipt ? s_cm[e0 + k] : 0u;
            }
            if (threadIdx.x == 0) s_first = s_sl[0];  // the tile's first slot
            __syncthreads();  // s_buf is the lists' below
        }
        // groups to validate: when every request is granted, every recorded
        // group without split bits at its charged member; else the granted
        // candidates without split bits
        bool lst[kMaxIpt];
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            f[k] = leaves_of(cm[k] & kSplitMask);
            lst[k] = sl[k] != kNull && !(cm[k] & kSplitMask) &&
                     (all_granted ? (cm[k] & kGrpMin) != 0u : ((cm[k] & kCand) && (cm[k] & kMergeGrant)));
            if (lst[k]) s_list[atomicAdd(s_n, 1u)] = e0 + k;
        }
        __syncthreads();
        const uint32_t n = *s_n;
        for (uint32_t q = threadIdx.x; q < n; q += kFThreads) {
            const uint32_t e = s_list[q];
            const uint32_t i = c.lt * S + e;
            s_fate[e] = all_granted ? fate_group_granted(I, i, marks) : alloc_fate(I, i, kCand | kMergeGrant);
        }
        __syncthreads();
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k)
            if (lst[k]) f[k] = s_fate[e0 + k];
        Pair loc{0, 0};
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t na = f[k] & 7u;
            loc = padd(loc, Pair{na ? 1u : 0u, na});
        }
        Pair tot;
        const Pair ex = block_scan(loc, tot, s_warp);
        if (threadIdx.x == 0) bt.status[bt.Titems + t] = pack_pair(tot);
        // the bits this tile's changed items clear, per word tile: a block
        // histogram over the word tiles from the one holding the tile's first
        // slot (slots ascend with the live index); others go straight out
        uint32_t* s_hist = s_buf + kFBuf / 2;
        uint32_t* s_ml = s_buf;  // the tile's merges: local index << 13 | allocation offset
        const uint32_t hbase = (I.cap + s_first) >> tbits, nt = I.cap >> tbits;
        unsigned long long* tc = tile_counts(bt);
        s_hist[threadIdx.x] = 0u;
        if (threadIdx.x == 0) *s_n = 0;
        __syncthreads();
        auto cleared = [&](uint32_t slot) {
            const uint32_t node = (I.cap + slot) >> tbits;
            if (node - hbase < (uint32_t)kFThreads)
                atomicAdd(&s_hist[node - hbase], 1u);
            else if (node - nt < nt)
                atomicAdd(&tc[node - nt], 1ull);
        };
        uint32_t crun = ex.a, arun = ex.b;
#pragma unroll
        for (uint32_t k = 0; k < kMaxIpt; ++k) {
            const uint32_t na = f[k] & 7u;
            if (!na) continue;
            const uint32_t dw = (t << kLocBits) | arun;
            I.chgr[t * S + crun] = make_uint4(i0 + k, sl[k], cm[k], dw);
            // alloc_apply, with the clears counted; a merge is listed and
            // applied below, one per thread
            if (!(f[k] & 8u)) {
                *dest_ptr(I, sl[k]) = dw;
                count_stat(s_cnt, 0, true);
                cleared(sl[k]);
            } else {
                s_ml[atomicAdd(s_n, 1u)] = ((e0 + k) << kLocBits) | arun;
            }
            ++crun;
            arun += na;
        }
        __syncthreads();
        const uint32_t nm = *s_n;
        for (uint32_t q = threadIdx.x; q < nm; q += kFThreads) {
            const uint32_t e = s_ml[q] >> kLocBits, dw = (t << kLocBits) | (s_ml[q] & kLocMask);
            const uint4 m = I.grp[ts + e];
            const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (ms[r] == kNull || bad_slot(I, ms[r], kErrLink)) continue;
                atomicOr(cmd_ptr(I, ms[r]), kMerged);
                *dest_ptr(I, ms[r]) = dw + (r < 2 ? 0u : 1u);
                cleared(ms[r]);
            }
            atomicAdd(&s_cnt[2], m.z == kNull ? 2u : 4u);
            count_stat(s_cnt, 1, true);
        }
        __syncthreads();
        if (s_hist[threadIdx.x] && hbase + threadIdx.x - nt < nt)
            atomicAdd(&tc[hbase + threadIdx.x - nt], (unsigned long long)s_hist[threadIdx.x]);
        stats_flush(s_cnt, I.g, kStSplitBis, kStMergeGroups, kStMergedBis);
        __syncthreads();
    }
    // the last frame's final phase listed every zero bit of this frame's
    // starting bitfield, unless another form of the frame ran since
    if (!carried) free_list(bt, c, s_w, all_granted, tile_counts(bt));
}

// P5 (single instance): every block scans the tiles' (changed, allocation)
// totals into shared memory; the changed records of the frame, one range
// strided evenly over the grid, are then filled with their destinations
// resolved through the allocation offsets. The records are FillNewBlocks +
// UpdateNeighbors + UpdateBitfield, the bit changes also moving the word
// tiles' sum-tree nodes.
__device__ void phase_fill1(const BatchDev& bt, FCtx& c, bool all_granted, uint32_t* s_cnt, uint32_t* s_buf,
                            Pair* s_warp) {
    stats_reset(s_cnt);
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    const Inst& I = bt.inst0;
    const uint32_t T = bt.bg->total_stiles, S = kFThreads * bt.bg->scan_ipt;
    uint32_t* s_cpre = s_buf;
    uint32_t* s_apre = s_buf + kMaxTiles1;
    if (T > kMaxTiles1) {  // alloc has set the error word
        __syncthreads();
        return;
    }
    const Pair carry = block_table(
        T, [&](uint32_t t) { return unpack_pair(__ldcg(bt.status + bt.Titems + t)); },
        [&](uint32_t t, Pair ex) {
            s_cpre[t] = ex.a;
            s_apre[t] = ex.b;
        },
        s_warp);
    const uint32_t C = carry.a;
    const uint64_t req = all_granted ? __ldcg(&I.g->rq_merge) + __ldcg(&I.g->rq_split)
                                     : (uint64_t)I.g->Mg + (uint64_t)I.g->Stot;
    const uint32_t bound = (uint32_t)min((uint64_t)c.F, req);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        I.g->A = carry.b;
        I.g->C = C;
        I.g->stats[kStAllocated] = carry.b;
        if (carry.b > bound) set_err(I.g, kErrOverflow);
    }
    const DestTiles dm{s_apre, min(carry.b, bound)};
    uint32_t relinked = 0;
    // 32 records per warp, warp-major over the grid: with fewer records than
    // threads, every SM still gets its share
    for (uint32_t q = ((threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32u + (threadIdx.x & 31u); q < C;
         q += gridDim.x * kFThreads) {
        uint32_t lo = 0, hi = T;  // the last tile whose first record is at or before q
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_cpre[mid] <= q)
                lo = mid + 1u;
            else
                hi = mid;
        }
        const uint32_t t = lo - 1u;
        const uint4 r = I.chgr[t * S + (q - s_cpre[t])];
        relinked += fill_item_dm(I, r.x, r.y, r.z, dm(r.w), dm);
    }
    if (relinked) atomicAdd(&s_cnt[0], relinked);
    __syncthreads();
    stats_flush(s_cnt, I.g, kStRelinked);
    __syncthreads();
}

// P6 (single instance). Every block computes each word tile's new count
// from the tile counts of the frame (no bitfield read) and scans them into
// shared memory: the new live count and each tile's first row. Block 0
// writes the nodes above the tiles as differences of that scan; a warp per
// word tile rebuilds the tile's node and the nodes below it from its words
// (the count checked against the scan) and writes the tile's rows of the new
// live list. The vertices follow in their own phase, over the whole list.
__device__ void phase_final1(const BatchDev& bt, FCtx& c, uint32_t* s_buf, Pair* s_warp, uint32_t* s_tmp,
                             uint32_t tbits, bool carried) {
    ctx_tile(bt, bt.tile_base, 0, 1, c);
    const Inst& I = bt.inst0;
    const uint32_t W = I.W, TW = min(W, bt.tw), nt = I.cap >> tbits;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t* s_tpre = s_buf;
    if (nt > kMaxTiles1 || TW > 64u) {  // the host keeps pools within the tables
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(I.g, kErrOverflow);
        return;
    }
    // each word tile's new count: frame-start count - cleared + set, the set
    // ones being the tile's share of the first A zero bits
    const unsigned long long* tc = tile_counts(bt);
    const uint32_t A = __ldcg(&I.g->A), TS = 1u << tbits;
    // the ones before each tile at frame start: kept by the last frame's
    // final phase (`carried`: the last frame was this kernel) in the buffer of
    // this frame's parity, else scanned here from the tile counts (into
    // s_tpre); then the new counts from them, scanned in place, and kept for
    // the next frame in the other buffer
    const uint32_t par = bt.fp0.frame & 1u;
    const uint32_t* tpre_in = bt.tpre + par * bt.Twords;
    uint32_t* tpre_out = bt.tpre + (par ^ 1u) * bt.Twords;
    if (!carried)
        block_table(nt, [&](uint32_t t) { return Pair{(uint32_t)(__ldcg(tc + t) >> 32), 0u}; },
                    [&](uint32_t t, Pair ex) { s_tpre[t] = ex.a; }, s_warp);
    const Pair tot = block_table(
        nt,
        [&](uint32_t t) {
            const unsigned long long w = __ldcg(tc + t);
            const uint32_t old = (uint32_t)(w >> 32), clr = (uint32_t)w;
            const uint32_t before = carried ? __ldcg(tpre_in + t) : s_tpre[t];
            const long long zb = (long long)t * TS - before;  // zero bits before the tile at frame start
            const long long set = min(max((long long)A - zb, 0ll), (long long)(TS - old));
            return Pair{old - clr + (uint32_t)set, 0u};
        },
        [&](uint32_t t, Pair ex) { s_tpre[t] = ex.a; }, s_warp);
    for (uint32_t t = blockIdx.x + threadIdx.x * gridDim.x; t < nt; t += kFThreads * gridDim.x) tpre_out[t] = s_tpre[t];
    if (threadIdx.x == 0) s_tmp[0] = 0;
    __syncthreads();
    const uint32_t Nn = tot.a;
    if (blockIdx.x == 0) {
        // node m (1 <= m < nt) covers tile nodes [m 2^k, (m + 1) 2^k) at 2^k
        // tiles per node of its level
        const int lnt = 31 - __clz((int)nt);
        for (uint32_t m = 1u + threadIdx.x; m < nt; m += kFThreads) {
            const int k = lnt - (31 - __clz((int)m));
            const uint32_t a = (m << k) - nt, b = ((m + 1u) << k) - nt;
            I.sums[m] = (b < nt ? s_tpre[b] : Nn) - s_tpre[a];
        }
        if (threadIdx.x == 0) {
            I.g->stats[kStLiveAfter] = Nn;
            if (nt == 1u) I.sums[1] = Nn;
        }
    }
    // word tiles (TW <= 64 words: lane holds words lane and 32 + lane): the
    // levels below the tile node (whose value, from the scan, is checked
    // against the words' popcounts), then the tile's slice of the new live
    // list (Alg. 7 for every index, in slot order): word by word, lane b
    // tests bit b and the set ones take consecutive rows, so every store of
    // the list is one contiguous run
    // the instance's fields in registers (a store through a generic pointer
    // would otherwise make the compiler reload them from shared memory)
    uint32_t* const marks = chain_marks(I);
    uint32_t* const live = I.live;
    uint32_t* const freel = I.freel;
    uint32_t* const sums = I.sums;
    const uint32_t* const bits = I.bits;
    const uint32_t cap = I.cap;
    const uint32_t vmask = cap < 32u ? (1u << cap) - 1u : 0xFFFFFFFFu;  // the slots of a word
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // read by the next frame
        I.g->marks_clean = 1u;
        I.g->freel_full = 1u;
    }
    const uint32_t nwarps = gridDim.x * (kFThreads / 32u);
    const uint32_t lt_mask = (1u << lane) - 1u;
    // a word tile in Q parts of UW words, one warp each (warp-major over the
    // grid); every part reads the tile's words for its prefix, the first
    // also rebuilds the tile's levels of the sum tree
    const uint32_t Q = TW >= 64u ? 4u : TW >= 32u ? 2u : 1u, UW = TW / Q;
    for (uint32_t u = warp * gridDim.x + blockIdx.x; u < nt * Q; u += nwarps) {
        const uint32_t wt = u / Q, q = u % Q;
        const uint32_t w0 = wt * TW + lane, w1 = w0 + 32u;
        const uint32_t x0 = lane < TW ? __ldcg(bits + w0) : 0u;
        const uint32_t x1 = 32u + lane < TW ? __ldcg(bits + w1) : 0u;
        const uint32_t r0 = s_tpre[wt];
        uint32_t v0 = __popc(x0), v1 = __popc(x1);
        // ones in the tile before the part's first word q UW
        const uint32_t pre = __reduce_add_sync(0xFFFFFFFFu, (lane < q * UW ? v0 : 0u) + (32u + lane < q * UW ? v1 : 0u));
        if (q == 0u) {
            if (TW > 1u) {
                if (lane < TW) sums[W + w0] = v0;
                if (32u + lane < TW) sums[W + w1] = v1;
            }
#pragma unroll
            for (uint32_t L = 1; L <= 5; ++L) {
                v0 += __shfl_down_sync(0xFFFFFFFFu, v0, 1u << (L - 1u));
                v1 += __shfl_down_sync(0xFFFFFFFFu, v1, 1u << (L - 1u));
                if ((1u << L) < TW && (lane & ((1u << L) - 1u)) == 0u) {
                    if (lane < TW) sums[(W + w0) >> L] = v0;
                    if (32u + lane < TW) sums[(W + w1) >> L] = v1;
                }
            }
            const uint32_t half0 = __shfl_sync(0xFFFFFFFFu, v0, 0), half1 = __shfl_sync(0xFFFFFFFFu, v1, 0);
            const uint32_t node = (wt + 1u < nt ? s_tpre[wt + 1u] : Nn) - r0;
            if (lane == 0) {
                if (half0 + half1 != node) set_err(I.g, kErrLink);
                if (nt > 1u) sums[nt + wt] = node;  // (a single tile's node is the root, written above)
            }
        }
        // the part's rows of the live list and, from its zero bits, of the
        // next frame's free list (Alg. 8 for every rank; every earlier tile
        // holds 2^tbits slots)
        uint32_t row = r0 + pre, zrow = wt * TS - r0 + (q * UW * 32u - pre);
#pragma unroll 4
        for (uint32_t i = q * UW; i < (q + 1u) * UW; ++i) {
            const uint32_t x = __shfl_sync(0xFFFFFFFFu, i < 32u ? x0 : x1, i & 31u);
            const uint32_t z = ~x & vmask;
            const uint32_t sl = (wt * TW + i) * 32u + lane;
            const uint32_t r = row + __popc(x & lt_mask), zr = zrow + __popc(z & lt_mask);
            if (((x >> lane) & 1u) && r < cap) {
                live[r] = sl;
                marks[sl] = 0u;  // for the next frame's chain marks
            } else if (((z >> lane) & 1u) && zr < cap) {
                freel[zr] = sl;
            }
            row += __popc(x);
            zrow += __popc(z);
        }
    }
}

__global__ void __launch_bounds__(kFThreads, CBT_FRAME_MIN_BLOCKS) k_frame1(BatchDev bt, uint32_t tbits) {
    __shared__ FCtx s_c;
    __shared__ __align__(16) uint32_t s_tab[kDecTabWords];
    __shared__ __align__(16) uint32_t s_buf[kFBuf];
    __shared__ Pair s_warp[kFThreads / 32 + 1];
    __shared__ uint32_t s_red[4 * (kFThreads / 32)];
    __shared__ uint32_t s_cnt[kBlockStats];
    __shared__ uint32_t s_w[kFThreads / 32 + 1];
    __shared__ uint32_t s_tmp[4];
    __shared__ uint32_t s_n;
    const uint32_t epoch = ld_volatile(&bt.bg->bar_epoch);
    uint32_t nbar = 0;
    auto sync = [&]() {
        ++nbar;
        grid_sync(bt.bg, epoch, nbar);
    };
    stamp(bt, 0);
    // read before any block can reach the final phase, which sets it
    const bool carried = __ldcg(&bt.inst0.g->freel_full) != 0u;
    // the decode tables are fetched now and stored after prep's own loads
    // have gone out
    static_assert(kFThreads == 256, "dec_fetch splits the table over 256 threads");
    uint4 tab[kDecVecs / 256u + 1u];
    dec_fetch(tab);
    if (threadIdx.x == 0) s_c.b = kNull;
    phase_prep1(bt, tbits);
    dec_store(s_tab, tab);
    sync();
    stamp(bt, 1);
    phase_classify1(bt, s_c, s_tab, s_cnt, reinterpret_cast<uint4*>(s_buf));
    sync();
    stamp(bt, 2);
    phase_walks1(bt, s_c, s_cnt, s_buf, s_warp, s_tmp, &s_n);
    sync();
    stamp(bt, 3);
    const Globals* g = bt.inst0.g;
    const bool all_granted = __ldcg(&g->rq_merge) + __ldcg(&g->rq_split) <= (unsigned long long)s_c.F;
    if (!all_granted) {
        phase_gate<true>(bt, s_c, s_cnt, s_red, s_warp, s_tmp, &s_n, reinterpret_cast<uint2*>(s_buf), true);
        sync();
    }
    stamp(bt, 4);
    phase_alloc1(bt, s_c, all_granted, carried, tbits, s_cnt, s_warp, s_w, &s_n, s_buf);
    sync();
    stamp(bt, 5);
    phase_fill1(bt, s_c, all_granted, s_cnt, s_buf, s_warp);
    sync();
    stamp(bt, 6);
    phase_final1(bt, s_c, s_buf, s_warp, s_tmp, tbits, carried);
    if (bt.fp0.vout) {
        sync();
        stamp(bt, 7);
        vertices_of(bt.inst0, bt.fp0, s_tab, s_buf, &s_n);
    } else {
        stamp(bt, 7);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (bt.timing) atomicMax(&bt.bg->t[kFramePhases], global_ns());
        if (blockIdx.x == 0) {
            bt.bg->bar_epoch = epoch + nbar * gridDim.x;
            if (ld_volatile(&bt.bg->abort)) set_err(bt.inst0.g, kErrTimeout);
        }
    }
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

int frame1_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_frame1, kFThreads, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_frame1(const BatchDev& bt, int grid, uint32_t tbits, cudaStream_t s) {
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
    return cudaLaunchKernelEx(&cfg, k_frame1, bt, tbits);
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
