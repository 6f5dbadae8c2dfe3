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
// chain. Every wait is bounded and sets kErrTimeout instead of hanging.
#include "cbt_kernels.cuh"

namespace cbtgpu {

constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t* cmd_ptr(const Inst& I, uint32_t s) {
    return reinterpret_cast<uint32_t*>(I.cd + s);
}
__device__ __forceinline__ uint32_t* dest_ptr(const Inst& I, uint32_t s) {
    return reinterpret_cast<uint32_t*>(I.cd + s) + 1;
}
// Every slot read out of device memory is checked before it is used as an
// index; a bad one sets the error word and the access is skipped.
__device__ __forceinline__ bool bad_slot(const Inst& I, uint32_t s, uint32_t err) {
    if (s < I.cap) return false;
    set_err(I.g, err);
    return true;
}
__device__ __forceinline__ uint32_t link_of(const uint4& r, int e) {
    return e == 0 ? r.x : (e == 1 ? r.y : r.z);
}
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ const FrameP& frame_of(const BatchDev& bt, uint32_t b) {
    return bt.fps ? bt.fps[b] : bt.fp0;
}

// Largest b in [0, B) with base[b] <= t (base is non-decreasing, base[B] is
// the total): the instance owning global tile t.
__device__ __forceinline__ uint32_t find_inst(const uint32_t* base, uint32_t B, uint32_t t) {
    uint32_t lo = 0, hi = B;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= t)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------ block scans

// Exclusive scan of one Pair per thread over the block (up to 1024
// threads); returns the thread's exclusive prefix and the block total.
// s_warp needs blockDim.x / 32 + 1 Pairs.
__device__ __forceinline__ Pair block_scan(Pair x, Pair& total, Pair* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    Pair inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Pair y{__shfl_up_sync(0xFFFFFFFFu, inc.a, o), __shfl_up_sync(0xFFFFFFFFu, inc.b, o)};
        if (lane >= o) inc = padd(inc, y);
    }
    Pair ex{__shfl_up_sync(0xFFFFFFFFu, inc.a, 1), __shfl_up_sync(0xFFFFFFFFu, inc.b, 1)};
    if (lane == 0) ex = Pair{0, 0};
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        Pair w = lane < nw ? s_warp[lane] : Pair{0, 0};
        Pair wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Pair y{__shfl_up_sync(0xFFFFFFFFu, wi.a, o), __shfl_up_sync(0xFFFFFFFFu, wi.b, o)};
            if (lane >= o) wi = padd(wi, y);
        }
        Pair we{__shfl_up_sync(0xFFFFFFFFu, wi.a, 1), __shfl_up_sync(0xFFFFFFFFu, wi.b, 1)};
        if (lane == 0) we = Pair{0, 0};
        __syncwarp();
        if (lane < nw) s_warp[lane] = we;
        if (lane == nw - 1) s_warp[nw] = wi;
    }
    __syncthreads();
    const Pair r = padd(s_warp[warp], ex);
    total = s_warp[nw];
    __syncthreads();
    return r;
}

// Exclusive prefix of global tile `tile` (local tile > 0), by all lanes of
// warp 0 after the tile's aggregate has been published. Bounded waits.
__device__ Pair lookback(unsigned long long* status, uint32_t tile, Globals* g) {
    const int lane = threadIdx.x & 31;
    Pair excl{0, 0};
    int p = (int)tile - 1;
    while (p >= 0) {
        const int idx = p - lane;
        unsigned long long s = idx >= 0 ? ld_status(status + idx) : pack_status(kFlagIncl, Pair{0, 0});
        int iters = 0;
        bool timed_out = false;
        while (!__all_sync(0xFFFFFFFFu, status_flag(s) != 0ull)) {
            if (++iters > kSpinLimit) {
                timed_out = true;
                break;
            }
            __nanosleep(32);
            if (status_flag(s) == 0ull && idx >= 0) s = ld_status(status + idx);
        }
        if (timed_out) {
            if (lane == 0) set_err(g, kErrTimeout);
            break;
        }
        const unsigned incl = __ballot_sync(0xFFFFFFFFu, status_flag(s) == kFlagIncl);
        const int first = incl ? __ffs(incl) - 1 : 31;
        Pair v = lane <= first ? status_val(s) : Pair{0, 0};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = padd(v, Pair{__shfl_xor_sync(0xFFFFFFFFu, v.a, o), __shfl_xor_sync(0xFFFFFFFFu, v.b, o)});
        excl = padd(excl, v);
        if (incl) break;
        p -= 32;
    }
    return excl;
}

// Publishes the tile aggregate, looks back (unless it is the instance's
// first tile), publishes the inclusive prefix; returns the exclusive prefix.
__device__ __forceinline__ Pair tile_prefix(unsigned long long* status, uint32_t tile, bool first,
                                            Pair agg, Globals* g, Pair* s_excl) {
    if (threadIdx.x < 32) {
        Pair ex{0, 0};
        if (first) {
            if (threadIdx.x == 0) st_status(status + tile, pack_status(kFlagIncl, agg));
        } else {
            if (threadIdx.x == 0) st_status(status + tile, pack_status(kFlagAgg, agg));
            ex = lookback(status, tile, g);
            if (threadIdx.x == 0) st_status(status + tile, pack_status(kFlagIncl, padd(ex, agg)));
        }
        if (threadIdx.x == 0) *s_excl = ex;
    }
    __syncthreads();
    const Pair r = *s_excl;
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t next_ticket(BatchGlobals* bg, int which, uint32_t* s_tile) {
    if (threadIdx.x == 0) *s_tile = atomicAdd(&bg->tickets[which], 1u);
    __syncthreads();
    const uint32_t t = *s_tile;
    __syncthreads();
    return t;
}

// Statistics: warp-aggregated adds into per-block shared counters, flushed
// to the instance's counters once per tile (block-uniform points), so that a
// frame costs one global atomic per counter and tile.
constexpr int kBlockStats = 4;
__device__ __forceinline__ void count_stat(uint32_t* s_cnt, int k, bool pred) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (m && (int)(threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(&s_cnt[k], (uint32_t)__popc(m));
}
__device__ __forceinline__ void stats_reset(uint32_t* s_cnt) {
    if (threadIdx.x < kBlockStats) s_cnt[threadIdx.x] = 0;
}
// Call between __syncthreads with every thread of the block.
__device__ __forceinline__ void stats_flush(uint32_t* s_cnt, Globals* g, int i0, int i1 = -1, int i2 = -1,
                                            int i3 = -1) {
    const int idx[kBlockStats] = {i0, i1, i2, i3};
    if (threadIdx.x < kBlockStats && idx[threadIdx.x] >= 0 && s_cnt[threadIdx.x])
        atomicAdd(&g->stats[idx[threadIdx.x]], s_cnt[threadIdx.x]);
}

// Per-tile copies of the instance descriptor and frame parameters in shared
// memory: their fields are then read without reloads after global stores.
__device__ __forceinline__ void load_tile_ctx(const BatchDev& bt, uint32_t b, Inst* s_inst, FrameP* s_fp) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(bt.inst + b);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_inst);
    for (uint32_t k = threadIdx.x; k < sizeof(Inst) / 4; k += blockDim.x) dst[k] = src[k];
    if (s_fp) {
        const uint32_t* fs = reinterpret_cast<const uint32_t*>(bt.fps ? bt.fps + b : &bt.fp0);
        uint32_t* fd = reinterpret_cast<uint32_t*>(s_fp);
        for (uint32_t k = threadIdx.x; k < sizeof(FrameP) / 4; k += blockDim.x) fd[k] = fs[k];
    }
}

// Start of a tile: its instance and local index, the instance descriptor
// and frame parameters copied to shared memory, the block counters cleared.
__device__ __forceinline__ void tile_begin(const BatchDev& bt, const uint32_t* base, uint32_t t, uint32_t* s_b,
                                           Inst* s_inst, FrameP* s_fp, uint32_t* s_cnt, uint32_t& b,
                                           uint32_t& lt) {
    if (threadIdx.x == 0) *s_b = find_inst(base, bt.B, t);
    if (s_cnt) stats_reset(s_cnt);
    __syncthreads();
    b = *s_b;
    lt = t - base[b];
    load_tile_ctx(bt, b, s_inst, s_fp);
    __syncthreads();
}

// ------------------------------------------------------------------ prep

// Frame start: per-instance counters, the item-tile prefix over the batch
// (block 0), the look-back descriptors zeroed, and the camera-relative root
// tables. FP64 is used here only to subtract the eye from the root vertices.
__global__ void __launch_bounds__(kThreads) k_prep(BatchDev bt, int frame_start) {
    __shared__ uint32_t s_carry, s_scarry;
    __shared__ Pair s_warp[kThreads / 32 + 1];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    if (frame_start) {
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) s_carry = s_scarry = 0;
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
                    tiles = (N + kTileItems - 1u) / kTileItems;
                    g->ntiles = tiles;
                    stl = (N + kScanItems - 1u) / kScanItems;
                    g->nstiles = stl;
                    for (int k = 0; k < kStCount; ++k) g->stats[k] = 0;
                    g->stats[kStLiveBefore] = N;
                    g->stats[kStFreeBefore] = I.cap - N;
                    g->stats[kStFrame] = frame_of(bt, b).frame;
                    if (bt.nout) bt.nout[b] = N;
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
                for (int k = 0; k < 8; ++k) bt.bg->tickets[k] = 0;
            }
        }
        const uint32_t nstat = 2u * bt.Titems + bt.Twords;
        for (uint32_t k = tid; k < nstat; k += nth) bt.status[k] = 0ull;
    }
    for (uint32_t e = tid; e < bt.Trel; e += nth) {
        const uint32_t b = find_inst(bt.rel_base, bt.B, e);
        const Inst& I = bt.inst[b];
        const FrameP& fp = frame_of(bt, b);
        const uint32_t le = e - bt.rel_base[b];
        const double diff = __dsub_rn(I.root64[le], fp.eye[le % 3u]);
        if (fp.precision == 1) {
            const double sc = __dmul_rn(diff, pow2d(fp.shift));
            long long x = 0;
            if (fabs(sc) < 4.611686018427387904e18)
                x = __double2ll_rn(sc);
            else
                set_err(I.g, kErrRange);
            static_cast<long long*>(I.rel)[le] = x;
        } else if (fp.precision == 2) {
            static_cast<double*>(I.rel)[le] = diff;
        } else {
            static_cast<float*>(I.rel)[le] = __double2float_rn(diff);
        }
    }
}

// ----------------------------------------------------------- merge groups

struct Group {
    uint32_t m[4];
    uint64_t j[4];
    int n, imin, np;
};

// Alg. 4 on the frame-start state. Members: m[0] = s1, m[1] its sibling,
// m[2] the bisector across the outer half of the refinement edge, m[3] its
// sibling.
__device__ bool find_group(const Inst& I, uint32_t s1, Group& g) {
    const uint64_t j1 = I.heap[s1];
    if (depth_of(j1, I.ch) < 1) return false;
    const uint4 r1 = I.nb[s1];
    const bool bit = j1 & 1ull;
    const uint32_t s2 = bit ? r1.z : r1.y;
    const uint32_t s3 = bit ? r1.y : r1.z;
    if (s2 == kNull || bad_slot(I, s2, kErrLink)) return false;
    if (s3 != kNull && bad_slot(I, s3, kErrLink)) return false;
    const uint64_t j2 = I.heap[s2];
    if ((j2 >> 1) != (j1 >> 1)) return false;
    g.m[0] = s1; g.j[0] = j1;
    g.m[1] = s2; g.j[1] = j2;
    g.m[2] = g.m[3] = kNull;
    g.n = 2;
    g.np = 1;
    if (s3 != kNull) {
        const uint64_t j3 = I.heap[s3];
        if (bitlen64(j3) != bitlen64(j1) || (j3 >> 1) == (j1 >> 1)) return false;
        const uint4 r3 = I.nb[s3];
        const uint32_t s4 = bit ? r3.y : r3.z;
        if (s4 == kNull || bad_slot(I, s4, kErrLink)) return false;
        const uint64_t j4 = I.heap[s4];
        if ((j4 >> 1) != (j3 >> 1)) return false;
        g.m[2] = s3; g.j[2] = j3;
        g.m[3] = s4; g.j[3] = j4;
        g.n = 4;
        g.np = 2;
    }
    g.imin = 0;
    for (int k = 1; k < g.n; ++k)
        if (g.j[k] < g.j[g.imin]) g.imin = k;
    return true;
}

// -------------------------------------------------------------- classify

template <typename T>
__device__ __forceinline__ void lod_wishes(const Inst& I, const FrameP& fp, uint64_t j, int d,
                                           uint32_t h, const uint32_t* tab, bool& split, bool& merge) {
    T W[9], Wp[9];
    decode_weights<T>(j, d, W, Wp, tab);
    float r[9];
    eval_vertices<T>(W, d, fp.precision, fp.shift, I.rel, h, r);
    split = lod_test(r, fp) == 3u && d < (int)I.max_depth;
    merge = false;
    if (!split && d >= 1) {
        eval_vertices<T>(Wp, d - 1, fp.precision, fp.shift, I.rel, h, r);
        merge = lod_test(r, fp) != 3u;
    }
}

// Compatibility chain of bisector b on the frame-start state (command form
// of Alg. 3): returns its allocation count; with `scatter` it ORs R (and N or
// P on coarser members) into the command words.
__device__ uint32_t chain_walk(const Inst& I, uint32_t b, int d, bool scatter) {
    uint32_t cur = b, cost = 2;
    if (scatter) atomicOr(cmd_ptr(I, b), kR);
    int dcur = d;
    for (int guard = 0; guard < 64; ++guard) {
        const uint32_t t = I.nb[cur].x;
        if (t == kNull) return cost;
        if (bad_slot(I, t, kErrChain)) return cost;
        const uint4 tn = I.nb[t];
        if (tn.x == cur) {
            if (scatter) atomicOr(cmd_ptr(I, t), kR);
            return cost + 2;
        }
        uint32_t bits;
        if (tn.y == cur) {
            bits = kR | kN;
        } else if (tn.z == cur) {
            bits = kR | kP;
        } else {
            set_err(I.g, kErrChain);
            return cost;
        }
        if (scatter) {
            atomicOr(cmd_ptr(I, t), bits);
        } else if (depth_of(I.heap[t], I.ch) + 1 != dcur) {
            set_err(I.g, kErrChain);
            return cost;
        }
        cost += 3;
        cur = t;
        --dcur;
    }
    set_err(I.g, kErrChain);
    return cost;
}

__device__ __forceinline__ void classify_item(const Inst& I, const FrameP& fp, uint64_t key, uint32_t i,
                                              uint32_t s, uint64_t j, const uint32_t* tab, uint32_t* s_cnt) {
    const int d = depth_of(j, I.ch);
    const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
    bool split = false, merge = false;
    if (d < 0 || h >= I.H) {
        set_err(I.g, kErrLink);
        *cmd_ptr(I, s) = 0u;
        I.scan[i] = 0u;
        return;
    }
    switch (fp.mode) {
        case 0:
            if (d <= 31)
                lod_wishes<uint32_t>(I, fp, j, d, h, tab, split, merge);
            else
                lod_wishes<unsigned long long>(I, fp, j, d, h, tab, split, merge);
            break;
        case 1:
            split = d < (int)I.max_depth;
            break;
        case 2:
            merge = d >= 1;
            break;
        case 3:
            split = d < (int)I.max_depth && (splitmix64(j ^ key) & 7ull) == 0ull;
            merge = !split && d >= 1 && (splitmix64((j >> 1) ^ key) & 1ull);
            break;
        default:
            split = d < (int)I.max_depth && in_sorted(fp.split_list, fp.n_split, j);
            merge = !split && d >= 1 && in_sorted(fp.merge_list, fp.n_merge, j);
            break;
    }
    const uint32_t cmd = (split ? kSplitWish : 0u) | (merge ? kMergeWish : 0u) |
                         ((d & 1) ? kDepthOdd : 0u) | ((j & 1ull) ? kHeapOdd : 0u);
    *cmd_ptr(I, s) = cmd;
    // the paper's gate charges 3d + 4 without walking the chain (k_walk
    // computes the exact chain cost otherwise)
    I.scan[i] = (split && fp.gate == 1) ? 3u * (uint32_t)d + 4u : 0u;
    count_stat(s_cnt, 0, split);
}

// Pointer chases of the frame, after classify: the compatibility-chain cost
// of every split wish (command form of Alg. 3) and the Alg. 4 group of every
// merge wish with an even heap ID, whose smallest member records the members
// (for the gate, the allocation and the fill). The items that need a walk
// are packed per tile in shared memory first, so that whole warps walk.
__global__ void __launch_bounds__(kThreads) k_walk(BatchDev bt) {
    __shared__ uint32_t s_b, s_n;
    __shared__ Inst s_I;
    __shared__ uint32_t s_list[kTileItems];
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
            const uint32_t cmd = *cmd_ptr(I, I.live[i]);
            const bool need = ((cmd & kSplitWish) && chain) || ((cmd & kMergeWish) && !(cmd & kHeapOdd));
            if (need) s_list[atomicAdd(&s_n, 1u)] = i;
        }
        __syncthreads();
        const uint32_t n = s_n;
        for (uint32_t q = threadIdx.x; q < n; q += kThreads) {
            const uint32_t i = s_list[q];
            const uint32_t s = I.live[i];
            const uint32_t cmd = *cmd_ptr(I, s);
            if (cmd & kSplitWish) {
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
    __shared__ uint32_t s_tab[64 * 9];
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
                uint32_t mc = 0;
                if (cmd & kGrpMin) {
                    const uint4 m = I.grp[i];
                    const uint32_t ms[3] = {m.y, m.z, m.w};
                    bool all = true;
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (ms[q] != kNull) all = all && (*cmd_ptr(I, ms[q]) & kMergeWish);
                    if (all) mc = gate == 1 ? 2u : (m.z == kNull ? 1u : 2u);
                }
                v[k] = Pair{mc, I.scan[i]};
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

// ------------------------------------------------------------ allocation

__device__ __forceinline__ uint32_t leaves_of(uint32_t sb) {
    return sb ? 2u + ((sb >> 1) & 1u) + ((sb >> 2) & 1u) : 0u;
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
            const uint32_t s = I.live[i];
            const uint32_t cmd = *cmd_ptr(I, s);
            const uint32_t sb = cmd & kSplitMask;
            uint32_t na = 0, merge = 0;
            if (sb) {
                na = leaves_of(sb);
            } else if ((cmd & kCand) && (cmd & kMergeGrant)) {
                const uint4 m = I.grp[i];
                const uint32_t ms[3] = {m.y, m.z, m.w};
                bool ok = true;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (ms[q] == kNull) continue;
                    if (bad_slot(I, ms[q], kErrLink)) {
                        ok = false;
                        continue;
                    }
                    const uint32_t c = *cmd_ptr(I, ms[q]);
                    ok = ok && (c & kMergeWish) && !(c & kSplitMask);
                }
                if (ok) {
                    merge = 1;
                    na = m.z == kNull ? 1u : 2u;
                }
            }
            packed |= (na | (merge << 3)) << (4 * k);
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
            if (!(f & 8u)) {
                *dest_ptr(I, I.live[i]) = run;
                count_stat(s_cnt, 0, true);
            } else {
                const uint4 m = I.grp[i];
                const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (ms[q] == kNull) continue;
                    atomicOr(cmd_ptr(I, ms[q]), kMerged);
                    *dest_ptr(I, ms[q]) = run + (q < 2 ? 0u : 1u);
                }
                atomicAdd(&s_cnt[2], m.z == kNull ? 2u : 4u);
                count_stat(s_cnt, 1, true);
            }
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

// ---------------------------------------------------------- fill / relink

// Leaves of a split bisector j (Table 1 applied once, or twice for the N / P
// bits), in depth-first order, with each leaf edge either internal (partner
// leaf and its edge) or lying on an old edge E of j (whole, or the half at
// E's first / second vertex).
struct EdgeDesc {
    uint8_t ext, a, b;  // ext=0: partner leaf a, partner edge b; ext=1: old edge a, portion b
};
struct FamDesc {
    uint8_t n;
    uint8_t shift[4], off[4];
    EdgeDesc e[4][3];
};

#define INT_(a, b) {0, a, b}
#define EXT_(a, b) {1, a, b}
__constant__ FamDesc c_fam[4] = {
    // R: 2j, 2j+1
    {2, {1, 1, 0, 0}, {0, 1, 0, 0},
     {{EXT_(kPe, kWhole), INT_(1, kPe), EXT_(kT, kFirst)},
      {EXT_(kNe, kWhole), EXT_(kT, kSecond), INT_(0, kNe)},
      {}, {}}},
    // R+N: 2j, 4j+2, 4j+3
    {3, {1, 2, 2, 0}, {0, 2, 3, 0},
     {{EXT_(kPe, kWhole), INT_(1, kT), EXT_(kT, kFirst)},
      {INT_(0, kNe), INT_(2, kPe), EXT_(kNe, kSecond)},
      {EXT_(kT, kSecond), EXT_(kNe, kFirst), INT_(1, kNe)},
      {}}},
    // R+P: 4j, 4j+1, 2j+1
    {3, {2, 2, 1, 0}, {0, 1, 1, 0},
     {{EXT_(kT, kFirst), INT_(1, kPe), EXT_(kPe, kSecond)},
      {INT_(2, kPe), EXT_(kPe, kFirst), INT_(0, kNe)},
      {EXT_(kNe, kWhole), EXT_(kT, kSecond), INT_(1, kT)},
      {}}},
    // R+N+P: 4j, 4j+1, 4j+2, 4j+3
    {4, {2, 2, 2, 2}, {0, 1, 2, 3},
     {{EXT_(kT, kFirst), INT_(1, kPe), EXT_(kPe, kSecond)},
      {INT_(2, kT), EXT_(kPe, kFirst), INT_(0, kNe)},
      {INT_(1, kT), INT_(3, kPe), EXT_(kNe, kSecond)},
      {EXT_(kT, kSecond), EXT_(kNe, kFirst), INT_(2, kNe)}}},
};
#undef INT_
#undef EXT_

__device__ __forceinline__ int fam_case(uint32_t sb) { return (int)((sb >> 1) & 3u); }

// Does a family with split bits sb cover old edge E by halves?
__device__ __forceinline__ bool halves(uint32_t sb, int E) {
    return E == kT || (E == kNe && (sb & kN)) || (E == kPe && (sb & kP));
}

// Leaf of family `sb` covering portion p of old edge Ep, and that leaf's edge.
__device__ __forceinline__ bool family_leaf(uint32_t sb, int Ep, int p, uint32_t& leaf, uint32_t& edge) {
    const FamDesc& f = c_fam[fam_case(sb)];
    for (int l = 0; l < f.n; ++l)
        for (int e = 0; e < 3; ++e)
            if (f.e[l][e].ext && f.e[l][e].a == Ep && f.e[l][e].b == p) {
                leaf = (uint32_t)l;
                edge = (uint32_t)e;
                return true;
            }
    return false;
}

// What lies across the old edges of a changed bisector x on the new mesh:
// per old edge E its old neighbour y (and y's edge facing x, command word and
// destination), then the new neighbour per portion used ([0] whole or first
// half, [1] second half) and that neighbour's edge facing the new bisector.
struct Across {
    uint32_t y[3];
    uint32_t ep[3];
    uint2 yc[3];
    uint32_t slot[3][2];
    uint32_t rev[3][2];
};

// The three neighbour loads are independent, so they overlap.
__device__ __forceinline__ void across_load(const Inst& I, const uint4& rx, Across& a) {
#pragma unroll
    for (int E = 0; E < 3; ++E) {
        a.y[E] = link_of(rx, E);
        a.ep[E] = (rx.w >> (2 * E)) & 3u;
        a.yc[E] = make_uint2(0u, 0u);
        if (a.y[E] != kNull && !bad_slot(I, a.y[E], kErrLink))
            a.yc[E] = I.cd[a.y[E]];
        else
            a.y[E] = kNull;
    }
}

// Resolves old edge E of x (depth parity xodd), whole (hv = false) or by
// halves: a split neighbour gives the leaf of its family on the same
// portion, a merged one its parent, an unchanged one itself (R11 reading).
__device__ void across_resolve(const Inst& I, Across& a, int E, bool hv, bool xodd) {
    const uint32_t y = a.y[E];
    a.slot[E][0] = a.slot[E][1] = kNull;
    a.rev[E][0] = a.rev[E][1] = 3u;
    if (y == kNull) return;
    const int Ep = (int)a.ep[E];
    const uint2 yc = a.yc[E];
    const uint32_t ysb = yc.x & kSplitMask;
    const uint32_t A = I.g->A;
    if (Ep > 2) {
        set_err(I.g, kErrLink);
        return;
    }
    if (ysb) {
        const bool same = ((yc.x & kDepthOdd) != 0u) == xodd;
        for (int h = 0; h < (hv ? 2 : 1); ++h) {
            int p = hv ? (h == 0 ? kFirst : kSecond) : kWhole;
            if (p != kWhole && same) p = p == kFirst ? kSecond : kFirst;
            uint32_t leaf, edge;
            if (!family_leaf(ysb, Ep, p, leaf, edge) || yc.y + leaf >= A) {
                set_err(I.g, kErrLink);
                continue;
            }
            a.slot[E][h] = I.freel[yc.y + leaf];
            a.rev[E][h] = edge;
        }
    } else if (yc.x & kMerged) {
        if (hv || Ep != kT || yc.y >= A) {
            set_err(I.g, kErrLink);
            return;
        }
        a.slot[E][0] = I.freel[yc.y];
        a.rev[E][0] = (yc.x & kHeapOdd) ? (uint32_t)kNe : (uint32_t)kPe;
    } else {
        if (hv) {
            set_err(I.g, kErrLink);
            return;
        }
        a.slot[E][0] = y;
        a.rev[E][0] = (uint32_t)Ep;
    }
}

// An unchanged neighbour across old edge E of x now faces new bisector ns
// through ns's edge ne; that neighbour link has exactly one writer, this one.
__device__ __forceinline__ void push_keep(const Inst& I, const Across& a, int E, uint32_t ns, uint32_t ne,
                                          uint32_t* s_cnt) {
    const uint32_t y = a.y[E];
    if (y == kNull || (a.yc[E].x & (kSplitMask | kMerged))) return;
    uint32_t* yr = reinterpret_cast<uint32_t*>(I.nb + y);
    const int Ep = (int)a.ep[E];
    yr[Ep] = ns;
    atomicXor(yr + 3, ((uint32_t)E ^ ne) << (2 * Ep));
    atomicAdd(&s_cnt[0], 1u);
}

__device__ __forceinline__ void set_bit(const Inst& I, uint32_t s) {
    atomicOr(I.bits + (s >> 5), 1u << (s & 31u));
}
__device__ __forceinline__ void clear_bit(const Inst& I, uint32_t s) {
    atomicAnd(I.bits + (s >> 5), ~(1u << (s & 31u)));
}

__device__ void fill_split(const Inst& I, uint32_t s, uint32_t cmd, uint32_t dest, uint32_t* s_cnt) {
    const uint32_t sb = cmd & kSplitMask;
    const FamDesc& f = c_fam[fam_case(sb)];
    if (dest + f.n > I.g->A) {
        set_err(I.g, kErrOverflow);
        return;
    }
    const uint64_t j = I.heap[s];
    const uint4 rx = I.nb[s];
    uint32_t slots[4];
    for (int l = 0; l < f.n; ++l) slots[l] = I.freel[dest + (uint32_t)l];
    Across a;
    across_load(I, rx, a);
    const bool xodd = (cmd & kDepthOdd) != 0u;
#pragma unroll
    for (int E = 0; E < 3; ++E) across_resolve(I, a, E, halves(sb, E), xodd);
    for (int l = 0; l < f.n; ++l)
        if (bad_slot(I, slots[l], kErrOverflow)) return;
    for (int l = 0; l < f.n; ++l) {
        uint32_t lk[3], rv = 0;
        for (int e = 0; e < 3; ++e) {
            const EdgeDesc ed = f.e[l][e];
            uint32_t r;
            if (!ed.ext) {
                lk[e] = slots[ed.a];
                r = ed.b;
            } else {
                const int h = ed.b == kSecond ? 1 : 0;
                lk[e] = a.slot[ed.a][h];
                r = a.rev[ed.a][h];
                if (ed.b == kWhole) push_keep(I, a, ed.a, slots[l], (uint32_t)e, s_cnt);
            }
            rv |= r << (2 * e);
        }
        I.nb[slots[l]] = make_uint4(lk[0], lk[1], lk[2], rv);
        I.heap[slots[l]] = (j << f.shift[l]) + f.off[l];
        set_bit(I, slots[l]);
    }
}

// Parents of a valid merge group (Alg. 4), written by its smallest member:
// Next = across child 2p+1's Twin edge, Prev = across child 2p's Twin edge,
// Twin = the other parent (Table 1 read backwards, Alg. 6). Members m0, m1
// are the children of the smaller parent, m2, m3 of the other one.
__device__ void fill_merge(const Inst& I, uint32_t dest, const uint4 m, uint32_t* s_cnt) {
    const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
    const int np = m.z == kNull ? 1 : 2;
    if (dest + (uint32_t)np > I.g->A) {
        set_err(I.g, kErrOverflow);
        return;
    }
    uint32_t ps[2] = {kNull, kNull};
    for (int k = 0; k < np; ++k) {
        ps[k] = I.freel[dest + (uint32_t)k];
        if (bad_slot(I, ps[k], kErrOverflow)) return;
    }
    for (int pk = 0; pk < np; ++pk) {
        const uint32_t u = ms[2 * pk], v = ms[2 * pk + 1];
        if (bad_slot(I, u, kErrLink) || bad_slot(I, v, kErrLink)) return;
        const uint64_t ju = I.heap[u];
        const uint32_t a = (ju & 1ull) ? v : u;   // child 2p
        const uint32_t c1 = (ju & 1ull) ? u : v;  // child 2p+1
        const bool modd = (*cmd_ptr(I, a) & kDepthOdd) != 0u;
        Across xa, xb;
        const uint4 ra = I.nb[a], rb = I.nb[c1];
        across_load(I, rb, xb);
        across_load(I, ra, xa);
        across_resolve(I, xb, kT, false, modd);
        across_resolve(I, xa, kT, false, modd);
        push_keep(I, xb, kT, ps[pk], (uint32_t)kNe, s_cnt);
        push_keep(I, xa, kT, ps[pk], (uint32_t)kPe, s_cnt);
        const uint32_t tw = np == 2 ? ps[1 - pk] : kNull;
        const uint32_t rvT = np == 2 ? (uint32_t)kT : 3u;
        I.nb[ps[pk]] = make_uint4(tw, xb.slot[kT][0], xa.slot[kT][0],
                                  rvT | (xb.rev[kT][0] << 2) | (xa.rev[kT][0] << 4));
        I.heap[ps[pk]] = ju >> 1;
        set_bit(I, ps[pk]);
    }
}

// FillNewBlocks + UpdateNeighbors + UpdateBitfield for the changed
// bisectors, one per thread over the instance's compacted list (written in
// ascending slot order by k_alloc): a split bisector clears its bit and
// writes its family; the smallest member of a merge group clears its
// members' bits and writes the parents.
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
            if (c.x & kSplitMask) {
                clear_bit(I, s);
                fill_split(I, s, c.x, c.y, s_cnt);
            } else {
                const uint4 m = I.grp[i];
                const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (ms[q] != kNull && !bad_slot(I, ms[q], kErrLink)) clear_bit(I, ms[q]);
                fill_merge(I, c.y, m, s_cnt);
            }
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

__device__ __forceinline__ void vertex_item(const Inst& I, const FrameP& fp, uint32_t i, uint64_t j,
                                            const uint32_t* tab, float* out) {
    const int d = depth_of(j, I.ch);
    const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
    float r[9];
    if (d < 0 || h >= I.H) {
        set_err(I.g, kErrLink);
        return;
    }
    if (d <= 31) {
        uint32_t W[9], Wp[9];
        decode_weights<uint32_t>(j, d, W, Wp, tab);
        eval_vertices<uint32_t>(W, d, fp.precision, fp.shift, I.rel, h, r);
    } else {
        unsigned long long W[9], Wp[9];
        decode_weights<unsigned long long>(j, d, W, Wp, tab);
        eval_vertices<unsigned long long>(W, d, fp.precision, fp.shift, I.rel, h, r);
    }
    float* o = out + 9ull * i;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = r[k];
}

// Vertices of the live bisectors of every instance with an output buffer,
// over static tiles of its pool capacity (tiles past the live count exit).
__global__ void __launch_bounds__(kThreads, 3) k_vertices(BatchDev bt) {
    __shared__ uint32_t s_b;
    __shared__ Inst s_I;
    __shared__ FrameP s_fp;
    __shared__ uint32_t s_tab[64 * 9];
    load_dec6(s_tab);
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
            for (int k = 0; k < kItemsPerThread; ++k) {
                const uint32_t i = lt * kTileItems + (uint32_t)k * kThreads + threadIdx.x;
                if (i < N) vertex_item(I, fp, i, hj[k], s_tab, fp.vout);
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
