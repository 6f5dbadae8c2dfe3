// Kernels of one frame of the CBT bisection update for sm_103a.
//
// Frame = k_prep, k_classify, k_gate, k_scatter, k_alloc, k_free, k_fill,
// k_cbt. Every per-bisector kernel reads the live count from device memory
// (the CBT root) and walks a grid-stride loop, which replaces the paper's
// DispatchIndirect. The two prefix scans are single-pass decoupled look-back
// scans over tiles handed out by an atomic ticket, so a tile only ever waits
// for tiles already owned by running blocks; every wait is bounded and sets
// kErrTimeout instead of hanging.
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

// ------------------------------------------------------------ block scans

// Exclusive scan of one Pair per thread over a 256-thread block; returns the
// thread's exclusive prefix and the block total. s_warp needs 9 Pairs.
__device__ __forceinline__ Pair block_scan(Pair x, Pair& total, Pair* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
        Pair w = lane < kThreads / 32 ? s_warp[lane] : Pair{0, 0};
        Pair wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Pair y{__shfl_up_sync(0xFFFFFFFFu, wi.a, o), __shfl_up_sync(0xFFFFFFFFu, wi.b, o)};
            if (lane >= o) wi = padd(wi, y);
        }
        Pair we{__shfl_up_sync(0xFFFFFFFFu, wi.a, 1), __shfl_up_sync(0xFFFFFFFFu, wi.b, 1)};
        if (lane == 0) we = Pair{0, 0};
        __syncwarp();
        if (lane < kThreads / 32) s_warp[lane] = we;
        if (lane == kThreads / 32 - 1) s_warp[kThreads / 32] = wi;
    }
    __syncthreads();
    const Pair r = padd(s_warp[warp], ex);
    total = s_warp[kThreads / 32];
    __syncthreads();
    return r;
}

// Exclusive prefix of tile `tile` (called by all lanes of warp 0 after the
// tile's aggregate has been published). Bounded waits.
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

// Publishes the tile aggregate, looks back, publishes the inclusive prefix;
// returns the tile's exclusive prefix to every thread.
__device__ __forceinline__ Pair tile_prefix(unsigned long long* status, uint32_t tile, Pair agg,
                                            Globals* g, Pair* s_excl) {
    if (threadIdx.x < 32) {
        Pair ex{0, 0};
        if (tile == 0) {
            if (threadIdx.x == 0) st_status(status, pack_status(kFlagIncl, agg));
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

__device__ __forceinline__ uint32_t next_tile(Globals* g, int which, uint32_t* s_tile) {
    if (threadIdx.x == 0) *s_tile = atomicAdd(&g->tickets[which], 1u);
    __syncthreads();
    const uint32_t t = *s_tile;
    __syncthreads();
    return t;
}

// Warp-aggregated statistics counter.
__device__ __forceinline__ void count_stat(Globals* g, int idx, bool pred) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (m && (int)(threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(&g->stats[idx], (uint32_t)__popc(m));
}

// ------------------------------------------------------------------ prep

// Per-frame reset and camera-relative root table. FP64 is used here only to
// subtract the origin from the FP64 root vertices.
__global__ void __launch_bounds__(kThreads) k_prep(Inst I, FrameP fp, int frame_start) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    if (frame_start) {
        if (tid == 0) {
            const uint32_t N = I.sums[1];
            I.g->N = N;
            I.g->F = I.cap - N;
            I.g->A = 0;
            I.g->Mg = 0;
            I.g->done = 0;
            for (int k = 0; k < 4; ++k) I.g->tickets[k] = 0;
            for (int k = 0; k < kStCount; ++k) I.g->stats[k] = 0;
            I.g->stats[kStLiveBefore] = N;
            I.g->stats[kStFreeBefore] = I.cap - N;
            I.g->stats[kStFrame] = fp.frame;
        }
        const uint32_t nstat = 3u * I.ntiles_items + I.ntiles_words;
        for (uint32_t k = tid; k < nstat; k += nth) I.status[k] = 0ull;
    }
    const uint32_t n = 9u * I.H;
    for (uint32_t e = tid; e < n; e += nth) {
        const double diff = __dsub_rn(I.root64[e], fp.eye[e % 3u]);
        if (fp.precision == 1) {
            const double sc = __dmul_rn(diff, pow2d(fp.shift));
            long long x = 0;
            if (fabs(sc) < 4.611686018427387904e18)
                x = __double2ll_rn(sc);
            else
                set_err(I.g, kErrRange);
            static_cast<long long*>(I.rel)[e] = x;
        } else if (fp.precision == 2) {
            static_cast<double*>(I.rel)[e] = diff;
        } else {
            static_cast<float*>(I.rel)[e] = __double2float_rn(diff);
        }
    }
}

// -------------------------------------------------------------- classify

template <typename T>
__device__ __forceinline__ void lod_wishes(const Inst& I, const FrameP& fp, uint64_t j, int d,
                                           uint32_t h, bool& split, bool& merge) {
    T W[9], Wp[9];
    decode_weights<T>(j, d, W, Wp);
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

__global__ void __launch_bounds__(kThreads) k_classify(Inst I, FrameP fp) {
    const uint32_t N = ld_volatile(&I.g->N);
    const uint64_t key = splitmix64(((uint64_t)fp.seed << 32) | (uint64_t)fp.frame);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t s = I.live[i];
        const uint64_t j = I.heap[s];
        const int d = depth_of(j, I.ch);
        const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
        bool split = false, merge = false;
        if (d < 0 || h >= I.H) {
            set_err(I.g, kErrLink);
            *cmd_ptr(I, s) = 0u;
            I.scan[i] = 0u;
            continue;
        }
        switch (fp.mode) {
            case 0:
                if (d <= 31)
                    lod_wishes<uint32_t>(I, fp, j, d, h, split, merge);
                else
                    lod_wishes<unsigned long long>(I, fp, j, d, h, split, merge);
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
        uint32_t cost = 0;
        if (split) cost = fp.gate == 1 ? 3u * (uint32_t)d + 4u : chain_walk(I, s, d, false);
        I.scan[i] = cost;
        count_stat(I.g, kStSplitWishes, split);
    }
}

// ----------------------------------------------------------- merge groups

struct Group {
    uint32_t m[4];
    uint64_t j[4];
    int n, imin, np;
    uint64_t p[2];
};

// Alg. 4 on the frame-start state.
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
    g.n = 2;
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
    }
    g.imin = 0;
    for (int k = 1; k < g.n; ++k)
        if (g.j[k] < g.j[g.imin]) g.imin = k;
    g.p[0] = g.j[0] >> 1;
    g.np = 1;
    if (g.n == 4) {
        const uint64_t q = g.j[2] >> 1;
        if (q < g.p[0]) {
            g.p[1] = g.p[0];
            g.p[0] = q;
        } else {
            g.p[1] = q;
        }
        g.np = 2;
    }
    return true;
}

__device__ __forceinline__ int parent_index(const Group& g, int k) {
    return (g.np == 2 && (g.j[k] >> 1) == g.p[1]) ? 1 : 0;
}

// ------------------------------------------------------------------ gate

// Scan of (merge cost at the group's smallest member, split chain cost) in
// ascending slot order; merges are granted while their running total fits
// the free slots, then splits while (granted merges + their running total)
// fits (deterministic form of the allocation-counter test of Sec. 3.3).
__global__ void __launch_bounds__(kThreads) k_gate(Inst I, FrameP fp) {
    __shared__ uint32_t s_tile;
    __shared__ Pair s_warp[kThreads / 32 + 1];
    __shared__ Pair s_excl;
    const uint32_t N = ld_volatile(&I.g->N);
    const uint32_t F = ld_volatile(&I.g->F);
    const uint32_t ntiles = (N + kTileItems - 1) / kTileItems;
    unsigned long long* status = I.status;
    for (;;) {
        const uint32_t tile = next_tile(I.g, 0, &s_tile);
        if (tile >= ntiles) break;
        const uint32_t base = tile * kTileItems + threadIdx.x * kItemsPerThread;
        Pair v[kItemsPerThread];
        uint32_t slot[kItemsPerThread];
        Pair loc{0, 0};
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = base + k;
            v[k] = Pair{0, 0};
            slot[k] = kNull;
            if (i < N) {
                const uint32_t s = I.live[i];
                slot[k] = s;
                const uint32_t cmd = *cmd_ptr(I, s);
                uint32_t mc = 0;
                if (cmd & kMergeWish) {
                    Group g;
                    if (find_group(I, s, g) && g.imin == 0) {
                        bool all = true;
                        for (int m = 1; m < g.n; ++m) all = all && (*cmd_ptr(I, g.m[m]) & kMergeWish);
                        if (all) mc = fp.gate == 1 ? 2u : (uint32_t)g.np;
                    }
                }
                v[k] = Pair{mc, I.scan[i]};
                loc = padd(loc, v[k]);
            }
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        const Pair ex = tile_prefix(status, tile, tot, I.g, &s_excl);
        Pair run = padd(ex, tex);
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = base + k;
            run = padd(run, v[k]);
            if (i >= N) continue;
            const bool cand = v[k].a > 0;
            const bool granted = cand && run.a <= F;
            if (granted) {
                atomicOr(cmd_ptr(I, slot[k]), kMergeGrant);
                atomicMax(&I.g->Mg, run.a);
            }
            I.scan[i] = run.b;
            count_stat(I.g, kStMergeCand, cand);
            count_stat(I.g, kStMergeGranted, granted);
        }
    }
}

// --------------------------------------------------------------- scatter

__global__ void __launch_bounds__(kThreads) k_scatter(Inst I) {
    const uint32_t N = ld_volatile(&I.g->N);
    const uint64_t F = ld_volatile(&I.g->F);
    const uint64_t Mg = ld_volatile(&I.g->Mg);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t s = I.live[i];
        const uint32_t cmd = *cmd_ptr(I, s);
        bool granted = false;
        if (cmd & kSplitWish) {
            granted = Mg + (uint64_t)I.scan[i] <= F;
            if (granted) chain_walk(I, s, 0, true);
        }
        count_stat(I.g, kStSplitGranted, granted);
    }
}

// ------------------------------------------------------------ allocation

// Fates and the exclusive scan of allocation counts in ascending slot order
// (ReserveBlocks): a split bisector takes 2-4 leaves, a valid merge group
// its parents at its smallest member. dest = index into the free list.
__global__ void __launch_bounds__(kThreads) k_alloc(Inst I) {
    __shared__ uint32_t s_tile;
    __shared__ Pair s_warp[kThreads / 32 + 1];
    __shared__ Pair s_excl;
    const uint32_t N = ld_volatile(&I.g->N);
    const uint32_t ntiles = (N + kTileItems - 1) / kTileItems;
    unsigned long long* status = I.status + I.ntiles_items;
    for (;;) {
        const uint32_t tile = next_tile(I.g, 1, &s_tile);
        if (tile >= ntiles) break;
        const uint32_t base = tile * kTileItems + threadIdx.x * kItemsPerThread;
        uint32_t na[kItemsPerThread], slot[kItemsPerThread];
        uint8_t fate[kItemsPerThread];  // 0 keep, 1 split, 2 merged, 3 merged min
        Pair loc{0, 0};
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = base + k;
            na[k] = 0;
            fate[k] = 0;
            slot[k] = kNull;
            if (i >= N) continue;
            const uint32_t s = I.live[i];
            slot[k] = s;
            const uint32_t cmd = *cmd_ptr(I, s);
            const uint32_t sb = cmd & kSplitMask;
            if (sb) {
                na[k] = 2u + ((sb >> 1) & 1u) + ((sb >> 2) & 1u);
                fate[k] = 1;
            } else if (cmd & kMergeWish) {
                Group g;
                if (find_group(I, s, g)) {
                    bool ok = (*cmd_ptr(I, g.m[g.imin]) & kMergeGrant) != 0u;
                    for (int m = 0; m < g.n; ++m) {
                        const uint32_t c = *cmd_ptr(I, g.m[m]);
                        ok = ok && (c & kMergeWish) && !(c & kSplitMask);
                    }
                    if (ok) {
                        fate[k] = g.imin == 0 ? 3 : 2;
                        if (g.imin == 0) na[k] = (uint32_t)g.np;
                    }
                }
            }
            loc = padd(loc, Pair{0, na[k]});
        }
        Pair tot;
        const Pair tex = block_scan(loc, tot, s_warp);
        const Pair ex = tile_prefix(status, tile, tot, I.g, &s_excl);
        uint32_t run = ex.b + tex.b;
#pragma unroll
        for (int k = 0; k < kItemsPerThread; ++k) {
            const uint32_t i = base + k;
            if (i >= N) continue;
            const uint32_t s = slot[k];
            if (fate[k] == 1) {
                *dest_ptr(I, s) = run;
            } else if (fate[k] >= 2) {
                atomicOr(cmd_ptr(I, s), kMerged);
                if (fate[k] == 3) {
                    Group g;
                    find_group(I, s, g);
                    for (int m = 0; m < g.n; ++m) *dest_ptr(I, g.m[m]) = run + (uint32_t)parent_index(g, m);
                }
            }
            run += na[k];
            count_stat(I.g, kStSplitBis, fate[k] == 1);
            count_stat(I.g, kStMergedBis, fate[k] >= 2);
            count_stat(I.g, kStMergeGroups, fate[k] == 3);
        }
        if (tile == ntiles - 1 && threadIdx.x == kThreads - 1) {
            I.g->A = run;
            I.g->stats[kStAllocated] = run;
            if (run > I.g->F) set_err(I.g, kErrOverflow);
        }
    }
}

// ------------------------------------------------------------- free list

// freel[k] = slot of the k-th zero bit of the frame-start bitfield, k < A
// (Alg. 8 for the first A ranks at once): tiles of words find their zero
// offset from the sum tree and emit their zeros in order.
__global__ void __launch_bounds__(kThreads) k_free(Inst I) {
    __shared__ Pair s_warp[kThreads / 32 + 1];
    const uint32_t A = min(ld_volatile(&I.g->A), ld_volatile(&I.g->F));
    if (A == 0) return;
    const uint32_t TW = I.tile_words;
    for (uint32_t t = blockIdx.x; t < I.ntiles_words; t += gridDim.x) {
        uint32_t ones_before = 0;
        for (uint32_t n = I.ntiles_words + t; n > 1; n >>= 1)
            if (n & 1u) ones_before += I.sums[n - 1];
        const uint64_t zeros_before = (uint64_t)t * TW * 32u - ones_before;
        if (zeros_before >= A) break;
        uint32_t words[4] = {0, 0, 0, 0}, zc[4] = {0, 0, 0, 0};
        uint32_t total = 0;
        const uint32_t w0 = t * TW + threadIdx.x * 4u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = w0 + k;
            if (threadIdx.x * 4u + k < TW) {
                uint32_t valid = 0xFFFFFFFFu;
                if (I.cap < 32u) valid = (1u << I.cap) - 1u;
                words[k] = ~I.bits[w] & valid;
                zc[k] = __popc(words[k]);
                total += zc[k];
            }
        }
        Pair tot;
        const Pair ex = block_scan(Pair{0, total}, tot, s_warp);
        uint64_t r = zeros_before + ex.b;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t m = words[k];
            while (m && r < A) {
                const int b = __ffs(m) - 1;
                I.freel[r] = (w0 + k) * 32u + (uint32_t)b;
                ++r;
                m &= m - 1u;
            }
        }
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

// Neighbour across the portion `portion` of old edge E of old bisector x
// (record rx, depth parity xodd) for a new bisector at `newslot` whose edge
// `newedge` covers it. Returns the new neighbour slot and the neighbour's
// edge that faces it; an unchanged neighbour gets its own link rewritten
// (it has exactly one writer: the bisector across that edge).
__device__ uint32_t resolve(const Inst& I, const uint4& rx, bool xodd, int E, int portion,
                            uint32_t newslot, int newedge, uint32_t& rev) {
    const uint32_t y = link_of(rx, E);
    rev = 3u;
    if (y == kNull) return kNull;
    if (bad_slot(I, y, kErrLink)) return kNull;
    const int Ep = (int)((rx.w >> (2 * E)) & 3u);
    if (Ep > 2) {
        set_err(I.g, kErrLink);
        return kNull;
    }
    const uint2 yc = I.cd[y];
    const uint32_t A = I.g->A;
    const uint32_t ysb = yc.x & kSplitMask;
    if (ysb) {
        int py = portion;
        if (portion != kWhole && (((yc.x & kDepthOdd) != 0u) == xodd)) py = portion == kFirst ? kSecond : kFirst;
        const FamDesc& f = c_fam[fam_case(ysb)];
        for (int l = 0; l < f.n; ++l)
            for (int e = 0; e < 3; ++e)
                if (f.e[l][e].ext && f.e[l][e].a == Ep && f.e[l][e].b == py) {
                    if (yc.y + (uint32_t)l >= A) {
                        set_err(I.g, kErrLink);
                        return kNull;
                    }
                    rev = (uint32_t)e;
                    return I.freel[yc.y + (uint32_t)l];
                }
        set_err(I.g, kErrLink);
        return kNull;
    }
    if (yc.x & kMerged) {
        if (portion != kWhole || Ep != kT) set_err(I.g, kErrLink);
        if (yc.y >= A) {
            set_err(I.g, kErrLink);
            return kNull;
        }
        rev = (yc.x & kHeapOdd) ? (uint32_t)kNe : (uint32_t)kPe;
        return I.freel[yc.y];
    }
    if (portion != kWhole) set_err(I.g, kErrLink);
    uint32_t* yr = reinterpret_cast<uint32_t*>(I.nb + y);
    yr[Ep] = newslot;
    atomicXor(yr + 3, ((uint32_t)(E ^ newedge)) << (2 * Ep));
    atomicAdd(&I.g->stats[kStRelinked], 1u);
    rev = (uint32_t)Ep;
    return y;
}

__device__ __forceinline__ void set_bit(const Inst& I, uint32_t s) {
    atomicOr(I.bits + (s >> 5), 1u << (s & 31u));
}
__device__ __forceinline__ void clear_bit(const Inst& I, uint32_t s) {
    atomicAnd(I.bits + (s >> 5), ~(1u << (s & 31u)));
}

__device__ void fill_split(const Inst& I, uint32_t s, uint32_t cmd, uint32_t dest) {
    const uint64_t j = I.heap[s];
    const uint4 rx = I.nb[s];
    const bool xodd = (cmd & kDepthOdd) != 0u;
    const FamDesc& f = c_fam[fam_case(cmd & kSplitMask)];
    if (dest + f.n > I.g->A) {
        set_err(I.g, kErrOverflow);
        return;
    }
    uint32_t slots[4];
    for (int l = 0; l < f.n; ++l) {
        slots[l] = I.freel[dest + (uint32_t)l];
        if (bad_slot(I, slots[l], kErrOverflow)) return;
    }
    for (int l = 0; l < f.n; ++l) {
        uint32_t lk[3], rv = 0;
        for (int e = 0; e < 3; ++e) {
            const EdgeDesc ed = f.e[l][e];
            uint32_t r;
            if (!ed.ext) {
                lk[e] = slots[ed.a];
                r = ed.b;
            } else {
                lk[e] = resolve(I, rx, xodd, ed.a, ed.b, slots[l], e, r);
            }
            rv |= r << (2 * e);
        }
        I.nb[slots[l]] = make_uint4(lk[0], lk[1], lk[2], rv);
        I.heap[slots[l]] = (j << f.shift[l]) + f.off[l];
        set_bit(I, slots[l]);
    }
}

// Parents of a valid merge group (Alg. 4) written by its smallest member:
// Next = across child 2p+1's Twin edge, Prev = across child 2p's Twin edge,
// Twin = the other parent (Table 1 read backwards, Alg. 6).
__device__ void fill_merge(const Inst& I, uint32_t s, uint32_t dest) {
    Group g;
    if (!find_group(I, s, g)) {
        set_err(I.g, kErrLink);
        return;
    }
    const uint32_t base = dest - (uint32_t)parent_index(g, 0);
    if (base + (uint32_t)g.np > I.g->A) {
        set_err(I.g, kErrOverflow);
        return;
    }
    for (int pk = 0; pk < g.np; ++pk) {
        const uint64_t p = g.p[pk];
        uint32_t a = kNull, b = kNull;
        for (int m = 0; m < g.n; ++m) {
            if (g.j[m] == 2 * p) a = g.m[m];
            if (g.j[m] == 2 * p + 1) b = g.m[m];
        }
        const uint32_t ps = I.freel[base + (uint32_t)pk];
        const uint32_t tw = g.np == 2 ? I.freel[base + (uint32_t)(1 - pk)] : kNull;
        if (a == kNull || b == kNull || bad_slot(I, ps, kErrOverflow) || (tw != kNull && bad_slot(I, tw, kErrOverflow))) {
            set_err(I.g, kErrLink);
            return;
        }
        const uint32_t rvT = g.np == 2 ? (uint32_t)kT : 3u;
        uint32_t rvN, rvP;
        const uint4 rb = I.nb[b], ra = I.nb[a];
        const bool modd = (*cmd_ptr(I, a) & kDepthOdd) != 0u;
        const uint32_t nx = resolve(I, rb, modd, kT, kWhole, ps, kNe, rvN);
        const uint32_t pv = resolve(I, ra, modd, kT, kWhole, ps, kPe, rvP);
        I.nb[ps] = make_uint4(tw, nx, pv, rvT | (rvN << 2) | (rvP << 4));
        I.heap[ps] = p;
        set_bit(I, ps);
    }
}

// FillNewBlocks + UpdateNeighbors + UpdateBitfield for the changed bisectors.
__global__ void __launch_bounds__(kThreads) k_fill(Inst I) {
    const uint32_t N = ld_volatile(&I.g->N);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t s = I.live[i];
        const uint2 c = I.cd[s];
        const uint32_t sb = c.x & kSplitMask;
        if (!sb && !(c.x & kMerged)) continue;
        clear_bit(I, s);
        if (sb) {
            fill_split(I, s, c.x, c.y);
        } else {
            // The smallest member writes the parents; it is the member whose
            // dest is its own parent's first index with parent index 0 ...
            Group g;
            if (find_group(I, s, g) && g.imin == 0) fill_merge(I, s, c.y);
        }
    }
}

// ------------------------------------------------------ reduce + compact

// SumReduction over the updated bitfield fused with CachePointers' live list:
// each tile of words writes its part of the sum tree, finds its live-count
// prefix by look-back and writes the slots of its set bits; the last tile to
// finish builds the levels above the tiles.
__global__ void __launch_bounds__(kThreads) k_cbt(Inst I) {
    __shared__ uint32_t s_tile;
    __shared__ Pair s_warp[kThreads / 32 + 1];
    __shared__ Pair s_excl;
    __shared__ uint32_t s_lvl[2][kThreads];
    __shared__ uint32_t s_last;
    const uint32_t TW = I.tile_words, W = I.W;
    unsigned long long* status = I.status + 3u * I.ntiles_items;
    for (;;) {
        const uint32_t tile = next_tile(I.g, 2, &s_tile);
        if (tile >= I.ntiles_words) break;
        const uint32_t w0 = tile * TW + threadIdx.x * 4u;
        uint32_t wv[4] = {0, 0, 0, 0}, pc[4] = {0, 0, 0, 0};
        const bool mine = threadIdx.x * 4u < TW;
        if (mine) {
            if (TW >= 4u) {
                const uint4 q = *reinterpret_cast<const uint4*>(I.bits + w0);
                wv[0] = q.x; wv[1] = q.y; wv[2] = q.z; wv[3] = q.w;
            } else {
                for (uint32_t k = 0; k < TW; ++k) wv[k] = I.bits[w0 + k];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) pc[k] = __popc(wv[k]);
        // word level and the two levels above it, from registers
        if (mine) {
            for (uint32_t k = 0; k < 4u && threadIdx.x * 4u + k < TW; ++k) I.sums[W + w0 + k] = pc[k];
            if (TW >= 2u) {
                I.sums[(W + w0) >> 1] = pc[0] + pc[1];
                if (TW >= 4u) {
                    I.sums[((W + w0) >> 1) + 1] = pc[2] + pc[3];
                    I.sums[(W + w0) >> 2] = pc[0] + pc[1] + pc[2] + pc[3];
                }
            }
        }
        const uint32_t tsum = pc[0] + pc[1] + pc[2] + pc[3];
        // remaining levels of the tile in shared memory
        uint32_t cnt = TW >= 4u ? TW / 4u : 1u;  // nodes at the current level
        int lvl = TW >= 4u ? 2 : (TW >= 2u ? 1 : 0);
        s_lvl[0][threadIdx.x] = mine ? tsum : 0u;
        __syncthreads();
        int cur = 0;
        while (cnt > 1u) {
            cnt >>= 1;
            ++lvl;
            if (threadIdx.x < cnt) {
                const uint32_t v = s_lvl[cur][2 * threadIdx.x] + s_lvl[cur][2 * threadIdx.x + 1];
                s_lvl[cur ^ 1][threadIdx.x] = v;
                I.sums[((W + tile * TW) >> lvl) + threadIdx.x] = v;
            }
            cur ^= 1;
            __syncthreads();
        }
        // compaction of the set bits
        Pair tot;
        const Pair tex = block_scan(Pair{0, tsum}, tot, s_warp);
        const Pair ex = tile_prefix(status, tile, tot, I.g, &s_excl);
        uint32_t r = ex.b + tex.b;
        if (mine) {
            for (uint32_t k = 0; k < 4u && threadIdx.x * 4u + k < TW; ++k) {
                uint32_t m = wv[k];
                while (m) {
                    const int b = __ffs(m) - 1;
                    I.live[r++] = (w0 + k) * 32u + (uint32_t)b;
                    m &= m - 1u;
                }
            }
        }
        // last tile finished builds the top of the tree
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&I.g->done, 1u) == I.ntiles_words - 1u) ? 1u : 0u;
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (uint32_t n = I.ntiles_words >> 1; n >= 1u; n >>= 1) {
                for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
                    const uint32_t a = __ldcg(I.sums + 2u * (n + k)), b = __ldcg(I.sums + 2u * (n + k) + 1u);
                    I.sums[n + k] = a + b;
                }
                __threadfence();
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const uint32_t root = __ldcg(I.sums + 1);
                I.g->stats[kStLiveAfter] = root;
                I.g->done = 0;
            }
        }
    }
}

// ------------------------------------------------------------------ init

// Root bisectors (Sec. 3.3 "Initialization") and the root vertex table
// (Alg. 1, one FP64 centroid per face summed from its smallest halfedge).
__global__ void __launch_bounds__(kThreads) k_init(Inst I, const int32_t* twin, const int32_t* next,
                                                   const int32_t* prev, const int32_t* face,
                                                   const double* hpos) {
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
        (void)face;
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

__global__ void __launch_bounds__(kThreads) k_vertices(Inst I, FrameP fp, float* out, uint32_t cap) {
    const uint32_t N = min(I.sums[1], cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const uint32_t s = I.live[i];
        const uint64_t j = I.heap[s];
        const int d = depth_of(j, I.ch);
        const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
        float r[9];
        if (d < 0 || h >= I.H) {
            set_err(I.g, kErrLink);
            continue;
        }
        if (d <= 31) {
            uint32_t W[9], Wp[9];
            decode_weights<uint32_t>(j, d, W, Wp);
            eval_vertices<uint32_t>(W, d, fp.precision, fp.shift, I.rel, h, r);
        } else {
            unsigned long long W[9], Wp[9];
            decode_weights<unsigned long long>(j, d, W, Wp);
            eval_vertices<unsigned long long>(W, d, fp.precision, fp.shift, I.rel, h, r);
        }
        float* o = out + 9ull * i;
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = r[k];
    }
}

// ---------------------------------------------------------------- launch

void launch_prep(const Inst& I, const FrameP& fp, bool frame_start, int grid, cudaStream_t s) {
    k_prep<<<grid, kThreads, 0, s>>>(I, fp, frame_start ? 1 : 0);
}
void launch_classify(const Inst& I, const FrameP& fp, int grid, cudaStream_t s) {
    k_classify<<<grid, kThreads, 0, s>>>(I, fp);
}
void launch_gate(const Inst& I, const FrameP& fp, int grid, cudaStream_t s) {
    k_gate<<<grid, kThreads, 0, s>>>(I, fp);
}
void launch_scatter(const Inst& I, int grid, cudaStream_t s) { k_scatter<<<grid, kThreads, 0, s>>>(I); }
void launch_alloc(const Inst& I, int grid, cudaStream_t s) { k_alloc<<<grid, kThreads, 0, s>>>(I); }
void launch_free(const Inst& I, int grid, cudaStream_t s) { k_free<<<grid, kThreads, 0, s>>>(I); }
void launch_fill(const Inst& I, int grid, cudaStream_t s) { k_fill<<<grid, kThreads, 0, s>>>(I); }
void launch_cbt(const Inst& I, int grid, cudaStream_t s) { k_cbt<<<grid, kThreads, 0, s>>>(I); }
void launch_init(const Inst& I, const int32_t* twin, const int32_t* next, const int32_t* prev,
                 const int32_t* face, const double* hpos, int grid, cudaStream_t s) {
    k_init<<<grid, kThreads, 0, s>>>(I, twin, next, prev, face, hpos);
}
void launch_leaves(const Inst& I, uint32_t* slots, uint64_t* heap, uint32_t* links, int grid,
                   cudaStream_t s) {
    k_leaves<<<grid, kThreads, 0, s>>>(I, slots, heap, links);
}
void launch_vertices(const Inst& I, const FrameP& fp, float* out, uint32_t cap, int grid, cudaStream_t s) {
    k_vertices<<<grid, kThreads, 0, s>>>(I, fp, out, cap);
}

}  // namespace cbtgpu
