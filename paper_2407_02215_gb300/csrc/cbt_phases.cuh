// Device functions shared by the per-step kernels (cbt_kernels.cu) and the
// persistent one-launch-per-frame kernel (cbt_fused.cu): tile bookkeeping,
// block scans, the item-level steps of the frame and the word-tile steps
// of the CBT.
#pragma once
#include "cbt_device.cuh"

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
static __device__ Pair lookback(unsigned long long* status, uint32_t tile, Globals* g) {
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


// Entry le of an instance's camera-relative root table: the frame's eye
// subtracted in FP64, then rounded to the frame's precision (FP32, fixed
// point at 2^shift, or FP64; the sphere form keeps the absolute roots).
__device__ __forceinline__ void rel_store(const double* root64, void* rel, Globals* g, const double* eye,
                                          uint32_t precision, int32_t shift, uint32_t le) {
    const double diff = __dsub_rn(root64[le], eye[le % 3u]);
    if (precision == 1) {
        const double sc = __dmul_rn(diff, pow2d(shift));
        long long x = 0;
        if (fabs(sc) < 4.611686018427387904e18)
            x = __double2ll_rn(sc);
        else
            set_err(g, kErrRange);
        static_cast<long long*>(rel)[le] = x;
    } else if (precision == 2) {
        static_cast<double*>(rel)[le] = diff;
    } else if (precision == 3) {
        static_cast<double*>(rel)[le] = root64[le];  // absolute: the projection needs it
    } else {
        static_cast<float*>(rel)[le] = __double2float_rn(diff);
    }
}

// Entry e of the batch's root tables (instances laid out by rel_base).
__device__ __forceinline__ void rel_entry(const BatchDev& bt, uint32_t e) {
    const uint32_t b = find_inst(bt.rel_base, bt.B, e);
    const Inst& I = bt.inst[b];
    const FrameP& fp = frame_of(bt, b);
    rel_store(I.root64, I.rel, I.g, fp.eye, fp.precision, fp.shift, e - bt.rel_base[b]);
}

// Entries [e, e1) of the batch's root tables, by one warp: one instance
// lookup for the range, and the fields of the instance and its frame read
// once per instance the range crosses.
__device__ __forceinline__ void rel_range(const BatchDev& bt, uint32_t e, uint32_t e1) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t b = find_inst(bt.rel_base, bt.B, e);
    while (e < e1) {
        const uint32_t lo = bt.rel_base[b], hi = min(e1, bt.rel_base[b + 1]);
        const Inst& I = bt.inst[b];
        const FrameP& fp = frame_of(bt, b);
        const double* root64 = I.root64;
        void* rel = I.rel;
        Globals* g = I.g;
        const double eye[3] = {fp.eye[0], fp.eye[1], fp.eye[2]};
        const uint32_t precision = fp.precision;
        const int32_t shift = fp.shift;
        for (uint32_t x = e + lane; x < hi; x += 32u) rel_store(root64, rel, g, eye, precision, shift, x - lo);
        e = max(e, hi);
        ++b;
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
static __device__ bool find_group(const Inst& I, uint32_t s1, Group& g) {
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
    // the member with the smallest heap ID, by selects (the first of equal ones)
    uint64_t jm = g.j[0];
    g.imin = 0;
    if (g.j[1] < jm) {
        jm = g.j[1];
        g.imin = 1;
    }
    if (g.n == 4) {
        if (g.j[2] < jm) {
            jm = g.j[2];
            g.imin = 2;
        }
        if (g.j[3] < jm) g.imin = 3;
    }
    return true;
}

// -------------------------------------------------------------- classify

// The wishes from the bisector's camera-relative vertices r (R8 reading):
// split = visible, big and below the maximum depth; merge = no split, depth
// >= 1 and the parent not (visible and big). The parent's vertices are
// {nv, r0, r1} (nv its new vertex, from new_vertex() only when needed), its
// refinement edge (nv, r1) for an odd heap ID and (r0, nv) for an even one;
// its plane masks for r0 and r1 are the child's.
template <typename NV>
__device__ __forceinline__ void wishes_from(const float r[9], bool odd, int d, uint32_t max_depth, const FrameP& fp,
                                            NV new_vertex, bool& split, bool& merge) {
    // m01: the planes both r0 and r1 are behind (the parent's culling
    // candidates too); r2 and the parent's new vertex are tested only there
    const uint32_t m0 = plane_mask(r, fp);
    const uint32_t m01 = m0 ? plane_mask(r + 3, fp, m0) : 0u;
    const uint32_t m012 = m01 ? plane_mask(r + 6, fp, m01) : 0u;
    const bool big = edge_big(r, r + 3, fp.q);
    split = m012 == 0u && big && d < (int)max_depth;
    merge = false;
    if (!split && d >= 1) {
        float nv[3];
        new_vertex(nv);
        const bool pvis = (m01 ? plane_mask(nv, fp, m01) : 0u) == 0u;
        float a[3], b[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c] = odd ? nv[c] : r[c];
            b[c] = odd ? r[3 + c] : nv[c];
        }
        merge = !(pvis && edge_big(a, b, fp.q));
    }
}

template <typename T>
__device__ __forceinline__ void lod_wishes(const Inst& I, const FrameP& fp, uint64_t j, int d,
                                           uint32_t h, const uint32_t* tab, bool& split, bool& merge,
                                           float* keep) {
    T W[9], Wp[9];
    decode_weights<T>(j, d, W, Wp, tab);
    float r[9];
    eval_vertices<T>(W, d, fp, I.rel, h, r);
    if (keep)
#pragma unroll
        for (int k = 0; k < 9; ++k) keep[k] = r[k];
    // Two vertices of the parent are the child's: a 0 bit makes the child's
    // rows (2 r0, 2 r2, r0 + r1) of the parent's, a 1 bit (2 r2, 2 r1,
    // r0 + r1) (Eq. 1), and a row doubled over a doubled denominator
    // evaluates to the same value in every precision form. The new vertex is
    // the parent's v0 (1 bit) or v1 (0 bit); the row is picked by selects so
    // that every lane takes the same path.
    const bool odd = (j & 1ull) != 0ull;
    wishes_from(r, odd, d, I.max_depth, fp,
                [&](float nv[3]) {
                    T row[9];
#pragma unroll
                    for (int k = 0; k < 3; ++k) row[k] = odd ? Wp[k] : Wp[3 + k];
                    eval_vertex<T>(row, 0, d - 1, fp, I.rel, h, nv);
                },
                split, merge);
}

// The sphere form (R13) with a point cache attached. A vertex's FP64 point
// p and scale f depend on the heap ID, the mesh and the shape (radius and
// displacement) only, so classify keeps the four vertices the LOD test reads
// (the bisector's three, then the parent's new one) per slot, tagged with the
// heap ID and the cache generation (a new generation whenever the shape
// changes). A bisector whose slot still holds them evaluates only
// r = float(fma(p, f, -eye)) per coordinate: 24 FP64 operations in place of
// the decode, four projections with their Newton steps and the displacement.
// The floats are those of a fresh evaluation (the same operations).
template <typename T>
__device__ __forceinline__ void sphere_points(const Inst& I, const FrameP& fp, uint64_t j, int d, uint32_t h,
                                           const uint32_t* tab, uint32_t s) {
    T W[9], Wp[9];
    decode_weights<T>(j, d, W, Wp, tab);
    const double* V = static_cast<const double*>(I.rel) + 9u * h;
    const size_t cap = I.cap;
    double* pc = I.pc + s;
#pragma unroll 1
    for (int v = 0; v < 3; ++v) {
        double pf[4];
        sphere_point<T>(W, v, d, fp, V, pf);
#pragma unroll
        for (int k = 0; k < 4; ++k) pc[(size_t)(4 * v + k) * cap] = pf[k];
    }
    double pf[4] = {0.0, 0.0, 0.0, 0.0};  // a root has no parent (never read)
    if (d >= 1) {
        // the parent's new vertex: its v0 (odd heap ID) or v1 (even), as in
        // lod_wishes
        const bool odd = (j & 1ull) != 0ull;
        T row[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) row[k] = odd ? Wp[k] : Wp[3 + k];
        sphere_point<T>(row, 0, d - 1, fp, V, pf);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) pc[(size_t)(12 + k) * cap] = pf[k];
}

__device__ __forceinline__ void sphere_wishes(const Inst& I, const FrameP& fp, uint32_t s, uint64_t j, int d,
                                              uint32_t h, const uint32_t* tab, bool& split, bool& merge,
                                              float* keep) {
    const unsigned long long gen = I.g->pc_gen;
    const ulonglong2 tag = I.pct[s];
    if (tag.x != j || tag.y != gen) {
        if (d <= 31)
            sphere_points<uint32_t>(I, fp, j, d, h, tab, s);
        else
            sphere_points<unsigned long long>(I, fp, j, d, h, tab, s);
        I.pct[s] = make_ulonglong2(j, gen);
    }
    const size_t cap = I.cap;
    const double* pc = I.pc + s;
    float r[9];
#pragma unroll
    for (int v = 0; v < 3; ++v)
        sphere_rel(pc[(size_t)(4 * v) * cap], pc[(size_t)(4 * v + 1) * cap], pc[(size_t)(4 * v + 2) * cap],
                   pc[(size_t)(4 * v + 3) * cap], fp, r + 3 * v);
    if (keep)
#pragma unroll
        for (int k = 0; k < 9; ++k) keep[k] = r[k];
    wishes_from(r, (j & 1ull) != 0ull, d, I.max_depth, fp,
                [&](float nv[3]) { sphere_rel(pc[12 * cap], pc[13 * cap], pc[14 * cap], pc[15 * cap], fp, nv); },
                split, merge);
}

// A new generation of the sphere-point cache when a LOD frame of the sphere
// form has a shape (radius, displacement) other than the one the current
// generation was made with. Called for each instance by one thread, at the
// frame's start, before any classify.
__device__ __forceinline__ void pc_generation(Globals* g, const FrameP& fp) {
    if (fp.precision != 3u || fp.mode != 0u) return;
    const unsigned long long rb = (unsigned long long)__double_as_longlong(fp.radius);
    const uint32_t a = __float_as_uint(fp.damp), f = __float_as_uint(fp.dfreq);
    if (g->pc_gen == 0ull || g->pc_radius != rb || g->pc_damp != a || g->pc_dfreq != f || g->pc_doct != fp.doct ||
        g->pc_dseed != fp.dseed) {
        g->pc_gen += 1ull;
        g->pc_radius = rb;
        g->pc_damp = a;
        g->pc_dfreq = f;
        g->pc_doct = fp.doct;
        g->pc_dseed = fp.dseed;
    }
}

// Compatibility chain of bisector b on the frame-start state (command form
// of Alg. 3): returns its allocation count; with `scatter` it ORs R (and N or
// P on coarser members) into the command words. With `rec` (cost mode) it
// also records the members after b: up to four as slot | code << 30 (code
// 1 = R, 2 = R+N, 3 = R+P; 0 = no member) in x, y, z, w, or all kNull when
// the chain is longer or broken (the marking then walks it again).
__device__ __forceinline__ uint32_t chain_code_bits(uint32_t code) {
    return code == 1u ? kR : (code == 2u ? (kR | kN) : (kR | kP));
}

// With `more`, a chain of more than four members after b keeps its first
// four in rec and sets *more (else the record is all kNull).
static __device__ uint32_t chain_walk(const Inst& I, uint32_t b, int d, bool scatter, uint4* rec = nullptr,
                                      bool check = false, uint32_t* marks = nullptr, bool* more = nullptr) {
    auto mark = [&](uint32_t x, uint32_t bits) { atomicOr(marks ? marks + x : cmd_ptr(I, x), bits); };
    uint32_t cur = b, cost = 2;
    uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0, n = 0;
    bool over = false;
    auto note = [&](uint32_t t, uint32_t code) {
        const uint32_t v = t | (code << 30);
        if (n == 0)
            m0 = v;
        else if (n == 1)
            m1 = v;
        else if (n == 2)
            m2 = v;
        else if (n == 3)
            m3 = v;
        else
            over = true;
        ++n;
    };
    auto done = [&](uint32_t c, bool ok) {
        if (rec)
            *rec = (ok && (!over || more)) ? make_uint4(m0, m1, m2, m3) : make_uint4(kNull, kNull, kNull, kNull);
        if (more) *more = ok && over;
        return c;
    };
    if (scatter) mark(b, kR);
    int dcur = d;
    for (int guard = 0; guard < 64; ++guard) {
        const uint32_t t = I.nb[cur].x;
        if (t == kNull) return done(cost, true);
        if (bad_slot(I, t, kErrChain)) return done(cost, false);
        const uint4 tn = I.nb[t];
        if (tn.x == cur) {
            if (scatter) mark(t, kR);
            note(t, 1u);
            return done(cost + 2, true);
        }
        uint32_t bits;
        if (tn.y == cur) {
            bits = kR | kN;
        } else if (tn.z == cur) {
            bits = kR | kP;
        } else {
            set_err(I.g, kErrChain);
            return done(cost, false);
        }
        if (scatter) mark(t, bits);
        if ((!scatter || check) && depth_of(I.heap[t], I.ch) + 1 != dcur) {
            set_err(I.g, kErrChain);
            return done(cost, false);
        }
        note(t, bits == (kR | kN) ? 2u : 3u);
        cost += 3;
        cur = t;
        --dcur;
    }
    set_err(I.g, kErrChain);
    return done(cost, false);
}

// Split and merge wishes of bisector j (Sec. 3.3 GenerateCommands): the LOD
// reading R8 (mode 0), forced splits or merges, seeded random requests, or
// sorted request lists. Returns false when j does not decode to a root of
// this mesh.
//
// keep (optional): where the LOD test's vertices of j are stored (only the
// LOD mode evaluates them; `kept` says whether it did).
__device__ __forceinline__ bool item_wishes(const Inst& I, const FrameP& fp, uint64_t key, uint32_t s, uint64_t j,
                                            const uint32_t* tab, bool& split, bool& merge, float* keep = nullptr,
                                            bool* kept = nullptr) {
    const int d = depth_of(j, I.ch);
    const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
    split = merge = false;
    if (kept) *kept = false;
    if (d < 0 || h >= I.H) return false;
    switch (fp.mode) {
        case 0:
            if (fp.precision == 3u && I.pc)
                sphere_wishes(I, fp, s, j, d, h, tab, split, merge, keep);
            else if (d <= 31)
                lod_wishes<uint32_t>(I, fp, j, d, h, tab, split, merge, keep);
            else
                lod_wishes<unsigned long long>(I, fp, j, d, h, tab, split, merge, keep);
            if (kept) *kept = keep != nullptr;
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
    return true;
}

// With `cache` (the one-launch frame exporting sphere-form or displaced
// vertices) the LOD test's vertices go to vc[s] and the command word says so
// (kVcValid): the export then copies them instead of evaluating them again.
// With `merge_in` the word is ORed in: it was cleared before the phase and
// other bisectors' chain walks may mark it while this one classifies.
__device__ __forceinline__ uint32_t classify_item(const Inst& I, const FrameP& fp, uint64_t key, uint32_t i,
                                                  uint32_t s, uint64_t j, const uint32_t* tab, uint32_t* s_cnt,
                                                  bool cache = false, bool merge_in = false) {
    bool split, merge, kept;
    if (!item_wishes(I, fp, key, s, j, tab, split, merge, cache ? I.vc + 9ull * s : nullptr, &kept)) {
        set_err(I.g, kErrLink);
        if (!merge_in) *cmd_ptr(I, s) = 0u;
        I.scan[i] = 0u;
        return 0u;
    }
    const int d = depth_of(j, I.ch);
    const uint32_t cmd = (split ? kSplitWish : 0u) | (merge ? kMergeWish : 0u) |
                         ((d & 1) ? kDepthOdd : 0u) | ((j & 1ull) ? kHeapOdd : 0u) | (kept ? kVcValid : 0u);
    if (merge_in)
        atomicOr(cmd_ptr(I, s), cmd);
    else
        *cmd_ptr(I, s) = cmd;
    // the paper's gate charges 3d + 4 without walking the chain (k_walk
    // computes the exact chain cost otherwise)
    I.scan[i] = (split && fp.gate == 1) ? 3u * (uint32_t)d + 4u : 0u;
    count_stat(s_cnt, 0, split);
    return cmd;
}

// Pointer chases of the frame, after classify: the compatibility-chain cost
// of every split wish (command form of Alg. 3) and the Alg. 4 group of every
// merge wish with an even heap ID, whose smallest member records the members
// (for the gate, the allocation and the fill). The items that need a walk
// are packed per tile in shared memory first, so that whole warps walk.

// ------------------------------------------------------------ allocation

__device__ __forceinline__ uint32_t leaves_of(uint32_t sb) {
    return sb ? 2u + ((sb >> 1) & 1u) + ((sb >> 2) & 1u) : 0u;
}

// Gate value of a merge request at the smallest member of its group: the
// parents it allocates (1 or 2; the paper's gate charges 2) when every member
// wishes to merge, else 0.
__device__ __forceinline__ uint32_t merge_cost(const Inst& I, uint32_t i, uint32_t cmd, uint32_t gate) {
    if (!(cmd & kGrpMin)) return 0u;
    const uint4 m = I.grp[i];
    const uint32_t ms[3] = {m.y, m.z, m.w};
    uint32_t c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = ms[q] != kNull ? *cmd_ptr(I, ms[q]) : kMergeWish;
    if (!(c[0] & c[1] & c[2] & kMergeWish)) return 0u;
    return gate == 1 ? 2u : (m.z == kNull ? 1u : 2u);
}

// Fate of live index i after the chains are marked, 4 bits: its allocation
// count (0-4) and bit 3 when it is the smallest member of a valid merge group
// (granted, every member wishing to merge and none split).
__device__ __forceinline__ uint32_t alloc_fate(const Inst& I, uint32_t i, uint32_t cmd) {
    const uint32_t sb = cmd & kSplitMask;
    if (sb) return leaves_of(sb);
    if (!((cmd & kCand) && (cmd & kMergeGrant))) return 0u;
    const uint4 m = I.grp[i];
    const uint32_t ms[3] = {m.y, m.z, m.w};
    bool ok = true;
    uint32_t c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const bool bad = ms[q] != kNull && bad_slot(I, ms[q], kErrLink);
        ok = ok && !bad;
        c[q] = (ms[q] != kNull && !bad) ? *cmd_ptr(I, ms[q]) : kMergeWish;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) ok = ok && (c[q] & kMergeWish) && !(c[q] & kSplitMask);
    return ok ? ((m.z == kNull ? 1u : 2u) | 8u) : 0u;
}

// Records the free-list index `run` of a changed item's first new record: a
// split keeps it in its own dest word; a merge marks every member merged and
// gives each the index of its parent. s_cnt: split bisectors, merge groups,
// merged bisectors.
__device__ __forceinline__ void alloc_apply(const Inst& I, uint32_t i, uint32_t f, uint32_t run,
                                            uint32_t* s_cnt) {
    if (!(f & 8u)) {
        *dest_ptr(I, I.live[i]) = run;
        count_stat(s_cnt, 0, true);
        return;
    }
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
constexpr FamDesc kFam[4] = {
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

// The family tables packed into immediates, so that a lane reads its case
// from registers instead of a constant-memory table indexed differently by
// every lane: per case, the 12 edge descriptors as 5-bit codes (ext << 4 |
// a << 2 | b) at bit 5 (3 l + e); the leaf count and the per-leaf heap-ID
// shift and offset (n | shift[l] << (3 + 2 l) | off[l] << (11 + 2 l)); and
// the inverse map, old edge E and portion p to (leaf, edge) as 5-bit codes
// (valid << 4 | leaf << 2 | edge) at bit 5 (3 E + p).
constexpr uint64_t fam_edges(int c) {
    uint64_t w = 0;
    for (int l = 0; l < 4; ++l)
        for (int e = 0; e < 3; ++e) {
            const EdgeDesc d = kFam[c].e[l][e];
            w |= (uint64_t)((d.ext << 4) | (d.a << 2) | d.b) << (5 * (3 * l + e));
        }
    return w;
}
constexpr uint32_t fam_misc(int c) {
    uint32_t w = kFam[c].n;
    for (int l = 0; l < 4; ++l) w |= (uint32_t)kFam[c].shift[l] << (3 + 2 * l) | (uint32_t)kFam[c].off[l] << (11 + 2 * l);
    return w;
}
constexpr uint64_t fam_leafof(int c) {
    uint64_t w = 0;
    for (int l = 0; l < kFam[c].n; ++l)
        for (int e = 0; e < 3; ++e) {
            const EdgeDesc d = kFam[c].e[l][e];
            if (d.ext) w |= (uint64_t)(16 | (l << 2) | e) << (5 * (3 * d.a + d.b));
        }
    return w;
}
constexpr uint64_t kFamE0 = fam_edges(0), kFamE1 = fam_edges(1), kFamE2 = fam_edges(2), kFamE3 = fam_edges(3);
constexpr uint32_t kFamM0 = fam_misc(0), kFamM1 = fam_misc(1), kFamM2 = fam_misc(2), kFamM3 = fam_misc(3);
constexpr uint64_t kFamL0 = fam_leafof(0), kFamL1 = fam_leafof(1), kFamL2 = fam_leafof(2), kFamL3 = fam_leafof(3);

template <typename T>
__device__ __forceinline__ T pick_case(int c, T v0, T v1, T v2, T v3) {
    return c == 0 ? v0 : (c == 1 ? v1 : (c == 2 ? v2 : v3));
}

__device__ __forceinline__ int fam_case(uint32_t sb) { return (int)((sb >> 1) & 3u); }

// Does a family with split bits sb cover old edge E by halves?
__device__ __forceinline__ bool halves(uint32_t sb, int E) {
    return E == kT || (E == kNe && (sb & kN)) || (E == kPe && (sb & kP));
}

// Leaf of family `sb` covering portion p of old edge Ep, and that leaf's edge.
__device__ __forceinline__ bool family_leaf(uint32_t sb, int Ep, int p, uint32_t& leaf, uint32_t& edge) {
    const uint32_t code =
        (uint32_t)(pick_case(fam_case(sb), kFamL0, kFamL1, kFamL2, kFamL3) >> (5 * (3 * Ep + p))) & 31u;
    leaf = (code >> 2) & 3u;
    edge = code & 3u;
    return (code & 16u) != 0u;
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

__device__ __forceinline__ void set_bit(const Inst& I, uint32_t s) {
    atomicOr(I.bits + (s >> 5), 1u << (s & 31u));
}
__device__ __forceinline__ void clear_bit(const Inst& I, uint32_t s) {
    atomicAnd(I.bits + (s >> 5), ~(1u << (s & 31u)));
}

// How the fill reads a destination word and updates the bitfield: here the
// word is the free-list index itself and A the frame's allocation count
// (the single-instance frame has a form that resolves tile-local words).
struct DestPlain {
    uint32_t A;
    __device__ __forceinline__ uint32_t operator()(uint32_t d) const { return d; }
    __device__ __forceinline__ void set(const Inst& I, uint32_t s) const { set_bit(I, s); }
    __device__ __forceinline__ void clear(const Inst& I, uint32_t s) const { clear_bit(I, s); }
};

// Resolves old edge E of x (depth parity xodd), whole (hv = false) or by
// halves: a split neighbour gives the leaf of its family on the same
// portion, a merged one its parent, an unchanged one itself (R11 reading).
template <typename DM>
static __device__ void across_resolve(const Inst& I, Across& a, int E, bool hv, bool xodd, const DM& dm) {
    const uint32_t y = a.y[E];
    a.slot[E][0] = a.slot[E][1] = kNull;
    a.rev[E][0] = a.rev[E][1] = 3u;
    if (y == kNull) return;
    const int Ep = (int)a.ep[E];
    const uint2 yc = a.yc[E];
    const uint32_t ysb = yc.x & kSplitMask;
    const uint32_t A = dm.A;
    if (Ep > 2) {
        set_err(I.g, kErrLink);
        return;
    }
    if (ysb) {
        const uint32_t yd = dm(yc.y);
        const bool same = ((yc.x & kDepthOdd) != 0u) == xodd;
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // unrolled: a.slot and a.rev stay in registers
            if (h == 1 && !hv) break;
            int p = hv ? (h == 0 ? kFirst : kSecond) : kWhole;
            if (p != kWhole && same) p = p == kFirst ? kSecond : kFirst;
            uint32_t leaf, edge;
            if (!family_leaf(ysb, Ep, p, leaf, edge) || yd + leaf >= A) {
                set_err(I.g, kErrLink);
                continue;
            }
            a.slot[E][h] = I.freel[yd + leaf];
            a.rev[E][h] = edge;
        }
    } else if (yc.x & kMerged) {
        const uint32_t yd = dm(yc.y);
        if (hv || Ep != kT || yd >= A) {
            set_err(I.g, kErrLink);
            return;
        }
        a.slot[E][0] = I.freel[yd];
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

// Element i (0..2) of three values, by selects (no indexed local array).
__device__ __forceinline__ uint32_t sel3(uint32_t i, uint32_t v0, uint32_t v1, uint32_t v2) {
    return i == 0u ? v0 : (i == 1u ? v1 : v2);
}

// An unchanged neighbour across old edge E of x now faces new bisector ns
// through ns's edge ne; that neighbour link has exactly one writer, this one.
// Returns the number of links written (0 or 1).
__device__ __forceinline__ uint32_t push_keep(const Inst& I, const Across& a, int E, uint32_t ns, uint32_t ne) {
    const uint32_t e = (uint32_t)E;
    const uint32_t y = sel3(e, a.y[0], a.y[1], a.y[2]);
    const uint32_t ycx = sel3(e, a.yc[0].x, a.yc[1].x, a.yc[2].x);
    if (y == kNull || (ycx & (kSplitMask | kMerged))) return 0u;
    uint32_t* yr = reinterpret_cast<uint32_t*>(I.nb + y);
    const uint32_t Ep = sel3(e, a.ep[0], a.ep[1], a.ep[2]);
    yr[Ep] = ns;
    atomicXor(yr + 3, (e ^ ne) << (2u * Ep));
    return 1u;
}


// Both fills return the number of unchanged neighbours relinked; dest is
// the free-list index of the first new record.
template <typename DM = DestPlain>
static __device__ uint32_t fill_split(const Inst& I, uint32_t s, uint32_t cmd, uint32_t dest, const DM& dm) {
    const uint32_t sb = cmd & kSplitMask;
    const int fc = fam_case(sb);
    const uint64_t edges = pick_case(fc, kFamE0, kFamE1, kFamE2, kFamE3);
    const uint32_t misc = pick_case(fc, kFamM0, kFamM1, kFamM2, kFamM3);
    const uint32_t n = misc & 7u;
    if (dest + n > dm.A) {
        set_err(I.g, kErrOverflow);
        return 0u;
    }
    const uint64_t j = I.heap[s];
    const uint4 rx = I.nb[s];
    uint32_t slots[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) slots[l] = (uint32_t)l < n ? I.freel[dest + (uint32_t)l] : 0u;
    Across a;
    across_load(I, rx, a);
    const bool xodd = (cmd & kDepthOdd) != 0u;
#pragma unroll
    for (int E = 0; E < 3; ++E) across_resolve(I, a, E, halves(sb, E), xodd, dm);
#pragma unroll
    for (int l = 0; l < 4; ++l)
        if ((uint32_t)l < n && bad_slot(I, slots[l], kErrOverflow)) return 0u;
    uint32_t relinked = 0;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if ((uint32_t)l >= n) break;
        uint32_t lk[3], rv = 0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const uint32_t code = (uint32_t)(edges >> (5 * (3 * l + e))) & 31u;
            const uint32_t ea = (code >> 2) & 3u, eb = code & 3u;
            uint32_t r;
            if (!(code & 16u)) {
                lk[e] = ea == 0u ? slots[0] : (ea == 1u ? slots[1] : (ea == 2u ? slots[2] : slots[3]));
                r = eb;
            } else {
                const bool h = eb == (uint32_t)kSecond;
                lk[e] = sel3(ea, h ? a.slot[0][1] : a.slot[0][0], h ? a.slot[1][1] : a.slot[1][0],
                             h ? a.slot[2][1] : a.slot[2][0]);
                r = sel3(ea, h ? a.rev[0][1] : a.rev[0][0], h ? a.rev[1][1] : a.rev[1][0],
                         h ? a.rev[2][1] : a.rev[2][0]);
                if (eb == (uint32_t)kWhole) relinked += push_keep(I, a, (int)ea, slots[l], (uint32_t)e);
            }
            rv |= r << (2 * e);
        }
        const uint32_t sh = (misc >> (3 + 2 * l)) & 3u, off = (misc >> (11 + 2 * l)) & 3u;
        I.nb[slots[l]] = make_uint4(lk[0], lk[1], lk[2], rv);
        I.heap[slots[l]] = (j << sh) + off;
        *cmd_ptr(I, slots[l]) = 0u;  // a new record: no cached vertices
        dm.set(I, slots[l]);
    }
    return relinked;
}

// One old edge of a merged child on the new mesh, taken whole: the
// neighbour y across it (its edge facing the child, command word and
// destination), then the parent's new neighbour there and that neighbour's
// edge facing the parent (across_load and across_resolve for one edge).
struct Edge1 {
    uint32_t y, ep;
    uint2 yc;
    uint32_t slot, rev;
};

__device__ __forceinline__ void edge_load(const Inst& I, const uint4& rx, int E, Edge1& a) {
    a.y = link_of(rx, E);
    a.ep = (rx.w >> (2 * E)) & 3u;
    a.yc = make_uint2(0u, 0u);
    if (a.y != kNull && !bad_slot(I, a.y, kErrLink))
        a.yc = I.cd[a.y];
    else
        a.y = kNull;
}

template <typename DM>
__device__ __forceinline__ void edge_resolve(const Inst& I, Edge1& a, const DM& dm) {
    a.slot = kNull;
    a.rev = 3u;
    if (a.y == kNull) return;
    const int Ep = (int)a.ep;
    const uint32_t ysb = a.yc.x & kSplitMask;
    if (Ep > 2) {
        set_err(I.g, kErrLink);
        return;
    }
    if (ysb) {
        const uint32_t yd = dm(a.yc.y);
        uint32_t leaf, edge;
        if (!family_leaf(ysb, Ep, kWhole, leaf, edge) || yd + leaf >= dm.A) {
            set_err(I.g, kErrLink);
            return;
        }
        a.slot = I.freel[yd + leaf];
        a.rev = edge;
    } else if (a.yc.x & kMerged) {
        const uint32_t yd = dm(a.yc.y);
        if (Ep != kT || yd >= dm.A) {
            set_err(I.g, kErrLink);
            return;
        }
        a.slot = I.freel[yd];
        a.rev = (a.yc.x & kHeapOdd) ? (uint32_t)kNe : (uint32_t)kPe;
    } else {
        a.slot = a.y;
        a.rev = (uint32_t)Ep;
    }
}

// push_keep for one edge E taken whole.
__device__ __forceinline__ uint32_t push_keep1(const Inst& I, const Edge1& a, uint32_t E, uint32_t ns, uint32_t ne) {
    if (a.y == kNull || (a.yc.x & (kSplitMask | kMerged))) return 0u;
    uint32_t* yr = reinterpret_cast<uint32_t*>(I.nb + a.y);
    yr[a.ep] = ns;
    atomicXor(yr + 3, (E ^ ne) << (2u * a.ep));
    return 1u;
}

// Parents of a valid merge group (Alg. 4), written by its smallest member:
// Next = across child 2p+1's Twin edge, Prev = across child 2p's Twin edge,
// Twin = the other parent (Table 1 read backwards, Alg. 6). Members m0, m1
// are the children of the smaller parent, m2, m3 of the other one. Both
// parents' reads go out in three rounds (the members' records, the
// neighbours across their Twin edges, those neighbours' new records) before
// any write, so that a group costs three dependent loads, not six.
template <typename DM = DestPlain>
static __device__ uint32_t fill_merge(const Inst& I, uint32_t dest, const uint4 m, const DM& dm) {
    const uint32_t ms[4] = {m.x, m.y, m.z, m.w};
    const int np = m.z == kNull ? 1 : 2;
    if (dest + (uint32_t)np > dm.A) {
        set_err(I.g, kErrOverflow);
        return 0u;
    }
    uint32_t ps[2] = {kNull, kNull};
    uint64_t ju[2] = {0ull, 0ull};
    uint4 ru[2], rv[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // unrolled loops keep everything in registers
        if (k == np) break;
        ps[k] = I.freel[dest + (uint32_t)k];
        const uint32_t u = ms[2 * k], v = ms[2 * k + 1];
        if (bad_slot(I, u, kErrLink) || bad_slot(I, v, kErrLink)) return 0u;
        ju[k] = I.heap[u];
        ru[k] = I.nb[u];
        rv[k] = I.nb[v];
    }
    Edge1 xa[2], xb[2];  // across child 2p's and child 2p+1's Twin edges
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == np) break;
        if (bad_slot(I, ps[k], kErrOverflow)) return 0u;
        const bool odd = (ju[k] & 1ull) != 0ull;  // u is child 2p+1
        edge_load(I, odd ? rv[k] : ru[k], kT, xa[k]);
        edge_load(I, odd ? ru[k] : rv[k], kT, xb[k]);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == np) break;
        edge_resolve(I, xb[k], dm);
        edge_resolve(I, xa[k], dm);
    }
    uint32_t relinked = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == np) break;
        relinked += push_keep1(I, xb[k], (uint32_t)kT, ps[k], (uint32_t)kNe);
        relinked += push_keep1(I, xa[k], (uint32_t)kT, ps[k], (uint32_t)kPe);
        const uint32_t tw = np == 2 ? ps[1 - k] : kNull;
        const uint32_t rvT = np == 2 ? (uint32_t)kT : 3u;
        I.nb[ps[k]] = make_uint4(tw, xb[k].slot, xa[k].slot, rvT | (xb[k].rev << 2) | (xa[k].rev << 4));
        I.heap[ps[k]] = ju[k] >> 1;
        *cmd_ptr(I, ps[k]) = 0u;  // a new record: no cached vertices
        dm.set(I, ps[k]);
    }
    return relinked;
}

// FillNewBlocks + UpdateNeighbors + UpdateBitfield for the changed
// bisectors, one per thread over the instance's compacted list (written in
// ascending slot order by k_alloc): a split bisector clears its bit and
// writes its family; the smallest member of a merge group clears its
// members' bits and writes the parents.

// The three vertices of bisector j into r; false (error word set, r not
// written) when j does not decode to a root of this mesh.
__device__ __forceinline__ bool vertex_eval(const Inst& I, const FrameP& fp, uint64_t j, const uint32_t* tab,
                                            float r[9]) {
    const int d = depth_of(j, I.ch);
    const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
    if (d < 0 || h >= I.H) {
        set_err(I.g, kErrLink);
        return false;
    }
    if (d <= 31) {
        uint32_t W[9], Wp[9];
        decode_weights<uint32_t>(j, d, W, Wp, tab);
        eval_vertices<uint32_t>(W, d, fp, I.rel, h, r);
    } else {
        unsigned long long W[9], Wp[9];
        decode_weights<unsigned long long>(j, d, W, Wp, tab);
        eval_vertices<unsigned long long>(W, d, fp, I.rel, h, r);
    }
    return true;
}

__device__ __forceinline__ void vertex_item(const Inst& I, const FrameP& fp, uint32_t i, uint64_t j,
                                            const uint32_t* tab, float* out) {
    float r[9];
    if (!vertex_eval(I, fp, j, tab, r)) return;
    float* o = out + 9ull * i;
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = r[k];
}

// A warp's 32 consecutive output rows of 9 floats (rows row0 .. row0 + 31,
// the first `valid` of them real), written through the warp's 288-float
// staging area (16-byte aligned): lane l's row goes to stage[9 l ..] (odd
// stride, no bank conflicts), then the warp stores the rows' words with
// 16-byte stores when their first word is 16-byte aligned (else word by
// word). One row of 36 bytes per lane would take nine strided stores per
// warp.
__device__ __forceinline__ void warp_rows_out(const float r[9], float* stage, float* out, uint64_t row0,
                                              uint32_t valid) {
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int k = 0; k < 9; ++k) stage[9u * lane + (uint32_t)k] = r[k];
    __syncwarp();
    const uint32_t words = 9u * valid;
    float* dst = out + 9ull * row0;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0u) {
        const uint32_t nv = words >> 2;
        for (uint32_t v = lane; v < nv; v += 32u)
            reinterpret_cast<float4*>(dst)[v] = reinterpret_cast<const float4*>(stage)[v];
        done = nv << 2;
    }
    for (uint32_t w = done + lane; w < words; w += 32u) dst[w] = stage[w];
    __syncwarp();
}

// Vertices of the live bisector in slot s at output row i: in the sphere
// and displaced forms copied from the frame's cache when the LOD test stored
// them, else evaluated.
__device__ __forceinline__ void vertex_item_cached(const Inst& I, const FrameP& fp, uint32_t i, uint32_t s,
                                                   const uint32_t* tab, float* out) {
    if (vc_form(fp) && (*cmd_ptr(I, s) & kVcValid)) {
        const float* src = I.vc + 9ull * s;
        float* o = out + 9ull * i;
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = src[k];
    } else {
        vertex_item(I, fp, i, I.heap[s], tab, out);
    }
}


}  // namespace cbtgpu
