// Device-side data layout and helpers of the CBT bisection update.
//
// Per instance (one halfedge mesh, one pool of 2^D slots) the workspace holds:
//   heap[cap]  u64   bisector heap ID j (Sec. 2.3; root of h = 2^ch + h)
//   nb[cap]    uint4 {Twin, Next, Prev, rev}: neighbour slots across the edges
//                    (v0,v1), (v1,v2), (v2,v0); rev holds, per link, which edge
//                    of the neighbour points back (2 bits each, 3 = none)
//   cd[cap]    uint2 {cmd, dest}: per-frame command word and the index into
//                    the free list of the bisector's first new record
//   bits[W]    u32   CBT bitfield, W = max(1, cap / 32) words
//   sums[2W]   u32   CBT sum tree above the words in heap order: sums[1] is the
//                    root, sums[W + w] = popc(bits[w]) (Sec. 3.1)
//   live[cap]  u32   slots of the live bisectors, ascending (Alg. 7 for all i)
//   freel[cap] u32   the first A zero bits of the frame-start bitfield (Alg. 8)
//   scan[cap]  u32   per live index: split cost, then its running total
//   grp[cap]   uint4 per live index: the members of the merge group whose
//                    smallest member it is, or of a split wish's chain
//   chg[cap]   u32   live indices of the frame's changed bisectors, ascending
//   chgr[cap]  uint4 the same as records {live index, slot, cmd, dest}
//   vc[cap]    9 x f32 in the sphere and displaced forms, the vertices the LOD test
//                    evaluated this frame (valid while the slot's cmd has
//                    kVcValid), copied by the vertex export
// and, when a point cache is attached (caller memory of its own):
//   pc[16][cap] f64  sphere form: per slot the frame-independent part of the
//                    LOD test's four vertices (its three and the parent's new
//                    one), {p_x, p_y, p_z, f} each (component-major: entry k
//                    of slot s at pc[k cap + s])
//   pct[cap]   u64x2 the tag of pc[.][s]: {heap ID, cache generation}
//   root64[H*9], rel[H*9]: root vertices (FP64) and their per-frame offsets
//                    from the camera (FP32, fixed point or FP64)
//   corner[H*3] u32  global points of the root corners (mesh vertex ids, and
//                    V + face id for the face centroid), for the indexed export
// and, per batch (a single instance carries a batch of one), the instance
// table, per-instance frame parameters, tile prefixes and the look-back
// tile descriptors of the two scans and the reduction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cbtgpu {

constexpr uint32_t kNull = 0xFFFFFFFFu;

// cmd word bits.
constexpr uint32_t kR = 1u, kN = 2u, kP = 4u;  // split bits (R5 reading)
constexpr uint32_t kSplitMask = 7u;
constexpr uint32_t kMerged = 1u << 3;
constexpr uint32_t kSplitWish = 1u << 4;
constexpr uint32_t kMergeWish = 1u << 5;
constexpr uint32_t kMergeGrant = 1u << 6;
constexpr uint32_t kDepthOdd = 1u << 7;
constexpr uint32_t kHeapOdd = 1u << 8;
constexpr uint32_t kCand = 1u << 9;    // smallest member of a mergeable group (members in grp[i])
constexpr uint32_t kGrpMin = 1u << 10; // smallest member of a merge group whose members are in grp[i]
constexpr uint32_t kVcValid = 1u << 11; // vc[slot] holds this frame's vertices (sphere or displaced form, one-launch frame)
// scan word of a live index: split cost in bits 0-23, merge cost in bits
// 24-30, and (single-instance frame) bit 31 when the split's chain has more
// members than its record keeps
constexpr uint32_t kScanMore = 1u << 31;
constexpr uint32_t kMergeCostMask = 0x7Fu;

// Edge indices of a bisector: Twin (v0,v1), Next (v1,v2), Prev (v2,v0).
constexpr int kT = 0, kNe = 1, kPe = 2;
// Portion of an old edge covered by a new edge: whole, the half at the
// edge's first vertex, the half at its second vertex (in the bisector's own
// vertex order: Twin v0->v1, Next v1->v2, Prev v2->v0).
constexpr int kWhole = 0, kFirst = 1, kSecond = 2;

// Device error bits (mirrors CBT_DERR_*).
constexpr uint32_t kErrChain = 1u, kErrLink = 2u, kErrTimeout = 4u, kErrRange = 8u,
                   kErrOverflow = 16u;

enum StatIdx {
    kStLiveBefore = 0, kStLiveAfter, kStFreeBefore, kStSplitWishes, kStMergeCand,
    kStSplitGranted, kStMergeGranted, kStSplitBis, kStMergedBis, kStMergeGroups,
    kStAllocated, kStRelinked, kStFrame, kStCount
};

// Per-instance counters (256 bytes at the start of the instance workspace).
struct Globals {
    uint32_t N;         // live bisectors at frame start (CBT root)
    uint32_t F;         // free slots at frame start
    uint32_t A;         // allocations of this frame
    uint32_t Mg;        // granted merge cost of this frame
    uint32_t err;       // sticky error bits
    uint32_t done;      // finished word tiles of the reduction
    uint32_t ntiles;    // item tiles of this frame: ceil(N / kTileItems)
    uint32_t C;         // changed bisectors of this frame (split, or smallest member of a merge)
    uint32_t nstiles;   // scan tiles of this frame: ceil(N / kScanItems)
    uint32_t Stot;      // total split cost requested this frame (one-launch frame)
    uint32_t stats[kStCount];
    uint32_t pc_pad;
    unsigned long long pc_gen;     // sphere-point cache generation (0: none made yet)
    unsigned long long pc_radius;  // the shape it was made with: radius (FP64 bits),
    uint32_t pc_damp, pc_dfreq, pc_doct, pc_dseed;  // displacement (FP32 bits)
    // single-instance frame: the frame's merge cost (groups whose members all
    // wish to merge) and requested split cost, summed by the walks; when their
    // sum fits the free slots every request is granted without the prefix gate
    unsigned long long rq_merge, rq_split;
    uint32_t nwalk;  // single-instance frame: entries of the frame's walk list
    uint32_t marks_clean;  // 1 when the chain-mark words (chg) of the live slots are 0 (the
                           // single-instance frame leaves them so; the other frames clear this)
    uint32_t freel_full;   // 1 when freel lists every zero bit of the bitfield in slot order
                           // (the single-instance frame leaves it so; the other frames clear this)
    uint32_t pad[64 - 39];
};
static_assert(sizeof(Globals) == 256, "Globals must be 256 bytes");
static_assert(10 + kStCount + 1 == 24, "pc_gen must sit at byte 96");

// Per-instance device arrays and sizes.
struct Inst {
    uint64_t* heap;
    uint4* nb;
    uint2* cd;
    uint32_t* bits;
    uint32_t* sums;
    uint32_t* live;
    uint32_t* freel;
    uint32_t* scan;
    uint4* grp;  // per live index: members of the group whose smallest member it is
    uint32_t* chg;  // live indices of the changed bisectors, in ascending slot order
    uint4* chgr;    // one-launch frame: per changed bisector {live index, slot, cmd, dest}
    float* vc;      // per slot, the frame's FP32 vertices [3][3] (sphere form, one-launch frame)
    double* pc;     // optional point cache (sphere form): per slot {p, f} of the LOD test's four vertices, [16][cap]
    ulonglong2* pct;  // tag of pc[.][s]: {heap ID, generation}; both null without a cache
    double* root64;
    void* rel;
    Globals* g;
    uint32_t cap, W, D, H, ch, max_depth;
    uint32_t ntiles_items;  // ceil(cap / kTileItems)
    uint32_t pad_;
    const uint32_t* rbnd;   // bit h: halfedge h has no Twin (mesh boundary), [ceil(H / 32)]
};

struct FrameP {
    double eye[3];
    float planes[15];
    float q;
    uint32_t nplanes, mode, seed, precision;
    int32_t shift;
    uint32_t gate;
    const uint64_t* split_list;
    uint32_t n_split;
    const uint64_t* merge_list;
    uint32_t n_merge;
    uint32_t frame;  // frame counter (RANDOM mode key)
    float* vout;     // optional vertex export, vcap rows of 9 floats
    uint32_t vcap;
    double radius;   // precision 3: radius of the sphere about the world origin
    float damp;      // displacement amplitude (0: none), precisions 0 and 3
    float dfreq;     // displacement base frequency (lattice cells per unit)
    uint32_t doct;   // displacement octaves (1..8)
    uint32_t dseed;  // displacement lattice seed
};

constexpr int kFramePhases = 10;  // phases of the one-launch frame (a batch skips the last)

// Launch-wide counters of one batch (256 bytes).
struct BatchGlobals {
    uint32_t tickets[8];
    uint32_t total_tiles;   // item tiles of this frame over all instances
    uint32_t total_ctiles;  // tiles of changed bisectors (kThreads each) over all instances
    uint32_t total_stiles;  // scan tiles (kScanItems each) over all instances
    uint32_t bar_count;     // grid barrier of the one-launch frame: arrivals (monotonic),
    uint32_t bar_epoch;     // and their count when the current launch started
    uint32_t abort;         // a bounded wait ran out: later waits return at once
    uint32_t scan_ipt;      // one-launch frame: items per thread of its scan tiles
    uint32_t live_total;    // live bisectors of the batch at frame start (saturating)
    unsigned long long t[16];  // phase boundaries (ns) of the one-launch frame
    uint32_t pad[64 - 16 - 32];
};
static_assert(sizeof(BatchGlobals) == 256, "BatchGlobals must be 256 bytes");

// A batch of independent instances updated by one launch per kernel. Item
// tiles of instance b are the global tiles [tile_base[b], tile_base[b+1])
// (recomputed on the device every frame from the live counts); word tiles
// and vertex tiles use static prefixes. A single instance is a batch of one.
struct BatchDev {
    const Inst* inst;     // [B]
    const FrameP* fps;    // [B] in device memory, or null: fp0 for every instance
    FrameP fp0;
    Inst inst0;           // B == 1: a copy of inst[0] (read from the launch's parameters)
    uint32_t B;
    uint32_t tw;          // word-tile size of the reduction and free-list kernels
    uint32_t* tile_base;  // [B+1]
    uint32_t* ctile_base; // [B+1] tiles of kThreads changed bisectors, per frame
    uint32_t* stile_base; // [B+1] scan tiles of kScanItems live bisectors, per frame
    const uint32_t* wtile_base;  // [B+1] word tiles, min(W_b, tw) words each
    const uint32_t* vtile_base;  // [B+1] ceil(cap_b / kTileItems)
    const uint32_t* rel_base;    // [B+1] 9 * H_b
    BatchGlobals* bg;
    unsigned long long* status;  // [2 * Titems + Twords] look-back descriptors
    uint32_t Titems, Twords, Trel;
    uint32_t* nout;              // optional [B]: live count at frame start per instance
    uint32_t timing;             // one-launch frame: record phase boundaries
    uint32_t* tpre;              // single-instance frame: [2][Twords] ones before each word tile of
                                 // the next frame's starting bitfield, by frame parity
};

constexpr int kThreads = 256;
constexpr int kItemsPerThread = 4;
constexpr uint32_t kTileItems = kThreads * kItemsPerThread;  // 1024 live indices
// The two look-back scans use larger tiles, so that fewer tiles chain.
constexpr int kScanThreads = 512;
constexpr int kScanPerThread = 8;
constexpr uint32_t kScanItems = kScanThreads * kScanPerThread;  // 4096 live indices
constexpr uint32_t kMaxTileWords = 256;                       // up to 8192 bits per tile
constexpr uint32_t kMinTileWords = 64;

// ------------------------------------------------------------------ bits

__device__ __forceinline__ int bitlen64(uint64_t x) { return 64 - __clzll((long long)x); }
__device__ __forceinline__ int depth_of(uint64_t j, uint32_t ch) { return bitlen64(j) - 1 - (int)ch; }

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    // SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based hash.
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2d(int e) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ void set_err(Globals* g, uint32_t e) { atomicOr(&g->err, e); }

// ------------------------------------------------- Alg. 2 / Eq. 1 decode

// Integer form of Alg. 2 evaluated from the first split down: with W the
// weights over 2^k after k levels, a 0 bit maps the rows (r0, r1, r2) to
// (2 r0, 2 r2, r0 + r1) and a 1 bit to (2 r2, 2 r1, r0 + r1) (Eq. 1 times 2),
// i.e. W <- T_b W with T_0 = 2 M_0 and T_1 = 2 M_1. Eight levels at once are
// W <- P_c W with P_c = T_{c7} T_{c6} ... T_{c0} for the eight path bits c
// (most significant applied first), precomputed below for all 256 c; every
// entry of P_c is at most 2^8 (16 bits). Every row of W sums to 2^k (the
// rows of M are barycentric), so only the first two columns are carried
// and the third is 2^k minus them. W = 2^d M exactly while entries fit T
// (T = u32 for d <= 31). The first r < 8 levels from the identity are the
// first two columns of the r-level product, tabulated too (q: r-level
// entries for the 2^r prefixes c at q[2^r - 2 + c]).
struct alignas(16) DecTable {
    uint16_t p[256][9];
    uint16_t q[256][6];  // 254 used
};

constexpr void dec_product(int c, int levels, uint32_t m[9]) {
    for (int e = 0; e < 9; ++e) m[e] = (e % 4 == 0) ? 1u : 0u;
    for (int k = levels - 1; k >= 0; --k) {
        const int b = (c >> k) & 1;
        uint32_t n[9] = {};
        for (int col = 0; col < 3; ++col) {
            n[6 + col] = m[col] + m[3 + col];
            n[col] = 2u * (b ? m[6 + col] : m[col]);
            n[3 + col] = 2u * (b ? m[3 + col] : m[6 + col]);
        }
        for (int e = 0; e < 9; ++e) m[e] = n[e];
    }
}

constexpr DecTable make_dec8() {
    DecTable t{};
    for (int c = 0; c < 256; ++c) {
        uint32_t m[9] = {};
        dec_product(c, 8, m);
        for (int e = 0; e < 9; ++e) t.p[c][e] = static_cast<uint16_t>(m[e]);
    }
    for (int r = 1; r < 8; ++r)
        for (int c = 0; c < (1 << r); ++c) {
            uint32_t m[9] = {};
            dec_product(c, r, m);
            for (int row = 0; row < 3; ++row)
                for (int col = 0; col < 2; ++col)
                    t.q[(1 << r) - 2 + c][2 * row + col] = static_cast<uint16_t>(m[3 * row + col]);
        }
    return t;
}

// In global memory, not constant memory: the copy below reads it with a
// different address in every lane, which the constant cache serializes.
__device__ const DecTable g_dec8 = make_dec8();
constexpr uint32_t kDecTabWords = sizeof(DecTable) / 4u;  // the table in 32-bit words
static_assert(sizeof(DecTable) % 16u == 0u, "the table is copied 16 bytes at a time");

// Copies the tables into shared memory (kDecTabWords words, s_tab 16-byte
// aligned; call with the whole block, then __syncthreads()).
__device__ __forceinline__ void load_dec6(uint32_t* s_tab) {
    const uint4* src = reinterpret_cast<const uint4*>(&g_dec8.p[0][0]);
    for (uint32_t k = threadIdx.x; k < kDecTabWords / 4u; k += blockDim.x)
        reinterpret_cast<uint4*>(s_tab)[k] = __ldg(src + k);
}
// The same copy in two halves (blocks of 256 threads): the loads into
// registers, then the stores, so that other loads can go out in between.
constexpr uint32_t kDecVecs = kDecTabWords / 4u;
__device__ __forceinline__ void dec_fetch(uint4 (&r)[kDecVecs / 256u + 1u]) {
    const uint4* src = reinterpret_cast<const uint4*>(&g_dec8.p[0][0]);
#pragma unroll
    for (uint32_t k = 0; k < kDecVecs / 256u + 1u; ++k) {
        const uint32_t i = threadIdx.x + 256u * k;
        r[k] = i < kDecVecs ? __ldg(src + i) : make_uint4(0u, 0u, 0u, 0u);
    }
}
__device__ __forceinline__ void dec_store(uint32_t* s_tab, const uint4 (&r)[kDecVecs / 256u + 1u]) {
#pragma unroll
    for (uint32_t k = 0; k < kDecVecs / 256u + 1u; ++k) {
        const uint32_t i = threadIdx.x + 256u * k;
        if (i < kDecVecs) reinterpret_cast<uint4*>(s_tab)[i] = r[k];
    }
}

// One level on the first two columns, a[2 r + c] (c = 0, 1).
template <typename T>
__device__ __forceinline__ void dec_step(T a[6], bool b) {
    T n[6];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        n[4 + c] = a[c] + a[2 + c];
        n[c] = (b ? a[4 + c] : a[c]) << 1;
        n[2 + c] = (b ? a[2 + c] : a[4 + c]) << 1;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = n[k];
}

template <typename T>
__device__ __forceinline__ void dec_chunk(T a[6], const uint16_t* P) {
    T n[6];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const T p0 = P[3 * r], p1 = P[3 * r + 1], p2 = P[3 * r + 2];
#pragma unroll
        for (int c = 0; c < 2; ++c) n[2 * r + c] = p0 * a[c] + p1 * a[2 + c] + p2 * a[4 + c];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = n[k];
}

// The 3 x 3 weights from the first two columns at 2^k.
template <typename T>
__device__ __forceinline__ void dec_expand(const T a[6], T pw, T W[9]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        W[3 * r] = a[2 * r];
        W[3 * r + 1] = a[2 * r + 1];
        W[3 * r + 2] = pw - a[2 * r] - a[2 * r + 1];
    }
}

// W = weights of bisector j at depth d, Wp = those of its parent (d >= 1);
// tab = the eight-level table in shared memory.
template <typename T>
__device__ __forceinline__ void decode_weights(uint64_t j, int d, T W[9], T Wp[9], const uint32_t* tab) {
    const uint16_t* tab16 = reinterpret_cast<const uint16_t*>(tab);
    T a[6] = {1, 0, 0, 1, 0, 0};
    if (d >= 1) {
        int lvl = d - 1;  // path bit applied next; the parent covers bits d-1 .. 1
        const int rem = (d - 1) & 7;
        if (rem) {  // the first rem levels from the identity: one lookup
            const uint32_t c = (uint32_t)((j >> (lvl - rem + 1)) & ((1ull << rem) - 1ull));
            const uint16_t* Q = tab16 + 256u * 9u + 6u * ((1u << rem) - 2u + c);
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] = Q[k];
            lvl -= rem;
        }
#pragma unroll 1
        for (; lvl >= 8; lvl -= 8) dec_chunk<T>(a, tab16 + 9u * (uint32_t)((j >> (lvl - 7)) & 255ull));
        dec_expand<T>(a, (T)1 << (d - 1), Wp);
        dec_step<T>(a, j & 1ull);
    } else {
        dec_expand<T>(a, (T)1, Wp);
    }
    dec_expand<T>(a, (T)1 << d, W);
}

// Round-to-nearest conversion of a weight to FP32 / FP64 (exact below 2^24 /
// 2^53; the 32-bit forms for 32-bit weights).
__device__ __forceinline__ float wfloat(uint32_t w) { return __uint2float_rn(w); }
__device__ __forceinline__ float wfloat(unsigned long long w) { return __ull2float_rn(w); }
__device__ __forceinline__ double wdouble(uint32_t w) { return __uint2double_rn(w); }
__device__ __forceinline__ double wdouble(unsigned long long w) { return __ull2double_rn(w); }

// Correctly rounded signed 128-bit integer -> float: shift down to 63
// significant bits with a sticky bit (round to odd), then one RN conversion.
__device__ __forceinline__ float i128_to_float(__int128 s) {
    const bool neg = s < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-s) : (unsigned __int128)s;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    float f;
    if (hi == 0 && (lo >> 63) == 0) {
        f = __ull2float_rn(lo);
    } else {
        const int bl = hi ? 128 - __clzll((long long)hi) : 64;
        const int sh = bl - 63;
        const unsigned __int128 mask = (((unsigned __int128)1) << sh) - 1;
        const uint64_t m = (uint64_t)(u >> sh) | (uint64_t)((u & mask) != 0);
        f = __fmul_rn(__ull2float_rn(m), pow2f(sh));
    }
    return neg ? -f : f;
}

// ------------------------------------------------------------ displacement

// Displacement of the tested and exported vertices by seeded fractal value
// noise, standing in for the wave layers and elevation data with which the
// paper displaces the projected vertices during refinement (Sec. 4; R14
// reading):
//   lattice value of integer point i at octave o: lowbias32 (Wellons,
//     "Prospecting for Hash Functions", 2018) chained from seed ^ o over the
//     coordinates, last to first; the top 24 bits give (h >> 8) 2^-23 - 1;
//   octave o: per axis s = x f 2^o clamped to +-2^30, corner floor(s),
//     weight u = t t (3 - 2 t) with t = s - floor(s); the 2^n corner values
//     blended along x, then y, then z, as a + u (b - a);
//   fbm = the sum over o < octaves of 2^-o times octave o, in order.
// Every FP32 operation rounds separately.
__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ float lattice_unit(uint32_t h) {
    return __fsub_rn(__fmul_rn(__uint2float_rn(h >> 8), 0x1p-23f), 1.0f);
}
__device__ __forceinline__ float blend(float a, float b, float u) {
    return __fadd_rn(a, __fmul_rn(u, __fsub_rn(b, a)));
}
// Corner index and weight of one axis at frequency fo.
__device__ __forceinline__ float noise_axis(float x, float fo, uint32_t& i) {
    const float s = fminf(fmaxf(__fmul_rn(x, fo), -0x1p30f), 0x1p30f);
    const float fl = floorf(s);
    i = (uint32_t)(int)fl;
    const float t = __fsub_rn(s, fl);
    return __fmul_rn(__fmul_rn(t, t), __fsub_rn(3.0f, __fmul_rn(2.0f, t)));
}

// 2-D fbm of (x0, x1); the hash prefix of each y corner is shared.
static __device__ __noinline__ float fbm2(float x0, float x1, float freq, uint32_t octaves, uint32_t seed) {
    float sum = 0.0f;
    for (uint32_t o = 0; o < octaves; ++o) {
        const float fo = __fmul_rn(freq, pow2f((int)o));
        uint32_t ix, iy;
        const float ux = noise_axis(x0, fo, ix), uy = noise_axis(x1, fo, iy);
        const uint32_t h0 = lowbias32(seed ^ o);
        const uint32_t hy0 = lowbias32(h0 ^ iy), hy1 = lowbias32(h0 ^ (iy + 1u));
        const float a = blend(lattice_unit(lowbias32(hy0 ^ ix)), lattice_unit(lowbias32(hy0 ^ (ix + 1u))), ux);
        const float b = blend(lattice_unit(lowbias32(hy1 ^ ix)), lattice_unit(lowbias32(hy1 ^ (ix + 1u))), ux);
        sum = __fadd_rn(sum, __fmul_rn(blend(a, b, uy), pow2f(-(int)o)));
    }
    return sum;
}

// 3-D fbm of (x0, x1, x2); hash prefixes shared per z and per (z, y).
static __device__ __noinline__ float fbm3(float x0, float x1, float x2, float freq, uint32_t octaves, uint32_t seed) {
    float sum = 0.0f;
    for (uint32_t o = 0; o < octaves; ++o) {
        const float fo = __fmul_rn(freq, pow2f((int)o));
        uint32_t ix, iy, iz;
        const float ux = noise_axis(x0, fo, ix), uy = noise_axis(x1, fo, iy), uz = noise_axis(x2, fo, iz);
        const uint32_t h0 = lowbias32(seed ^ o);
        float zc[2];
#pragma unroll
        for (uint32_t bz = 0; bz < 2; ++bz) {
            const uint32_t hz = lowbias32(h0 ^ (iz + bz));
            const uint32_t hzy0 = lowbias32(hz ^ iy), hzy1 = lowbias32(hz ^ (iy + 1u));
            const float a = blend(lattice_unit(lowbias32(hzy0 ^ ix)), lattice_unit(lowbias32(hzy0 ^ (ix + 1u))), ux);
            const float b = blend(lattice_unit(lowbias32(hzy1 ^ ix)), lattice_unit(lowbias32(hzy1 ^ (ix + 1u))), ux);
            zc[bz] = blend(a, b, uy);
        }
        sum = __fadd_rn(sum, __fmul_rn(blend(zc[0], zc[1], uz), pow2f(-(int)o)));
    }
    return sum;
}

// Forms whose vertices the one-launch frame caches from its LOD test for the
// export (a sphere projection or a displacement costs more to evaluate again
// than 36 bytes cost to store and load).
__device__ __forceinline__ bool vc_form(const FrameP& fp) { return fp.precision == 3u || fp.damp != 0.0f; }

// FP32 form: z += amplitude * fbm2 of the world (x, y), the vertex plus the
// origin rounded to FP32.
__device__ __forceinline__ void displace_plain(float r[3], const FrameP& fp) {
    const float wx = __fadd_rn(r[0], __double2float_rn(fp.eye[0]));
    const float wy = __fadd_rn(r[1], __double2float_rn(fp.eye[1]));
    r[2] = __fadd_rn(r[2], __fmul_rn(fp.damp, fbm2(wx, wy, fp.dfreq, fp.doct, fp.dseed)));
}

// Vertex v (0..2) of a bisector relative to the frame's origin, rounded to
// FP32, into r[0..2]:
//   FP32:   (w0 R0 + w1 R1) + w2 R2, w = float(W) 2^-d (no contraction);
//   FIXED:  float(sum W X) 2^-(d + shift), the sum exact in 128 bits;
//   FP64:   float((w0 D0 + w1 D1) + w2 D2), w = double(W) 2^-d;
//   SPHERE: the FP64 point p of the flat root triangle (V absolute) moved
//           radially onto the sphere about the world origin, relative to the
//           eye, rounded to FP32; with fused multiply-adds:
//             p_c = fma(w2, V2c, fma(w1, V1c, w0 V0c)),
//             n2  = fma(pz, pz, fma(py, py, px px)),
//             y   = 1 / sqrt(n2): the FP32 estimate 1 / sqrtf(float(n2)),
//                   then twice y = fma(y/2, fma(-n2, y y, 1), y) (Newton),
//             r_c = float(fma(p_c, radius y, -eye_c)).
// With a displacement the FP32 form adds amplitude * fbm2(world x, y) to z
// (displace_plain) and the sphere form takes radius + double(amplitude *
// fbm3(u)) for the radius, u_c = float(p_c y) the unit direction.
// The sphere form's frame-independent part of vertex v: pf = {p_x, p_y, p_z,
// f}, f = radius' y (V: the root triangle's absolute FP64 vertices). It
// depends on the heap ID, the mesh, the radius and the displacement only.
template <typename T>
__device__ __forceinline__ void sphere_point(const T W[9], int v, int d, const FrameP& fp, const double* V,
                                             double pf[4]) {
    const double sc = pow2d(-d);
    const double w0 = __dmul_rn(wdouble(W[3 * v + 0]), sc);
    const double w1 = __dmul_rn(wdouble(W[3 * v + 1]), sc);
    const double w2 = __dmul_rn(wdouble(W[3 * v + 2]), sc);
    double p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = __fma_rn(w2, V[6 + c], __fma_rn(w1, V[3 + c], __dmul_rn(w0, V[c])));
    const double n2 = __fma_rn(p[2], p[2], __fma_rn(p[1], p[1], __dmul_rn(p[0], p[0])));
    double y = (double)__frcp_rn(__fsqrt_rn(__double2float_rn(n2)));
#pragma unroll
    for (int it = 0; it < 2; ++it) y = __fma_rn(__dmul_rn(y, 0.5), __fma_rn(-n2, __dmul_rn(y, y), 1.0), y);
    double rad = fp.radius;
    if (fp.damp != 0.0f) {
        const float hgt = __fmul_rn(fp.damp, fbm3(__double2float_rn(__dmul_rn(p[0], y)),
                                                 __double2float_rn(__dmul_rn(p[1], y)),
                                                 __double2float_rn(__dmul_rn(p[2], y)), fp.dfreq, fp.doct,
                                                 fp.dseed));
        rad = __dadd_rn(rad, (double)hgt);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) pf[c] = p[c];
    pf[3] = __dmul_rn(rad, y);
}

// The per-frame part: the point relative to the eye, rounded to FP32.
__device__ __forceinline__ void sphere_rel(double px, double py, double pz, double f, const FrameP& fp,
                                           float r[3]) {
    r[0] = __double2float_rn(__fma_rn(px, f, -fp.eye[0]));
    r[1] = __double2float_rn(__fma_rn(py, f, -fp.eye[1]));
    r[2] = __double2float_rn(__fma_rn(pz, f, -fp.eye[2]));
}

template <typename T>
__device__ __forceinline__ void eval_vertex(const T W[9], int v, int d, const FrameP& fp, const void* rel,
                                            uint32_t h, float r[3]) {
    const uint32_t precision = fp.precision;
    if (precision == 3) {
        double pf[4];
        sphere_point<T>(W, v, d, fp, static_cast<const double*>(rel) + 9u * h, pf);
        sphere_rel(pf[0], pf[1], pf[2], pf[3], fp, r);
    } else if (precision == 1) {
        const long long* X = static_cast<const long long*>(rel) + 9u * h;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            __int128 s = (__int128)(unsigned long long)W[3 * v + 0] * (__int128)X[c];
            s += (__int128)(unsigned long long)W[3 * v + 1] * (__int128)X[3 + c];
            s += (__int128)(unsigned long long)W[3 * v + 2] * (__int128)X[6 + c];
            r[c] = __fmul_rn(i128_to_float(s), pow2f(-(d + fp.shift)));
        }
    } else if (precision == 2) {
        const double* Dp = static_cast<const double*>(rel) + 9u * h;
        const double sc = pow2d(-d);
        const double w0 = __dmul_rn(wdouble(W[3 * v + 0]), sc);
        const double w1 = __dmul_rn(wdouble(W[3 * v + 1]), sc);
        const double w2 = __dmul_rn(wdouble(W[3 * v + 2]), sc);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double t = __dadd_rn(__dadd_rn(__dmul_rn(w0, Dp[c]), __dmul_rn(w1, Dp[3 + c])),
                                       __dmul_rn(w2, Dp[6 + c]));
            r[c] = __double2float_rn(t);
        }
    } else {
        const float* R = static_cast<const float*>(rel) + 9u * h;
        const float sc = pow2f(-d);
        const float w0 = __fmul_rn(wfloat(W[3 * v + 0]), sc);
        const float w1 = __fmul_rn(wfloat(W[3 * v + 1]), sc);
        const float w2 = __fmul_rn(wfloat(W[3 * v + 2]), sc);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            r[c] = __fadd_rn(__fadd_rn(__fmul_rn(w0, R[c]), __fmul_rn(w1, R[3 + c])), __fmul_rn(w2, R[6 + c]));
        if (fp.damp != 0.0f) displace_plain(r, fp);
    }
}

// All three vertices, r[3 v + c] (the same roundings as eval_vertex; the
// root table is read once for the three).
template <typename T>
__device__ __forceinline__ void eval_vertices(const T W[9], int d, const FrameP& fp, const void* rel, uint32_t h,
                                              float r[9]) {
    const uint32_t precision = fp.precision;
    if (precision == 3) {
#pragma unroll
        for (int v = 0; v < 3; ++v) eval_vertex<T>(W, v, d, fp, rel, h, r + 3 * v);
    } else if (precision == 1) {
        const long long* X = static_cast<const long long*>(rel) + 9u * h;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                __int128 s = (__int128)(unsigned long long)W[3 * i + 0] * (__int128)X[c];
                s += (__int128)(unsigned long long)W[3 * i + 1] * (__int128)X[3 + c];
                s += (__int128)(unsigned long long)W[3 * i + 2] * (__int128)X[6 + c];
                r[3 * i + c] = __fmul_rn(i128_to_float(s), pow2f(-(d + fp.shift)));
            }
    } else if (precision == 2) {
        const double* Dp = static_cast<const double*>(rel) + 9u * h;
        const double sc = pow2d(-d);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double w0 = __dmul_rn(wdouble(W[3 * i + 0]), sc);
            const double w1 = __dmul_rn(wdouble(W[3 * i + 1]), sc);
            const double w2 = __dmul_rn(wdouble(W[3 * i + 2]), sc);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double t = __dadd_rn(__dadd_rn(__dmul_rn(w0, Dp[c]), __dmul_rn(w1, Dp[3 + c])),
                                           __dmul_rn(w2, Dp[6 + c]));
                r[3 * i + c] = __double2float_rn(t);
            }
        }
    } else {
        const float* R = static_cast<const float*>(rel) + 9u * h;
        const float sc = pow2f(-d);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float w0 = __fmul_rn(wfloat(W[3 * i + 0]), sc);
            const float w1 = __fmul_rn(wfloat(W[3 * i + 1]), sc);
            const float w2 = __fmul_rn(wfloat(W[3 * i + 2]), sc);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                r[3 * i + c] = __fadd_rn(__fadd_rn(__fmul_rn(w0, R[c]), __fmul_rn(w1, R[3 + c])), __fmul_rn(w2, R[6 + c]));
        }
        if (fp.damp != 0.0f)
#pragma unroll
            for (int i = 0; i < 3; ++i) displace_plain(r + 3 * i, fp);
    }
}

// LOD reading: a triangle is visible unless one plane has all three
// vertices strictly on its negative side, where a vertex r is on the
// negative side of plane n when (n.x r.x + n.y r.y) + n.z r.z < 0; it is
// big when |v1 - v0|^2 q > |(v0 + v1)/2|^2.
// The planes among `among` (a bit mask) on whose negative side vertex r
// lies, as a bit mask: a triangle is culled by a plane only if all three
// vertices are, so a vertex need only be tested against the planes the
// earlier ones failed (the same products, bit for bit, where they are made).
__device__ __forceinline__ uint32_t plane_mask(const float* r, const FrameP& fp, uint32_t among = 31u) {
    uint32_t m = 0u;
#pragma unroll
    for (uint32_t p = 0; p < 5u; ++p) {
        if (p >= fp.nplanes) break;
        if (!((among >> p) & 1u)) continue;
        const float s = __fadd_rn(__fadd_rn(__fmul_rn(fp.planes[3 * p], r[0]), __fmul_rn(fp.planes[3 * p + 1], r[1])),
                                  __fmul_rn(fp.planes[3 * p + 2], r[2]));
        m |= (s < 0.0f ? 1u : 0u) << p;
    }
    return m;
}
// |a - b|^2 q > |(a + b)/2|^2 for the refinement edge (a, b).
__device__ __forceinline__ bool edge_big(const float* a, const float* b, float q) {
    const float ex = __fsub_rn(b[0], a[0]), ey = __fsub_rn(b[1], a[1]), ez = __fsub_rn(b[2], a[2]);
    const float mx = __fmul_rn(0.5f, __fadd_rn(a[0], b[0]));
    const float my = __fmul_rn(0.5f, __fadd_rn(a[1], b[1]));
    const float mz = __fmul_rn(0.5f, __fadd_rn(a[2], b[2]));
    const float L2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
    const float R2 = __fadd_rn(__fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my)), __fmul_rn(mz, mz));
    return __fmul_rn(L2, q) > R2;
}
// bit0 visible, bit1 big.
__device__ __forceinline__ uint32_t lod_test(const float r[9], const FrameP& fp) {
    uint32_t out = plane_mask(r, fp);
    if (out) out = plane_mask(r + 3, fp, out);
    if (out) out = plane_mask(r + 6, fp, out);
    return (out == 0u ? 1u : 0u) | (edge_big(r, r + 3, fp.q) ? 2u : 0u);
}

__device__ __forceinline__ bool in_sorted(const uint64_t* a, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2u;
        if (a[mid] < x)
            lo = mid + 1u;
        else
            hi = mid;
    }
    return lo < n && a[lo] == x;
}

// --------------------------------------------------------- saturating pairs

constexpr uint32_t kSat = 0x7FFFFFFFu;

struct Pair {
    uint32_t a, b;
};

__device__ __forceinline__ Pair padd(Pair x, Pair y) {
    return Pair{min(x.a + y.a, kSat), min(x.b + y.b, kSat)};
}

constexpr unsigned long long kFlagAgg = 1ull, kFlagIncl = 2ull;

__device__ __forceinline__ unsigned long long pack_status(unsigned long long flag, Pair v) {
    return (flag << 62) | ((unsigned long long)v.a << 31) | (unsigned long long)v.b;
}
__device__ __forceinline__ unsigned long long status_flag(unsigned long long s) { return s >> 62; }
__device__ __forceinline__ Pair status_val(unsigned long long s) {
    return Pair{(uint32_t)((s >> 31) & kSat), (uint32_t)(s & kSat)};
}

}  // namespace cbtgpu
