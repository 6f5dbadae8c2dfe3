/* CPU oracle for the concurrent-binary-tree adaptive bisection update.
 *
 * TEST INFRASTRUCTURE ONLY. A plain, slow, sequential restatement of
 * "Concurrent Binary Trees for Large-Scale Game Components" (Benyoub &
 * Dupuy, 2024), used by the tests, the smoke check and the benchmark's CPU
 * baseline to check the CUDA library. It shares no code with that library.
 * Build: gcc -O2 -ffp-contract=off (no fast-math), so every floating-point
 * operation below is one IEEE round-to-nearest operation in source order.
 *
 * One frame (Sec. 3.3, the nine kernels of the update pipeline) is computed as:
 *   1. L = live slots: OneToBitID(i) for i < CBT root (Alg. 7, CachePointers);
 *   2. every b in L is classified on the frame-start state: vertices by
 *      Alg. 2 / Eq. 1, split and merge wishes by the LOD test
 *      (GenerateCommands);
 *   3. requests and the gate: a split wish costs its compatibility-chain
 *      allocation count, a mergeable group costs its parent count at its
 *      smallest-heap-ID member; merges first, then splits, each in ascending
 *      slot order, granted while the running total stays within the free
 *      bits (GenerateCommands' allocation-counter condition, made
 *      deterministic);
 *   4. granted splits set R/N/P command bits along their chains; a merge
 *      group is valid if all members wish to merge, none has command bits
 *      and its smallest member was granted (GenerateCommands, ReserveBlocks);
 *   5. the topology change is applied the textbook way, one request at a
 *      time on a node graph: Refine (Alg. 3) with the neighbour rules of
 *      Table 1 and RefinePointers (Alg. 5), then Decimate (Alg. 4) with
 *      DecimatePointers (Alg. 6);
 *   6. new bisectors take free slots ZeroToBitID(base + i) of the
 *      frame-start CBT (Alg. 8, ReserveBlocks) in ascending slot order of
 *      the bisector they come from (R7 reading);
 *   7. UpdateBitfield and SumReduction (Sec. 3.2, Alg. 9).
 * Step 5 must reproduce exactly the leaves that the command bits of step 4
 * predict; every disagreement is counted in or_stats.ab_mismatch.
 */
#include "cbt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define R_BIT 1u
#define N_BIT 2u
#define P_BIT 4u

struct or_state {
    int32_t H, D, max_depth, ch;
    uint32_t cap;
    uint32_t frame;
    uint32_t* cbt; /* 2^(D+1) entries, heap order, leaves at [cap, 2 cap) */
    uint64_t* heap;
    uint32_t* twn;
    uint32_t* nxt;
    uint32_t* prv;
    double* root; /* [H][3 vertices][xyz] */
    uint32_t* corner_id; /* [H][3] global point of each root corner: vert[h], vert[next h], V + face[h] */
    uint64_t order_seed; /* 0: textbook step in slot order; else a seeded permutation */
};

static int bitlen64(uint64_t x) {
    int n = 0;
    while (x) {
        ++n;
        x >>= 1;
    }
    return n;
}

static int ceil_log2_u32(uint32_t x) {
    int c = 0;
    while ((1ull << c) < (uint64_t)x) ++c;
    return c;
}

static int depth_of(const or_state* st, uint64_t j) { return bitlen64(j) - 1 - st->ch; }

static uint32_t root_of(const or_state* st, uint64_t j) {
    return (uint32_t)((j >> depth_of(st, j)) - (1ull << st->ch));
}

/* ------------------------------------------------------------------ CBT */

/* SumReduction (Sec. 3.1): every internal node is the sum of its children. */
void or_cbt_sum_reduction(int32_t D, uint32_t* cbt) {
    for (uint32_t k = (1u << D) - 1u; k >= 1u; --k) cbt[k] = cbt[2u * k] + cbt[2u * k + 1u];
}

/* Alg. 7: slot of the index-th bit set to one. */
uint32_t or_cbt_one_to_bit(int32_t D, const uint32_t* cbt, uint32_t index) {
    const uint32_t n = 1u << D;
    uint32_t bit = 1;
    while (bit < n) {
        bit *= 2u;
        if (index >= cbt[bit]) {
            index -= cbt[bit];
            bit += 1u;
        }
    }
    return bit - n;
}

/* CachePointers (Alg. 7 for every index): out[i] = OneToBitID(i) for every
 * i below the root. */
void or_cbt_compact(int32_t D, const uint32_t* cbt, uint32_t* out) {
    for (uint32_t i = 0; i < cbt[1]; ++i) out[i] = or_cbt_one_to_bit(D, cbt, i);
}

/* Alg. 8: slot of the index-th bit set to zero; c is the leaf count of the
 * subtree being examined, so c - CBT[node] counts its zeros. */
uint32_t or_cbt_zero_to_bit(int32_t D, const uint32_t* cbt, uint32_t index) {
    const uint32_t n = 1u << D;
    uint32_t bit = 1, c = n >> 1;
    while (bit < n) {
        bit *= 2u;
        const uint32_t zeros = c - cbt[bit];
        if (index >= zeros) {
            index -= zeros;
            bit += 1u;
        }
        c >>= 1;
    }
    return bit - n;
}

/* --------------------------------------------------------- halfedges */

typedef struct {
    int32_t a, b, h;
} edge_key;

static int cmp_edge_key(const void* x, const void* y) {
    const edge_key* p = (const edge_key*)x;
    const edge_key* q = (const edge_key*)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    return (p->h > q->h) - (p->h < q->h);
}

static int32_t find_key(const edge_key* k, int32_t n, int32_t a, int32_t b, int32_t* count) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (k[mid].a < a || (k[mid].a == a && k[mid].b < b))
            lo = mid + 1;
        else
            hi = mid;
    }
    int32_t c = 0;
    while (lo + c < n && k[lo + c].a == a && k[lo + c].b == b) ++c;
    *count = c;
    return c ? k[lo].h : -1;
}

/* Sec. 2.1: each face's halfedges go round the face; Twin is the halfedge
 * running the other way along the same edge, -1 on a border. */
int or_halfedges_from_faces(int32_t F, const int32_t* face_sizes, const int32_t* face_verts,
                            int32_t H, int32_t* twin, int32_t* next, int32_t* prev,
                            int32_t* vert, int32_t* face) {
    int32_t h = 0;
    for (int32_t f = 0; f < F; ++f) {
        const int32_t n = face_sizes[f];
        if (n < 3 || h + n > H) return OR_EINVAL;
        for (int32_t i = 0; i < n; ++i) {
            vert[h + i] = face_verts[h + i];
            next[h + i] = h + (i + 1) % n;
            prev[h + i] = h + (i + n - 1) % n;
            face[h + i] = f;
        }
        h += n;
    }
    if (h != H) return OR_EINVAL;
    edge_key* keys = (edge_key*)malloc(sizeof(edge_key) * (size_t)H);
    if (!keys) return OR_ENOMEM;
    for (int32_t e = 0; e < H; ++e) {
        keys[e].a = vert[e];
        keys[e].b = vert[next[e]];
        keys[e].h = e;
    }
    qsort(keys, (size_t)H, sizeof(edge_key), cmp_edge_key);
    int rc = OR_OK;
    for (int32_t e = 0; e < H && rc == OR_OK; ++e) {
        int32_t cnt = 0;
        find_key(keys, H, vert[e], vert[next[e]], &cnt);
        if (cnt != 1) rc = OR_EINVAL; /* an edge used twice in one direction */
        const int32_t t = find_key(keys, H, vert[next[e]], vert[e], &cnt);
        if (cnt > 1) rc = OR_EINVAL;
        twin[e] = t;
    }
    free(keys);
    return rc;
}

/* ------------------------------------------------------------ create */

int or_create(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
              const int32_t* vert, const int32_t* face, int32_t V, const double* pos,
              int32_t D, int32_t max_depth, or_state** out) {
    *out = NULL;
    if (H < 3 || V < 1) return OR_EINVAL;
    for (int32_t h = 0; h < H; ++h) {
        if (next[h] < 0 || next[h] >= H || prev[h] < 0 || prev[h] >= H) return OR_EINVAL;
        if (prev[next[h]] != h || next[prev[h]] != h) return OR_EINVAL;
        if (face[h] < 0 || face[h] >= H || face[next[h]] != face[h]) return OR_EINVAL;
        if (vert[h] < 0 || vert[h] >= V) return OR_EINVAL;
        if (twin[h] != -1) {
            const int32_t t = twin[h];
            if (t < 0 || t >= H || t == h || twin[t] != h) return OR_EINVAL;
            if (vert[t] != vert[next[h]] || vert[next[t]] != vert[h]) return OR_EINVAL;
        }
    }
    const int ch = ceil_log2_u32((uint32_t)H);
    if (D < 1 || D > 30) return OR_EINVAL;
    if (D < ch) return OR_ECAPACITY;
    if (max_depth < 0 || ch + 1 + max_depth > 63) return OR_EDEPTH;

    or_state* st = (or_state*)calloc(1, sizeof(or_state));
    if (!st) return OR_ENOMEM;
    st->H = H;
    st->D = D;
    st->max_depth = max_depth;
    st->ch = ch;
    st->cap = 1u << D;
    st->cbt = (uint32_t*)calloc((size_t)st->cap * 2u, sizeof(uint32_t));
    st->heap = (uint64_t*)calloc(st->cap, sizeof(uint64_t));
    st->twn = (uint32_t*)malloc(sizeof(uint32_t) * st->cap);
    st->nxt = (uint32_t*)malloc(sizeof(uint32_t) * st->cap);
    st->prv = (uint32_t*)malloc(sizeof(uint32_t) * st->cap);
    st->root = (double*)calloc((size_t)H * 9u, sizeof(double));
    st->corner_id = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)H * 3u);
    double* cen = (double*)calloc((size_t)H * 3u, sizeof(double));
    int32_t* first = (int32_t*)malloc(sizeof(int32_t) * (size_t)H);
    if (!st->cbt || !st->heap || !st->twn || !st->nxt || !st->prv || !st->root || !st->corner_id || !cen ||
        !first) {
        free(cen);
        free(first);
        or_destroy(st);
        return OR_ENOMEM;
    }
    /* Alg. 1 with one centroid per face (R3 reading): the FP64 sum starts at
     * the face's smallest halfedge index and follows Next. */
    for (int32_t f = 0; f < H; ++f) first[f] = -1;
    for (int32_t h = 0; h < H; ++h)
        if (first[face[h]] < 0) first[face[h]] = h;
    for (int32_t f = 0; f < H; ++f) {
        if (first[f] < 0) continue;
        double s[3] = {0, 0, 0};
        int32_t n = 0, h = first[f];
        do {
            for (int c = 0; c < 3; ++c) s[c] = s[c] + pos[3 * vert[h] + c];
            ++n;
            h = next[h];
        } while (h != first[f] && n <= H);
        for (int c = 0; c < 3; ++c) cen[3 * f + c] = s[c] / (double)n;
    }
    for (int32_t h = 0; h < H; ++h) {
        for (int c = 0; c < 3; ++c) {
            st->root[9 * h + 0 + c] = pos[3 * vert[h] + c];
            st->root[9 * h + 3 + c] = pos[3 * vert[next[h]] + c];
            st->root[9 * h + 6 + c] = cen[3 * face[h] + c];
        }
        st->corner_id[3 * h + 0] = (uint32_t)vert[h];
        st->corner_id[3 * h + 1] = (uint32_t)vert[next[h]];
        st->corner_id[3 * h + 2] = (uint32_t)V + (uint32_t)face[h];
    }
    free(cen);
    free(first);
    /* Sec. 3.3 "Initialization": H roots in the first H slots, neighbours
     * copied from the halfedge operators. */
    for (uint32_t s = 0; s < st->cap; ++s) st->twn[s] = st->nxt[s] = st->prv[s] = OR_NULL;
    for (int32_t h = 0; h < H; ++h) {
        st->heap[h] = (1ull << ch) + (uint64_t)h;
        st->twn[h] = twin[h] < 0 ? OR_NULL : (uint32_t)twin[h];
        st->nxt[h] = (uint32_t)next[h];
        st->prv[h] = (uint32_t)prev[h];
        st->cbt[st->cap + (uint32_t)h] = 1u;
    }
    or_cbt_sum_reduction(D, st->cbt);
    *out = st;
    return OR_OK;
}

void or_destroy(or_state* st) {
    if (!st) return;
    free(st->cbt);
    free(st->heap);
    free(st->twn);
    free(st->nxt);
    free(st->prv);
    free(st->root);
    free(st->corner_id);
    free(st);
}

uint32_t or_live_count(const or_state* st) { return st->cbt[1]; }
int32_t or_ceil_log2_H(const or_state* st) { return st->ch; }

void or_export(const or_state* st, uint32_t* cbt, uint64_t* heap, uint32_t* twin,
               uint32_t* next, uint32_t* prev) {
    if (cbt) memcpy(cbt, st->cbt, sizeof(uint32_t) * (size_t)st->cap * 2u);
    if (heap) memcpy(heap, st->heap, sizeof(uint64_t) * st->cap);
    if (twin) memcpy(twin, st->twn, sizeof(uint32_t) * st->cap);
    if (next) memcpy(next, st->nxt, sizeof(uint32_t) * st->cap);
    if (prev) memcpy(prev, st->prv, sizeof(uint32_t) * st->cap);
}

void or_root_table(const or_state* st, double* out) {
    memcpy(out, st->root, sizeof(double) * 9u * (size_t)st->H);
}

/* ------------------------------------------------- vertices (Alg. 2) */

/* Eq. 1 scaled by 2, so that products stay integral: T_b = 2 M_b. */
static const uint64_t T2[2][3][3] = {
    {{2, 0, 0}, {0, 0, 2}, {1, 1, 0}},
    {{0, 0, 2}, {0, 2, 0}, {1, 1, 0}},
};

/* Alg. 2: M = M_b(last) x ... x M_b(first), bits read from the least
 * significant end of j; returned as W = 2^d M (exact integers). */
void or_decode_weights(uint64_t j, int32_t ch, uint64_t* W9) {
    const int d = bitlen64(j) - 1 - ch;
    uint64_t M[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    uint64_t h = j;
    for (int s = 0; s < d; ++s) {
        const int b = (int)(h & 1u);
        uint64_t R[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                uint64_t acc = 0;
                for (int m = 0; m < 3; ++m) acc += M[r][m] * T2[b][m][c];
                R[r][c] = acc;
            }
        memcpy(M, R, sizeof(M));
        h >>= 1;
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) W9[3 * r + c] = M[r][c];
}

/* ------------------------------------------------------- displacement */

/* lowbias32 (Wellons, "Prospecting for Hash Functions", 2018): two
 * xorshift-multiply rounds and a final xorshift, a bijection of 32-bit
 * words. */
uint32_t or_lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

/* Value of lattice point idx[0..n) at octave o (R14): the hash chained from
 * seed ^ o over the coordinates, last to first; the top 24 bits mapped
 * exactly onto [-1, 1) in steps of 2^-23. */
static float lattice_value(uint32_t seed, uint32_t o, int n, const int32_t* idx) {
    uint32_t h = or_lowbias32(seed ^ o);
    for (int k = n - 1; k >= 0; --k) h = or_lowbias32(h ^ (uint32_t)idx[k]);
    return (float)(h >> 8) * 0x1p-23f - 1.0f;
}

/* Fractal value noise (R14): octave o samples the lattice at frequency
 * frequency * 2^o with weight 2^-o. In a cell the point has integer corner
 * floor(s) and offset t = s - floor(s) per axis (s clamped to +-2^30); the
 * 2^n corner values are blended along x, then y, then z, with
 * a + u (b - a) and the smoothstep weight u = t t (3 - 2 t). */
float or_fbm(const float* x, int32_t n, float frequency, uint32_t octaves, uint32_t seed) {
    float sum = 0.0f;
    for (uint32_t o = 0; o < octaves; ++o) {
        const float fo = ldexpf(frequency, (int)o);
        int32_t i0[3] = {0, 0, 0};
        float u[3] = {0.0f, 0.0f, 0.0f};
        for (int k = 0; k < n; ++k) {
            float s = x[k] * fo;
            s = fminf(fmaxf(s, -0x1p30f), 0x1p30f);
            const float fl = floorf(s);
            i0[k] = (int32_t)fl;
            const float t = s - fl;
            u[k] = (t * t) * (3.0f - 2.0f * t);
        }
        float c[8];
        for (int m = 0; m < (1 << n); ++m) { /* bit k of m: the upper corner along axis k */
            int32_t idx[3];
            for (int k = 0; k < n; ++k) idx[k] = i0[k] + ((m >> k) & 1);
            c[m] = lattice_value(seed, o, n, idx);
        }
        int cnt = 1 << n;
        for (int k = 0; k < n; ++k) {
            cnt >>= 1;
            for (int m = 0; m < cnt; ++m) c[m] = c[2 * m] + u[k] * (c[2 * m + 1] - c[2 * m]);
        }
        sum += c[0] * ldexpf(1.0f, -(int)o);
    }
    return sum;
}

static int disp_valid(const or_disp* D, uint32_t precision) {
    if (!D || D->amplitude == 0.0f) return 1;
    return isfinite(D->amplitude) && isfinite(D->frequency) && D->frequency > 0.0f && D->octaves >= 1u &&
           D->octaves <= 8u && (precision == OR_PREC_FP32 || precision == OR_PREC_SPHERE);
}

typedef struct {
    uint32_t precision;
    int32_t shift;
    or_disp disp;        /* amplitude 0: no displacement */
    float org32[3];      /* FP32 form: the origin rounded to FP32 (world x, y for the noise) */
    double radius;       /* PREC_SPHERE */
    double org[3];       /* PREC_SPHERE: the origin, subtracted after the projection */
    const double* abs64; /* PREC_SPHERE: the FP64 root vertices themselves */
    float* r32;   /* [H][9] FP32 root vertices minus the origin */
    int64_t* x;   /* [H][9] fixed point round((V - origin) 2^shift) */
    double* d64;  /* [H][9] FP64 root vertices minus the origin */
} rel_roots;

static int make_rel(const or_state* st, const double org[3], uint32_t precision, int32_t shift,
                    double radius, const or_disp* disp, rel_roots* R) {
    memset(R, 0, sizeof(*R));
    R->precision = precision;
    R->shift = shift;
    R->radius = radius;
    if (disp) R->disp = *disp;
    for (int c = 0; c < 3; ++c) {
        R->org[c] = org[c];
        R->org32[c] = (float)org[c];
    }
    R->abs64 = st->root;
    if (precision == OR_PREC_SPHERE && !(radius > 0.0)) return OR_EINVAL;
    if (!disp_valid(disp, precision)) return OR_EINVAL;
    const size_t n = (size_t)st->H * 9u;
    R->r32 = (float*)malloc(sizeof(float) * n);
    R->x = (int64_t*)malloc(sizeof(int64_t) * n);
    R->d64 = (double*)malloc(sizeof(double) * n);
    if (!R->r32 || !R->x || !R->d64) return OR_ENOMEM;
    for (size_t i = 0; i < n; ++i) {
        const double diff = st->root[i] - org[i % 3u];
        R->d64[i] = diff;
        R->r32[i] = (float)diff;
        const double sc = ldexp(diff, shift);
        if (precision == OR_PREC_FIXED && !(fabs(sc) < 4.611686018427387904e18)) return OR_EINVAL;
        R->x[i] = precision == OR_PREC_FIXED ? (int64_t)llrint(sc) : 0;
    }
    return OR_OK;
}

static void free_rel(rel_roots* R) {
    free(R->r32);
    free(R->x);
    free(R->d64);
}

/* Vertices of bisector j relative to the origin, rounded to FP32 (R9/R10
 * readings): exact integer weights W, then
 *   FP32:  (w0 R0 + w1 R1) + w2 R2 with w = float(W) 2^-d,
 *   FIXED: float(sum W X) 2^-(d + shift), the integer sum exact in 128 bits,
 *   FP64:  float((w0 D0 + w1 D1) + w2 D2) with w = double(W) 2^-d,
 *   SPHERE: the FP64 point p of the flat root triangle (V absolute) moved
 *           radially onto the sphere about the world origin, then taken
 *           relative to the origin and rounded to FP32 (the paper projects
 *           the vertices onto a sphere during refinement, Sec. 4; R13
 *           reading). In FP64 with fused multiply-adds:
 *             p_c = fma(w2, V2c, fma(w1, V1c, w0 V0c)),
 *             n2  = fma(pz, pz, fma(py, py, px px)),
 *             y   = 1 / sqrt(n2): the FP32 estimate 1/sqrtf(float(n2)),
 *                   then twice y = fma(y/2, fma(-n2, y y, 1), y) (Newton),
 *             out = float(fma(p_c, radius y, -origin_c)).
 * With a displacement (R14) the FP32 form adds amplitude * fbm(x, y) to z,
 * (x, y) = the vertex plus the origin rounded to FP32; the sphere form uses
 * the radius + double(amplitude * fbm(u)) in place of the radius, u_c =
 * float(p_c y) the unit direction. */
static void bisector_rel(const or_state* st, const rel_roots* R, uint64_t j, float out[9]) {
    const int d = depth_of(st, j);
    const uint32_t h = root_of(st, j);
    uint64_t W[9];
    or_decode_weights(j, st->ch, W);
    if (R->precision == OR_PREC_SPHERE) {
        for (int i = 0; i < 3; ++i) {
            const double w0 = ldexp((double)W[3 * i + 0], -d);
            const double w1 = ldexp((double)W[3 * i + 1], -d);
            const double w2 = ldexp((double)W[3 * i + 2], -d);
            double p[3];
            for (int c = 0; c < 3; ++c) {
                const size_t b = 9u * h + (size_t)c;
                p[c] = fma(w2, R->abs64[b + 6], fma(w1, R->abs64[b + 3], w0 * R->abs64[b + 0]));
            }
            const double n2 = fma(p[2], p[2], fma(p[1], p[1], p[0] * p[0]));
            double y = (double)(1.0f / sqrtf((float)n2));
            for (int it = 0; it < 2; ++it) y = fma(y * 0.5, fma(-n2, y * y, 1.0), y);
            double rad = R->radius;
            if (R->disp.amplitude != 0.0f) {
                const float u[3] = {(float)(p[0] * y), (float)(p[1] * y), (float)(p[2] * y)};
                const float hgt =
                    R->disp.amplitude * or_fbm(u, 3, R->disp.frequency, R->disp.octaves, R->disp.seed);
                rad = rad + (double)hgt;
            }
            const double f = rad * y;
            for (int c = 0; c < 3; ++c) out[3 * i + c] = (float)fma(p[c], f, -R->org[c]);
        }
        return;
    }
    for (int i = 0; i < 3; ++i) {
        for (int c = 0; c < 3; ++c) {
            const size_t b = 9u * h + (size_t)c;
            if (R->precision == OR_PREC_FIXED) {
                __int128 s = (__int128)W[3 * i + 0] * (__int128)R->x[b + 0];
                s += (__int128)W[3 * i + 1] * (__int128)R->x[b + 3];
                s += (__int128)W[3 * i + 2] * (__int128)R->x[b + 6];
                out[3 * i + c] = ldexpf((float)s, -(d + R->shift));
            } else if (R->precision == OR_PREC_FP64) {
                const double w0 = ldexp((double)W[3 * i + 0], -d);
                const double w1 = ldexp((double)W[3 * i + 1], -d);
                const double w2 = ldexp((double)W[3 * i + 2], -d);
                const double t = (w0 * R->d64[b + 0] + w1 * R->d64[b + 3]) + w2 * R->d64[b + 6];
                out[3 * i + c] = (float)t;
            } else {
                const float w0 = ldexpf((float)W[3 * i + 0], -d);
                const float w1 = ldexpf((float)W[3 * i + 1], -d);
                const float w2 = ldexpf((float)W[3 * i + 2], -d);
                out[3 * i + c] = (w0 * R->r32[b + 0] + w1 * R->r32[b + 3]) + w2 * R->r32[b + 6];
            }
        }
        if (R->precision == OR_PREC_FP32 && R->disp.amplitude != 0.0f) {
            const float xy[2] = {out[3 * i] + R->org32[0], out[3 * i + 1] + R->org32[1]};
            const float hgt = R->disp.amplitude * or_fbm(xy, 2, R->disp.frequency, R->disp.octaves, R->disp.seed);
            out[3 * i + 2] = out[3 * i + 2] + hgt;
        }
    }
}

void or_vertices(const or_state* st, const double origin[3], uint32_t precision,
                 int32_t fixed_shift, double sphere_radius, const or_disp* disp, float* out) {
    rel_roots R;
    if (make_rel(st, origin, precision, fixed_shift, sphere_radius, disp, &R) == OR_OK) {
        uint32_t i = 0;
        for (uint32_t s = 0; s < st->cap; ++s)
            if (st->cbt[st->cap + s]) bisector_rel(st, &R, st->heap[s], out + 9u * (size_t)i++);
    }
    free_rel(&R);
}

void or_vertices_f64(const or_state* st, double* out) {
    uint32_t i = 0;
    for (uint32_t s = 0; s < st->cap; ++s) {
        if (!st->cbt[st->cap + s]) continue;
        const uint64_t j = st->heap[s];
        const int d = depth_of(st, j);
        const uint32_t h = root_of(st, j);
        uint64_t W[9];
        or_decode_weights(j, st->ch, W);
        for (int v = 0; v < 3; ++v)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    acc += ldexp((double)W[3 * v + k], -d) * st->root[9u * h + 3u * (unsigned)k + (unsigned)c];
                out[9u * (size_t)i + 3u * (unsigned)v + (unsigned)c] = acc;
            }
        ++i;
    }
}

/* ------------------------------------------------------ indexed export */

/* Identity of a bisector corner as a point of the subdivided surface (R15
 * reading): the exact integer weights of its row (R9, over 2^d) reduced to
 * lowest terms (halved while all are even and d > 0), each nonzero weight
 * paired with the global point of its root corner (mesh vertex, or V + face
 * for a face centroid), the pairs in ascending point order. Corners of two
 * bisectors are the same vertex exactly when these are equal. */
typedef struct {
    uint32_t d, n;
    uint32_t id[3];
    uint64_t w[3];
    uint32_t occ; /* 3 i + corner */
} vkey;

static void corner_key(const or_state* st, uint64_t j, int v, uint32_t occ, vkey* k) {
    int d = depth_of(st, j);
    const uint32_t h = root_of(st, j);
    uint64_t W[9];
    or_decode_weights(j, st->ch, W);
    uint64_t w[3] = {W[3 * v + 0], W[3 * v + 1], W[3 * v + 2]};
    while (d > 0 && !((w[0] | w[1] | w[2]) & 1u)) {
        for (int c = 0; c < 3; ++c) w[c] >>= 1;
        --d;
    }
    memset(k, 0, sizeof(*k));
    k->d = (uint32_t)d;
    k->occ = occ;
    for (int c = 0; c < 3; ++c) k->id[c] = OR_NULL;
    for (int c = 0; c < 3; ++c) {
        if (!w[c]) continue;
        /* insert (id, w) keeping the ids ascending */
        const uint32_t id = st->corner_id[3 * h + (uint32_t)c];
        int p = (int)k->n;
        while (p > 0 && k->id[p - 1] > id) {
            k->id[p] = k->id[p - 1];
            k->w[p] = k->w[p - 1];
            --p;
        }
        k->id[p] = id;
        k->w[p] = w[c];
        ++k->n;
    }
}

static int vkey_cmp(const void* pa, const void* pb) {
    const vkey* a = (const vkey*)pa;
    const vkey* b = (const vkey*)pb;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int c = 0; c < 3; ++c) {
        if (a->id[c] != b->id[c]) return a->id[c] < b->id[c] ? -1 : 1;
        if (a->w[c] != b->w[c]) return a->w[c] < b->w[c] ? -1 : 1;
    }
    if (a->occ != b->occ) return a->occ < b->occ ? -1 : 1;
    return 0;
}

static int vkey_same(const vkey* a, const vkey* b) {
    if (a->d != b->d || a->n != b->n) return 0;
    for (int c = 0; c < 3; ++c)
        if (a->id[c] != b->id[c] || a->w[c] != b->w[c]) return 0;
    return 1;
}

int or_export_indexed(const or_state* st, const float* tri_vertices, float* vertices, uint32_t* indices,
                      uint64_t* tri_ids, uint32_t* n_vertices) {
    const uint32_t N = st->cbt[1];
    const uint32_t n3 = 3u * N;
    vkey* keys = (vkey*)malloc(sizeof(vkey) * (n3 ? n3 : 1u));
    uint32_t* rep = (uint32_t*)malloc(sizeof(uint32_t) * (n3 ? n3 : 1u));
    uint32_t* vid = (uint32_t*)malloc(sizeof(uint32_t) * (n3 ? n3 : 1u));
    if (!keys || !rep || !vid) {
        free(keys);
        free(rep);
        free(vid);
        return OR_ENOMEM;
    }
    uint32_t i = 0;
    for (uint32_t s = 0; s < st->cap; ++s) {
        if (!st->cbt[st->cap + s]) continue;
        for (int c = 0; c < 3; ++c) corner_key(st, st->heap[s], c, 3u * i + (uint32_t)c, &keys[3u * i + (uint32_t)c]);
        if (tri_ids) tri_ids[i] = st->heap[s];
        ++i;
    }
    /* each corner's vertex is represented by its first occurrence */
    qsort(keys, n3, sizeof(vkey), vkey_cmp);
    for (uint32_t a = 0; a < n3;) {
        uint32_t b = a + 1u;
        while (b < n3 && vkey_same(&keys[a], &keys[b])) ++b;
        for (uint32_t k = a; k < b; ++k) rep[keys[k].occ] = keys[a].occ;
        a = b;
    }
    /* vertices numbered in order of first occurrence */
    uint32_t nv = 0;
    for (uint32_t o = 0; o < n3; ++o)
        if (rep[o] == o) {
            vid[o] = nv;
            if (vertices && tri_vertices)
                for (int c = 0; c < 3; ++c) vertices[3u * nv + (uint32_t)c] = tri_vertices[3u * o + (uint32_t)c];
            ++nv;
        }
    for (uint32_t o = 0; o < n3; ++o) indices[o] = vid[rep[o]];
    *n_vertices = nv;
    free(keys);
    free(rep);
    free(vid);
    return OR_OK;
}

/* ------------------------------------------------------------ LOD test */

/* The LOD criterion is left to the application (Sec. 3.3, kernel 4); the
 * reading used here (R8): visible unless one frustum plane through the eye
 * has all three vertices on its negative side; big when the refinement edge
 * (v0, v1) seen from the eye exceeds the pixel threshold: |e|^2 q > |m|^2,
 * e = v1 - v0, m = (v0 + v1) / 2. */
uint32_t or_lod_test(const float* r, const float* pl, uint32_t nplanes, float q) {
    uint32_t vis = 1u;
    for (uint32_t p = 0; p < nplanes && vis; ++p) {
        int all_out = 1;
        for (int v = 0; v < 3; ++v) {
            const float s = (pl[3 * p + 0] * r[3 * v + 0] + pl[3 * p + 1] * r[3 * v + 1]) +
                            pl[3 * p + 2] * r[3 * v + 2];
            if (!(s < 0.0f)) {
                all_out = 0;
                break;
            }
        }
        if (all_out) vis = 0u;
    }
    const float ex = r[3] - r[0], ey = r[4] - r[1], ez = r[5] - r[2];
    const float mx = 0.5f * (r[0] + r[3]), my = 0.5f * (r[1] + r[4]), mz = 0.5f * (r[2] + r[5]);
    const float L2 = (ex * ex + ey * ey) + ez * ez;
    const float R2 = (mx * mx + my * my) + mz * mz;
    const uint32_t big = (L2 * q > R2) ? 1u : 0u;
    return vis | (big << 1);
}

/* SplitMix64 (Steele, Lea & Flood 2014): counter-based hash for RANDOM mode. */
uint64_t or_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int in_sorted(const uint64_t* a, uint32_t n, uint64_t x) {
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

static void classify(const or_state* st, const or_frame* fr, const rel_roots* R, uint64_t j,
                     uint8_t* split, uint8_t* merge) {
    const int d = depth_of(st, j);
    int s = 0, m = 0;
    if (fr->mode == OR_MODE_LOD) {
        float r[9];
        bisector_rel(st, R, j, r);
        s = or_lod_test(r, &fr->planes[0][0], fr->nplanes, fr->q) == 3u && d < st->max_depth;
        if (!s && d >= 1) {
            bisector_rel(st, R, j >> 1, r);
            m = or_lod_test(r, &fr->planes[0][0], fr->nplanes, fr->q) != 3u;
        }
    } else if (fr->mode == OR_MODE_FORCE_SPLIT) {
        s = d < st->max_depth;
    } else if (fr->mode == OR_MODE_FORCE_MERGE) {
        m = d >= 1;
    } else if (fr->mode == OR_MODE_RANDOM) {
        const uint64_t key = or_splitmix64(((uint64_t)fr->seed << 32) | (uint64_t)st->frame);
        s = d < st->max_depth && (or_splitmix64(j ^ key) & 7u) == 0u;
        m = !s && d >= 1 && (or_splitmix64((j >> 1) ^ key) & 1u);
    } else if (fr->mode == OR_MODE_LIST) {
        s = d < st->max_depth && in_sorted(fr->split_list, fr->n_split, j);
        m = !s && d >= 1 && in_sorted(fr->merge_list, fr->n_merge, j);
    }
    *split = (uint8_t)s;
    *merge = (uint8_t)m;
}

/* ------------------------------------------------ chains and groups */

/* Command form of Alg. 3 on the frame-start state (R5 reading): R on b,
 * then along Twin: a diamond partner gets R and ends the chain; a coarser
 * bisector t gets R plus N (P) when b's refinement edge is t's Next (Prev)
 * edge, and the walk continues from t. Returns the allocation count
 * 2 + 3 * (coarser members) + 2 * (diamond end). */
static int chain(const or_state* st, uint32_t b, uint8_t* bits, uint32_t* cost) {
    uint32_t cur = b, c = 2;
    if (bits) bits[b] |= R_BIT;
    for (int guard = 0;; ++guard) {
        if (guard > 64) return OR_EINTERNAL;
        const uint32_t t = st->twn[cur];
        if (t == OR_NULL) break;
        if (st->twn[t] == cur) {
            if (bits) bits[t] |= R_BIT;
            c += 2;
            break;
        }
        if (depth_of(st, st->heap[t]) + 1 != depth_of(st, st->heap[cur])) return OR_EINTERNAL;
        if (st->nxt[t] == cur) {
            if (bits) bits[t] |= R_BIT | N_BIT;
        } else if (st->prv[t] == cur) {
            if (bits) bits[t] |= R_BIT | P_BIT;
        } else {
            return OR_EINTERNAL;
        }
        c += 3;
        cur = t;
    }
    *cost = c;
    return OR_OK;
}

typedef struct {
    uint32_t m[4];
    int n;
    uint32_t minm;
    uint64_t parent[2];
    int np;
} group_t;

/* Alg. 4 on the frame-start state: the sibling j2, the bisector j3 across
 * the outer half of the refinement edge; a border pair when j3 is null, a
 * quad when j3 and its sibling j4 are at the same depth. */
static int find_group(const or_state* st, uint32_t s1, group_t* g) {
    const uint64_t j1 = st->heap[s1];
    if (depth_of(st, j1) < 1) return 0;
    const int bit = (int)(j1 & 1u);
    const uint32_t s2 = bit ? st->prv[s1] : st->nxt[s1];
    const uint32_t s3 = bit ? st->nxt[s1] : st->prv[s1];
    if (s2 == OR_NULL || (st->heap[s2] >> 1) != (j1 >> 1)) return 0;
    g->m[0] = s1;
    g->m[1] = s2;
    if (s3 == OR_NULL) {
        g->n = 2;
    } else {
        const uint64_t j3 = st->heap[s3];
        if (bitlen64(j3) != bitlen64(j1) || (j3 >> 1) == (j1 >> 1)) return 0;
        const uint32_t s4 = bit ? st->nxt[s3] : st->prv[s3];
        if (s4 == OR_NULL || (st->heap[s4] >> 1) != (j3 >> 1)) return 0;
        g->m[2] = s3;
        g->m[3] = s4;
        g->n = 4;
    }
    g->minm = g->m[0];
    for (int i = 1; i < g->n; ++i)
        if (st->heap[g->m[i]] < st->heap[g->minm]) g->minm = g->m[i];
    g->np = 0;
    for (int i = 0; i < g->n; ++i) {
        const uint64_t p = st->heap[g->m[i]] >> 1;
        int seen = 0;
        for (int k = 0; k < g->np; ++k) seen |= g->parent[k] == p;
        if (!seen) g->parent[g->np++] = p;
    }
    if (g->np == 2 && g->parent[1] < g->parent[0]) {
        const uint64_t t = g->parent[0];
        g->parent[0] = g->parent[1];
        g->parent[1] = t;
    }
    return 1;
}

/* ------------------------------------------ textbook node graph (B) */

typedef struct {
    or_state* st;
    uint32_t cap;
    uint8_t* alive_old; /* [cap] */
    uint64_t* heap;     /* new nodes, id = cap + k */
    uint32_t *tw, *nx, *pv, *origin;
    uint8_t* alive;
    uint32_t nn, ncap;
    int err;
} graph;

static uint32_t* G_TW(graph* G, uint32_t id) { return id < G->cap ? &G->st->twn[id] : &G->tw[id - G->cap]; }
static uint32_t* G_NX(graph* G, uint32_t id) { return id < G->cap ? &G->st->nxt[id] : &G->nx[id - G->cap]; }
static uint32_t* G_PV(graph* G, uint32_t id) { return id < G->cap ? &G->st->prv[id] : &G->pv[id - G->cap]; }
static uint64_t G_HEAP(graph* G, uint32_t id) { return id < G->cap ? G->st->heap[id] : G->heap[id - G->cap]; }
static uint32_t G_ORIGIN(graph* G, uint32_t id) { return id < G->cap ? id : G->origin[id - G->cap]; }
static uint8_t* G_ALIVE(graph* G, uint32_t id) { return id < G->cap ? &G->alive_old[id] : &G->alive[id - G->cap]; }

static uint32_t g_new(graph* G, uint64_t heap, uint32_t origin) {
    if (G->nn == G->ncap) {
        const uint32_t nc = G->ncap ? 2u * G->ncap : 1024u;
        G->heap = (uint64_t*)realloc(G->heap, sizeof(uint64_t) * nc);
        G->tw = (uint32_t*)realloc(G->tw, sizeof(uint32_t) * nc);
        G->nx = (uint32_t*)realloc(G->nx, sizeof(uint32_t) * nc);
        G->pv = (uint32_t*)realloc(G->pv, sizeof(uint32_t) * nc);
        G->origin = (uint32_t*)realloc(G->origin, sizeof(uint32_t) * nc);
        G->alive = (uint8_t*)realloc(G->alive, nc);
        if (!G->heap || !G->tw || !G->nx || !G->pv || !G->origin || !G->alive) {
            G->err = OR_ENOMEM;
            return OR_NULL;
        }
        G->ncap = nc;
    }
    const uint32_t k = G->nn++;
    G->heap[k] = heap;
    G->tw[k] = G->nx[k] = G->pv[k] = OR_NULL;
    G->origin[k] = origin;
    G->alive[k] = 1;
    return G->cap + k;
}

/* Alg. 5: the neighbours of the split bisector x now see its children. */
static int refine_pointers(graph* G, uint32_t x, uint32_t next, uint32_t prev, uint32_t c0, uint32_t c1) {
    if (next != OR_NULL) {
        if (*G_PV(G, next) == x)
            *G_PV(G, next) = c1;
        else if (*G_TW(G, next) == x)
            *G_TW(G, next) = c1;
        else
            return OR_EINTERNAL;
    }
    if (prev != OR_NULL) {
        if (*G_NX(G, prev) == x)
            *G_NX(G, prev) = c0;
        else if (*G_TW(G, prev) == x)
            *G_TW(G, prev) = c0;
        else
            return OR_EINTERNAL;
    }
    return OR_OK;
}

/* Split of a mutual-twin pair (x, k) with the links of Table 1. */
static int g_split_pair(graph* G, uint32_t x, uint32_t k) {
    const uint64_t jx = G_HEAP(G, x), jk = G_HEAP(G, k);
    const uint32_t ox = G_ORIGIN(G, x), ok = G_ORIGIN(G, k);
    const uint32_t nxx = *G_NX(G, x), pvx = *G_PV(G, x), nxk = *G_NX(G, k), pvk = *G_PV(G, k);
    if (nxx == k || pvx == k || nxk == x || pvk == x) return OR_EINTERNAL;
    const uint32_t c0 = g_new(G, 2 * jx, ox), c1 = g_new(G, 2 * jx + 1, ox);
    const uint32_t e0 = g_new(G, 2 * jk, ok), e1 = g_new(G, 2 * jk + 1, ok);
    if (G->err) return G->err;
    *G_NX(G, c0) = c1; *G_PV(G, c0) = e1; *G_TW(G, c0) = pvx;
    *G_NX(G, c1) = e0; *G_PV(G, c1) = c0; *G_TW(G, c1) = nxx;
    *G_NX(G, e0) = e1; *G_PV(G, e0) = c1; *G_TW(G, e0) = pvk;
    *G_NX(G, e1) = c0; *G_PV(G, e1) = e0; *G_TW(G, e1) = nxk;
    int e = refine_pointers(G, x, nxx, pvx, c0, c1);
    if (!e) e = refine_pointers(G, k, nxk, pvk, e0, e1);
    *G_ALIVE(G, x) = 0;
    *G_ALIVE(G, k) = 0;
    return e;
}

/* Split of a border bisector (null Twin), Table 1 with b_k = null. */
static int g_split_one(graph* G, uint32_t x) {
    const uint64_t jx = G_HEAP(G, x);
    const uint32_t ox = G_ORIGIN(G, x);
    const uint32_t nxx = *G_NX(G, x), pvx = *G_PV(G, x);
    const uint32_t c0 = g_new(G, 2 * jx, ox), c1 = g_new(G, 2 * jx + 1, ox);
    if (G->err) return G->err;
    *G_NX(G, c0) = c1; *G_PV(G, c0) = OR_NULL; *G_TW(G, c0) = pvx;
    *G_NX(G, c1) = OR_NULL; *G_PV(G, c1) = c0; *G_TW(G, c1) = nxx;
    const int e = refine_pointers(G, x, nxx, pvx, c0, c1);
    *G_ALIVE(G, x) = 0;
    return e;
}

/* Alg. 3. After the recursive call Twin(x) points to the child of the old
 * twin that faces x (reading of the pseudocode, which passes the stale b_k). */
static int g_refine(graph* G, uint32_t x, int guard) {
    if (guard > 70 || !*G_ALIVE(G, x)) return OR_EINTERNAL;
    uint32_t k = *G_TW(G, x);
    if (k == OR_NULL) return g_split_one(G, x);
    if (*G_TW(G, k) != x) {
        const int e = g_refine(G, k, guard + 1);
        if (e) return e;
        k = *G_TW(G, x);
        if (k == OR_NULL || *G_TW(G, k) != x) return OR_EINTERNAL;
    }
    if (bitlen64(G_HEAP(G, x)) != bitlen64(G_HEAP(G, k))) return OR_EINTERNAL;
    return g_split_pair(G, x, k);
}

/* Alg. 4 merge with the parent links (Table 1 read backwards) and Alg. 6. */
static int g_decimate(graph* G, const group_t* g) {
    uint32_t a[2], b[2], P[2];
    for (int pi = 0; pi < g->np; ++pi) {
        a[pi] = b[pi] = OR_NULL;
        for (int i = 0; i < g->n; ++i) {
            const uint64_t j = G_HEAP(G, g->m[i]);
            if (j == 2 * g->parent[pi]) a[pi] = g->m[i];
            if (j == 2 * g->parent[pi] + 1) b[pi] = g->m[i];
        }
        if (a[pi] == OR_NULL || b[pi] == OR_NULL) return OR_EINTERNAL;
        for (int i = 0; i < g->n; ++i)
            if (!*G_ALIVE(G, g->m[i])) return OR_EINTERNAL;
    }
    for (int pi = 0; pi < g->np; ++pi) P[pi] = g_new(G, g->parent[pi], g->minm);
    if (G->err) return G->err;
    for (int pi = 0; pi < g->np; ++pi) {
        *G_NX(G, P[pi]) = *G_TW(G, b[pi]);
        *G_PV(G, P[pi]) = *G_TW(G, a[pi]);
        *G_TW(G, P[pi]) = g->np == 2 ? P[1 - pi] : OR_NULL;
    }
    for (int pi = 0; pi < g->np; ++pi) {
        const uint32_t next = *G_TW(G, b[pi]), prev = *G_TW(G, a[pi]);
        if (next != OR_NULL) {
            if (*G_PV(G, next) == b[pi])
                *G_PV(G, next) = P[pi];
            else if (*G_TW(G, next) == b[pi])
                *G_TW(G, next) = P[pi];
            else
                return OR_EINTERNAL;
        }
        if (prev != OR_NULL) {
            if (*G_NX(G, prev) == a[pi])
                *G_NX(G, prev) = P[pi];
            else if (*G_TW(G, prev) == a[pi])
                *G_TW(G, prev) = P[pi];
            else
                return OR_EINTERNAL;
        }
    }
    for (int i = 0; i < g->n; ++i) *G_ALIVE(G, g->m[i]) = 0;
    return OR_OK;
}

typedef struct {
    uint32_t rank;
    uint64_t key; /* heap ID shifted left to 64 significant bits */
    uint64_t heap;
    uint32_t id;
} new_item;

static int cmp_new_item(const void* x, const void* y) {
    const new_item* p = (const new_item*)x;
    const new_item* q = (const new_item*)y;
    if (p->rank != q->rank) return p->rank < q->rank ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return 0;
}

/* Heap IDs of the leaves of a SPLIT bisector j with command bits, in
 * depth-first order, child-0 subtree first (R5/R7 readings); comparing heap
 * IDs left-aligned to the same bit length gives the same order. */
static int family_heaps(uint64_t j, uint8_t bits, uint64_t out[4]) {
    int n = 0;
    if (bits & P_BIT) {
        out[n++] = 4 * j;
        out[n++] = 4 * j + 1;
    } else {
        out[n++] = 2 * j;
    }
    if (bits & N_BIT) {
        out[n++] = 4 * j + 2;
        out[n++] = 4 * j + 3;
    } else {
        out[n++] = 2 * j + 1;
    }
    return n;
}

/* ------------------------------------------------------------- update */

int or_update(or_state* st, const or_frame* fr, or_stats* stats) {
    const uint32_t cap = st->cap;
    const int32_t D = st->D;
    const uint32_t N = st->cbt[1];
    const uint32_t F = cap - N;
    or_stats S;
    memset(&S, 0, sizeof(S));
    S.live_before = N;
    S.free_before = F;
    S.frame = st->frame;
    int rc = OR_OK;

    uint32_t* L = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
    uint32_t* rank = (uint32_t*)malloc(sizeof(uint32_t) * cap);
    uint8_t* sw = (uint8_t*)calloc(cap, 1);
    uint8_t* mw = (uint8_t*)calloc(cap, 1);
    uint8_t* sgrant = (uint8_t*)calloc(cap, 1);
    uint8_t* mgrant = (uint8_t*)calloc(cap, 1);
    uint8_t* bits = (uint8_t*)calloc(cap, 1);
    uint8_t* merged = (uint8_t*)calloc(cap, 1);
    uint32_t* scost = (uint32_t*)calloc(N ? N : 1, sizeof(uint32_t));
    uint32_t* mcost = (uint32_t*)calloc(N ? N : 1, sizeof(uint32_t));
    graph G;
    memset(&G, 0, sizeof(G));
    G.st = st;
    G.cap = cap;
    G.alive_old = (uint8_t*)calloc(cap, 1);
    rel_roots R;
    memset(&R, 0, sizeof(R));
    new_item* items = NULL;
    uint32_t* nslot = NULL;
    if (!L || !rank || !sw || !mw || !sgrant || !mgrant || !bits || !merged || !scost || !mcost ||
        !G.alive_old) {
        rc = OR_ENOMEM;
        goto done;
    }

    /* 1. CachePointers: the i-th live bisector (Alg. 7). */
    for (uint32_t i = 0; i < N; ++i) {
        L[i] = or_cbt_one_to_bit(D, st->cbt, i);
        rank[L[i]] = i;
        G.alive_old[L[i]] = 1;
    }

    /* 2. GenerateCommands, decision part: wishes on the frame-start state. */
    if (fr->mode == OR_MODE_LOD) {
        rc = make_rel(st, fr->eye, fr->precision, fr->fixed_shift, fr->sphere_radius, &fr->disp, &R);
        if (rc) goto done;
    }
    for (uint32_t i = 0; i < N; ++i) classify(st, fr, &R, st->heap[L[i]], &sw[L[i]], &mw[L[i]]);

    /* 3. Requests and the gate: merges first, then splits, ascending slot. */
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t s = L[i];
        if (sw[s]) {
            ++S.split_wishes;
            if (fr->gate == OR_GATE_PAPER) {
                scost[i] = 3u * (uint32_t)depth_of(st, st->heap[s]) + 4u;
            } else {
                rc = chain(st, s, NULL, &scost[i]);
                if (rc) goto done;
            }
        }
        if (mw[s]) {
            group_t g;
            if (find_group(st, s, &g) && g.minm == s) {
                int all = 1;
                for (int k = 0; k < g.n; ++k) all &= mw[g.m[k]];
                if (all) {
                    mcost[i] = fr->gate == OR_GATE_PAPER ? 2u : (uint32_t)g.np;
                    ++S.merge_candidates;
                }
            }
        }
    }
    uint64_t mp = 0, mg = 0, sp = 0;
    for (uint32_t i = 0; i < N; ++i)
        if (mcost[i]) {
            mp += mcost[i];
            if (mp <= F) {
                mgrant[L[i]] = 1;
                mg = mp;
                ++S.merge_granted;
            }
        }
    for (uint32_t i = 0; i < N; ++i)
        if (scost[i]) {
            sp += scost[i];
            if (mg + sp <= F) {
                sgrant[L[i]] = 1;
                ++S.split_granted;
            }
        }

    /* 4. Command bits along the granted chains; merge validity. */
    for (uint32_t i = 0; i < N; ++i)
        if (sgrant[L[i]]) {
            uint32_t c;
            rc = chain(st, L[i], bits, &c);
            if (rc) goto done;
        }
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t s = L[i];
        group_t g;
        if (!mw[s] || bits[s] || !find_group(st, s, &g)) continue;
        int ok = mgrant[g.minm];
        for (int k = 0; k < g.n; ++k) ok &= mw[g.m[k]] && !bits[g.m[k]];
        merged[s] = (uint8_t)ok;
    }

    /* 5. The textbook topology change, one request at a time (in slot order,
     *    or in a seeded permutation to check that the order does not matter). */
    {
        uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
        if (!order) {
            rc = OR_ENOMEM;
            goto done;
        }
        for (uint32_t i = 0; i < N; ++i) order[i] = L[i];
        if (st->order_seed) {
            uint64_t key = st->order_seed;
            for (uint32_t i = N; i > 1; --i) {
                key = or_splitmix64(key);
                const uint32_t r = (uint32_t)(key % i);
                const uint32_t t = order[i - 1];
                order[i - 1] = order[r];
                order[r] = t;
            }
        }
        for (uint32_t i = 0; i < N && !rc; ++i) {
            const uint32_t s = order[i];
            if (sgrant[s] && *G_ALIVE(&G, s)) rc = g_refine(&G, s, 0);
        }
        for (uint32_t i = 0; i < N && !rc; ++i) {
            const uint32_t s = order[i];
            group_t g;
            if (!merged[s] || !find_group(st, s, &g) || g.minm != s) continue;
            rc = g_decimate(&G, &g);
            ++S.merge_groups;
        }
        free(order);
        if (rc) goto done;
    }

    /* 6. Slots for the new bisectors (R7): in ascending slot of the bisector
     *    they come from, then depth-first; with the (A)/(B) cross-check. */
    uint32_t A = 0;
    items = (new_item*)malloc(sizeof(new_item) * (G.nn ? G.nn : 1));
    nslot = (uint32_t*)malloc(sizeof(uint32_t) * (G.nn ? G.nn : 1));
    if (!items || !nslot) {
        rc = OR_ENOMEM;
        goto done;
    }
    for (uint32_t k = 0; k < G.nn; ++k) {
        nslot[k] = OR_NULL;
        if (!G.alive[k]) continue;
        items[A].rank = rank[G.origin[k]];
        items[A].heap = G.heap[k];
        items[A].key = G.heap[k] << (64 - bitlen64(G.heap[k]));
        items[A].id = k;
        ++A;
    }
    qsort(items, A, sizeof(new_item), cmp_new_item);
    if (A > F) {
        rc = OR_EINTERNAL;
        goto done;
    }
    for (uint32_t a = 0; a < A; ++a) nslot[items[a].id] = or_cbt_zero_to_bit(D, st->cbt, a);
    {
        uint32_t a = 0;
        for (uint32_t i = 0; i < N; ++i) {
            const uint32_t s = L[i];
            const int keep = !bits[s] && !merged[s];
            if (keep != (int)G.alive_old[s]) ++S.ab_mismatch;
            uint64_t expect[4];
            int ne = 0;
            if (bits[s]) {
                ne = family_heaps(st->heap[s], bits[s], expect);
                ++S.split_bisectors;
            } else if (merged[s]) {
                ++S.merged_bisectors;
                group_t g;
                if (find_group(st, s, &g) && g.minm == s) {
                    ne = g.np;
                    for (int p = 0; p < g.np; ++p) expect[p] = g.parent[p];
                }
            }
            int got = 0;
            while (a < A && items[a].rank == i) {
                if (got >= ne || items[a].heap != expect[got]) ++S.ab_mismatch;
                ++got;
                ++a;
            }
            if (got != ne) ++S.ab_mismatch;
        }
    }

    /* 7. Write the new records, UpdateBitfield, SumReduction. */
#define MAPID(id) ((id) == OR_NULL ? OR_NULL : ((id) < cap ? (id) : nslot[(id) - cap]))
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t s = L[i];
        if (!G.alive_old[s]) continue;
        st->twn[s] = MAPID(st->twn[s]);
        st->nxt[s] = MAPID(st->nxt[s]);
        st->prv[s] = MAPID(st->prv[s]);
    }
    for (uint32_t a = 0; a < A; ++a) {
        const uint32_t k = items[a].id, slot = nslot[k];
        st->heap[slot] = G.heap[k];
        st->twn[slot] = MAPID(G.tw[k]);
        st->nxt[slot] = MAPID(G.nx[k]);
        st->prv[slot] = MAPID(G.pv[k]);
    }
#undef MAPID
    for (uint32_t i = 0; i < N; ++i)
        if (!G.alive_old[L[i]]) st->cbt[cap + L[i]] = 0u;
    for (uint32_t a = 0; a < A; ++a) st->cbt[cap + nslot[items[a].id]] = 1u;
    or_cbt_sum_reduction(D, st->cbt);
    /* Every link of a live bisector must name a live bisector. */
    for (uint32_t s = 0; s < cap; ++s) {
        if (!st->cbt[cap + s]) continue;
        const uint32_t l[3] = {st->twn[s], st->nxt[s], st->prv[s]};
        for (int e = 0; e < 3; ++e)
            if (l[e] != OR_NULL && (l[e] >= cap || !st->cbt[cap + l[e]])) rc = OR_EINTERNAL;
        const int d = depth_of(st, st->heap[s]);
        if ((uint32_t)d > S.max_depth) S.max_depth = (uint32_t)d;
    }
    S.allocated = A;
    S.live_after = st->cbt[1];
    st->frame += 1u;

done:
    free(L);
    free(rank);
    free(sw);
    free(mw);
    free(sgrant);
    free(mgrant);
    free(bits);
    free(merged);
    free(scost);
    free(mcost);
    free(G.alive_old);
    free(G.heap);
    free(G.tw);
    free(G.nx);
    free(G.pv);
    free(G.origin);
    free(G.alive);
    free(items);
    free(nslot);
    free_rel(&R);
    if (stats) *stats = S;
    return rc;
}

void or_set_order_seed(or_state* st, uint64_t seed) { st->order_seed = seed; }

int or_chain_cost(const or_state* st, uint32_t slot, uint32_t* cost) {
    if (slot >= st->cap || !st->cbt[st->cap + slot]) return OR_EINVAL;
    return chain(st, slot, NULL, cost);
}

uint32_t or_leaves(const or_state* st, uint32_t* slots, uint64_t* heap, uint32_t* links) {
    uint32_t n = 0;
    for (uint32_t s = 0; s < st->cap; ++s) {
        if (!st->cbt[st->cap + s]) continue;
        if (slots) slots[n] = s;
        if (heap) heap[n] = st->heap[s];
        if (links) {
            links[3 * n + 0] = st->twn[s];
            links[3 * n + 1] = st->nxt[s];
            links[3 * n + 2] = st->prv[s];
        }
        ++n;
    }
    return n;
}
