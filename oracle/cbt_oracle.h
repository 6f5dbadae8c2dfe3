/* CPU oracle for the concurrent-binary-tree adaptive bisection update.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, sequential restatement of
 * "Concurrent Binary Trees for Large-Scale Game Components" (Benyoub & Dupuy,
 * 2024). Only the tests, the package smoke check and the benchmark's CPU
 * baseline leg may load it. It shares no code with the CUDA library.
 *
 * Conventions (both implementations receive the same inputs):
 *   - bisector heap ID j: root of halfedge h is 2^ceil(log2 H) + h, children
 *     of j are 2j and 2j+1 (Sec. 2.3 "Notation"; Sec. 3.3 "Initialization",
 *     read with a marker bit above the root index);
 *   - per bisector three neighbour slots Twin/Next/Prev, null = 0xFFFFFFFF;
 *   - the CBT is the paper's binary heap of 2^(D+1) u32 (Sec. 3.1), leaves
 *     cbt[2^D + slot] hold the bitfield.
 */
#ifndef CBT_ORACLE_H
#define CBT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_NULL 0xFFFFFFFFu

enum { OR_OK = 0, OR_EINVAL = 1, OR_ECAPACITY = 2, OR_EDEPTH = 3, OR_ENOMEM = 4, OR_EINTERNAL = 10 };
enum { OR_MODE_LOD = 0, OR_MODE_FORCE_SPLIT = 1, OR_MODE_FORCE_MERGE = 2, OR_MODE_RANDOM = 3, OR_MODE_LIST = 4 };
enum { OR_PREC_FP32 = 0, OR_PREC_FIXED = 1, OR_PREC_FP64 = 2, OR_PREC_SPHERE = 3 };
enum { OR_GATE_CHAIN = 0, OR_GATE_PAPER = 1 };

/* Displacement of the LOD-tested and exported vertices (R14 reading; the
 * paper displaces the projected vertices with wave layers or elevation data
 * during refinement, Sec. 4): amplitude * fbm(position), fbm = fractal value
 * noise of `octaves` octaves (1..8) at base frequency `frequency` (lattice
 * cells per world unit), seeded by `seed`. Plain FP32 form: +z by the noise
 * of the world (x, y); sphere form: radially, by the noise of the unit
 * direction. amplitude 0 = off. */
typedef struct {
    float amplitude;
    float frequency;
    uint32_t octaves;
    uint32_t seed;
} or_disp;

typedef struct {
    double eye[3];
    float planes[5][3];
    float q;
    uint32_t nplanes;
    uint32_t mode;
    uint32_t seed;
    uint32_t precision;
    int32_t fixed_shift;
    uint32_t gate;
    const uint64_t* split_list; /* sorted, MODE_LIST only */
    uint32_t n_split;
    const uint64_t* merge_list; /* sorted, MODE_LIST only */
    uint32_t n_merge;
    double sphere_radius;       /* PREC_SPHERE: radius of the sphere about the origin */
    or_disp disp;               /* FP32 and sphere forms only */
} or_frame;

typedef struct {
    uint32_t live_before, live_after, free_before;
    uint32_t split_wishes, merge_candidates;
    uint32_t split_granted, merge_granted;
    uint32_t split_bisectors, merged_bisectors, merge_groups;
    uint32_t allocated;
    uint32_t max_depth;
    uint32_t ab_mismatch;
    uint32_t frame;
} or_stats;

typedef struct or_state or_state;

/* Faces -> halfedges (Sec. 2.1): halfedges of face f are consecutive in face
 * order; Twin matched by the reversed vertex pair, -1 on a border. */
int or_halfedges_from_faces(int32_t F, const int32_t* face_sizes, const int32_t* face_verts,
                            int32_t H, int32_t* twin, int32_t* next, int32_t* prev,
                            int32_t* vert, int32_t* face);

int or_create(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
              const int32_t* vert, const int32_t* face, int32_t V, const double* pos,
              int32_t D, int32_t max_depth, or_state** out);
void or_destroy(or_state* st);
int or_update(or_state* st, const or_frame* fr, or_stats* stats);

uint32_t or_live_count(const or_state* st);
int32_t or_ceil_log2_H(const or_state* st);
/* Copies of the whole state (dead slots hold stale values). */
void or_export(const or_state* st, uint32_t* cbt, uint64_t* heap, uint32_t* twin,
               uint32_t* next, uint32_t* prev);
/* Live bisectors in ascending slot order: slot, heap ID, links [N][3] as
 * (twin, next, prev). Returns N. */
uint32_t or_leaves(const or_state* st, uint32_t* slots, uint64_t* heap, uint32_t* links);
/* FP32 vertices [N][3][3] of the live bisectors relative to ``origin`` using
 * the given precision form; and the FP64 reference positions (absolute). */
void or_vertices(const or_state* st, const double origin[3], uint32_t precision,
                 int32_t fixed_shift, double sphere_radius, const or_disp* disp, float* out);
void or_vertices_f64(const or_state* st, double* out);
/* Indexed form of the live bisectors (R15 reading): corners that are the
 * same point of the subdivided surface share one vertex; vertices are
 * numbered in order of first occurrence over (live index, corner).
 * indices[N][3]; vertices[nv][3] copied from tri_vertices[N][3][3] (the
 * per-bisector vertices, as or_vertices writes them) at each vertex's first
 * occurrence (both may be NULL); tri_ids[N] = heap IDs (may be NULL). */
int or_export_indexed(const or_state* st, const float* tri_vertices, float* vertices, uint32_t* indices,
                      uint64_t* tri_ids, uint32_t* n_vertices);
void or_root_table(const or_state* st, double* out);

/* Test hooks: the order in which the textbook step applies the requests
 * (0 = ascending slot), and the compatibility-chain allocation count of a
 * live bisector on the current state. */
void or_set_order_seed(or_state* st, uint64_t seed);
int or_chain_cost(const or_state* st, uint32_t slot, uint32_t* cost);

/* Building blocks exposed for the pins. */
void or_cbt_sum_reduction(int32_t D, uint32_t* cbt);
uint32_t or_cbt_one_to_bit(int32_t D, const uint32_t* cbt, uint32_t index);
void or_cbt_compact(int32_t D, const uint32_t* cbt, uint32_t* out);
uint32_t or_cbt_zero_to_bit(int32_t D, const uint32_t* cbt, uint32_t index);
void or_decode_weights(uint64_t j, int32_t ch, uint64_t* W9);
uint64_t or_splitmix64(uint64_t x);
/* The displacement's parts: the lowbias32 integer hash and the fractal
 * value noise of n (2 or 3) FP32 coordinates. */
uint32_t or_lowbias32(uint32_t x);
float or_fbm(const float* x, int32_t n, float frequency, uint32_t octaves, uint32_t seed);
/* LOD test on three FP32 camera-relative vertices: bit0 visible, bit1 big. */
uint32_t or_lod_test(const float* r9, const float* planes15, uint32_t nplanes, float q);

#ifdef __cplusplus
}
#endif
#endif
