/* cbt.h - C ABI of the GB300 (sm_103a) adaptive-bisection library.
 *
 * Implements the per-frame update of "Concurrent Binary Trees for
 * Large-Scale Game Components" (Benyoub & Dupuy, 2024): every halfedge of a
 * polygon mesh is a root bisector (Sec. 2.2); each frame the live bisectors
 * are classified against a level-of-detail test, split conformingly along
 * their compatibility chains (Alg. 3, Table 1), merged back (Alg. 4) or kept,
 * and a concurrent binary tree (CBT, Sec. 3.1-3.2) serves as the memory pool
 * of 2^D bisector slots.
 *
 * Conventions
 *   - A bisector is identified by its 64-bit heap ID j: the root of halfedge
 *     h is 2^ceil(log2 H) + h and the children of j are 2j and 2j+1
 *     (Sec. 2.3 "Notation", Sec. 3.3 "Initialization").
 *   - Its depth is bitlength(j) - 1 - ceil(log2 H); its vertices are decoded
 *     from j by Alg. 2 / Eq. 1.
 *   - Each live bisector holds three neighbour slots Twin, Next, Prev (the
 *     bisectors across its edges (v0,v1), (v1,v2), (v2,v0)); a missing
 *     neighbour is CBT_NULL.
 *   - Slots are indices in [0, 2^D). Live bisectors are always reported in
 *     ascending slot order, which is the order of Alg. 7 (OneToBitID).
 *
 * Memory and streams
 *   - The caller owns all device memory: the workspace passed to cbt_create
 *     (size from cbt_workspace_bytes) must stay allocated and unmoved until
 *     cbt_destroy, and output buffers are caller-allocated device memory.
 *   - Host arrays passed to cbt_create are read during the call only.
 *   - A state is used by one host thread at a time. Calls on one state are
 *     ordered by the stream given to them; the caller orders streams when
 *     it uses more than one for the same state.
 *   - Calls marked "asynchronous" only enqueue work; calls marked
 *     "synchronous" wait for the stream.
 *
 * Errors: every entry point returns 0 (CBT_OK) or one of the codes below.
 * Device-side checks (a non-conforming neighbourhood, a bounded wait that
 * gave up) set a sticky error word read by cbt_stats().
 */
#ifndef CBT_H
#define CBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cbt_stream_t; /* a cudaStream_t; NULL = default stream */

#define CBT_NULL 0xFFFFFFFFu

enum {
    CBT_OK = 0,
    CBT_EINVAL = 1,     /* bad argument or malformed halfedge mesh */
    CBT_ECAPACITY = 2,  /* 2^D < H, or D outside [1, 30] */
    CBT_EDEPTH = 3,     /* ceil(log2 H) + 1 + max_depth > 63 */
    CBT_ENOMEM = 4,     /* workspace or output buffer too small */
    CBT_ECUDA = 5,      /* a CUDA launch or runtime call failed */
    CBT_EDEVICE = 6,    /* the sticky device error word is set */
    CBT_ETIMEOUT = 7    /* a bounded device wait gave up */
};

/* Sticky device error bits (cbt_frame_stats.error). */
enum {
    CBT_DERR_CHAIN = 1u,    /* compatibility chain not one level coarser */
    CBT_DERR_LINK = 2u,     /* non-conforming neighbourhood while relinking */
    CBT_DERR_TIMEOUT = 4u,  /* a look-back wait hit its iteration limit */
    CBT_DERR_RANGE = 8u,    /* fixed-point root offset outside 62 bits */
    CBT_DERR_OVERFLOW = 16u /* more allocations than free slots */
};

/* Wish modes: the LOD test of Sec. 3.3 kernel 4, or test modes. */
enum { CBT_MODE_LOD = 0, CBT_MODE_FORCE_SPLIT = 1, CBT_MODE_FORCE_MERGE = 2, CBT_MODE_RANDOM = 3,
       CBT_MODE_LIST = 4 };
/* Vertex evaluation: FP32, fixed point with exact integer sums, FP64, or
 * projected onto a sphere about the world origin (radius sphere_radius) in
 * FP64 before the camera offset (the paper projects the vertices onto a
 * sphere during refinement, Sec. 4). */
enum { CBT_PREC_FP32 = 0, CBT_PREC_FIXED = 1, CBT_PREC_FP64 = 2, CBT_PREC_SPHERE = 3 };
/* Allocation budget per request: exact chain cost, or the paper's 3d + 4. */
enum { CBT_GATE_CHAIN = 0, CBT_GATE_PAPER = 1 };

/* One frame's inputs (Sec. 3.3 kernel 4 leaves the LOD criterion to the
 * application; this library's criterion is described at cbt_update).
 * planes: inward normals of up to five planes through the eye, FP32.
 * q: ((viewport height / (2 tan(fovy / 2))) / threshold_px)^2 in FP32.
 * split_list / merge_list: sorted DEVICE arrays of heap IDs (LIST mode).
 * vertices_out: optional DEVICE buffer of vertices_cap * 9 floats (4-byte
 * aligned; 16-byte aligned lets the export store 16 bytes at a time); when
 * set, the frame ends by writing the vertices of the new live bisectors
 * (ascending slot order) relative to eye in the frame's precision, as
 * cbt_vertices does; rows beyond vertices_cap are not written (size it 2^D
 * rows to be safe).
 * sphere_radius: CBT_PREC_SPHERE only, the radius (> 0) of the sphere about
 * the world origin onto which the vertices (LOD test and export) are
 * projected.
 * disp_*: displacement of the vertices (LOD test and export) by seeded
 * fractal value noise, standing in for the paper's wave layers and elevation
 * data (Sec. 4). disp_amplitude 0 turns it off; otherwise CBT_PREC_FP32 or
 * CBT_PREC_SPHERE, disp_frequency > 0 (lattice cells per world unit at the
 * first octave; per unit of direction on the sphere) and disp_octaves in
 * 1..8, else CBT_EINVAL. FP32 form: z += amplitude * fbm(world x, y); sphere
 * form: the radius grows by amplitude * fbm(unit direction). The noise:
 * lowbias32 lattice hash chained from seed ^ octave over the coordinates
 * (last to first), values (h >> 8) 2^-23 - 1, smoothstep-weighted blends
 * along x, then y, then z, octave o at frequency f 2^o and weight 2^-o. */
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
    const uint64_t* split_list;
    uint32_t n_split;
    const uint64_t* merge_list;
    uint32_t n_merge;
    float* vertices_out;
    uint32_t vertices_cap;
    double sphere_radius; /* CBT_PREC_SPHERE: the sphere's radius (> 0), else unused */
    float disp_amplitude; /* displacement height scale, world units; 0 = off */
    float disp_frequency; /* lattice cells per unit at the first octave */
    uint32_t disp_octaves;
    uint32_t disp_seed;
} cbt_frame;

/* A pinhole camera, FP64 world units: the eye, the point looked at, an up
 * direction (need not be unit length), the vertical field of view in
 * radians, width / height, and the viewport in pixels. */
typedef struct {
    double eye[3];
    double target[3];
    double up[3];
    double fovy_rad;
    double aspect;
    int32_t width_px;
    int32_t height_px;
} cbt_camera;

/* The LOD inputs of a frame from a camera and a threshold of tau_px pixels
 * (the paper leaves the criterion to the application, Sec. 3.3 kernel 4;
 * this library's reading is described at cbt_update): writes frame->eye
 * (the camera's eye), frame->planes (the inward normals of the four side
 * planes of the view frustum and of the near plane, all through the eye),
 * frame->nplanes (5, or 0 when frustum is 0: no culling) and frame->q =
 * ((height_px / (2 tan(fovy / 2))) / tau_px)^2; the other fields are left
 * as they are. The derivation is FP64 with one rounding to FP32 at the end:
 * f = (target - eye) / |target - eye|; the up direction is replaced by +y
 * (by +x when |f.y| >= 0.9) when |f . up / |up|| > 0.999; r = f x up / |f x
 * up|; u = r x f; with t_y = tan(fovy / 2) and t_x = aspect t_y the planes
 * are t_x f + r, t_x f - r, t_y f + u, t_y f - u and f. Every norm is
 * sqrt((x x + y y) + z z) and every operation is rounded on its own.
 * Errors: CBT_EINVAL (NULL pointers, tau_px not positive and finite, fovy
 * outside (0, pi), aspect not positive, an empty viewport, eye = target, a
 * zero up direction or one along the view's axis after the fallback,
 * values that are not finite). Host only, synchronous. */
int cbt_frame_from_camera(const cbt_camera* cam, float tau_px, int frustum, cbt_frame* frame);

/* Per-frame counters (read with cbt_stats). */
typedef struct {
    uint32_t live_before, live_after, free_before;
    uint32_t split_wishes, merge_candidates;
    uint32_t split_granted, merge_granted;
    uint32_t split_bisectors, merged_bisectors, merge_groups;
    uint32_t allocated;
    uint32_t relinked;  /* links of unchanged bisectors rewritten */
    uint32_t frame;     /* frames completed so far */
    uint32_t error;     /* sticky CBT_DERR_* bits */
} cbt_frame_stats;

typedef struct cbt_state cbt_state;

/* Faces -> halfedge arrays (Sec. 2.1, halfedge figure): the halfedges of face
 * f are consecutive, in face order; Next/Prev go round the face; Twin is the
 * halfedge running the other way along the same edge, -1 on a border.
 * Host arrays: face_sizes[F], face_verts[sum of sizes]; outputs [H] each.
 * Returns CBT_EINVAL for a face with fewer than 3 vertices, a size mismatch
 * or an edge used twice in the same direction. Synchronous, host only. */
int cbt_halfedges_from_faces(int32_t F, const int32_t* face_sizes, const int32_t* face_verts,
                             int32_t H, int32_t* twin, int32_t* next, int32_t* prev,
                             int32_t* vert, int32_t* face);

/* Bytes of device workspace for a mesh of H halfedges and a pool of 2^D
 * bisectors (Table 2 and Sec. 4 "Memory Consumption" list the paper's
 * layout; this one keeps a 64-bit heap ID, three 32-bit links, a 32-bit
 * command word and a 32-bit destination per slot, the CBT as a bitfield plus
 * its sum tree, and per-frame scratch). Returns 0 for invalid sizes. */
size_t cbt_workspace_bytes(int32_t H, int32_t D);

/* Builds the H root bisectors in slots 0..H-1 (Sec. 3.3 "Initialization"):
 * heap IDs 2^ceil(log2 H) + h, neighbours copied from the halfedge operators,
 * first H bits of the CBT set, sum reduction done. Root vertices follow
 * Alg. 1 (v0 = Vert(h), v1 = Vert(Next(h)), v2 = face average, summed in FP64
 * from the face's smallest halfedge index), kept in FP64.
 *   twin/next/prev/vert/face: host int32[H] (twin -1 on a border);
 *   pos: host double[V][3];
 *   D: pool of 2^D slots, ceil(log2 H) <= D <= 30;
 *   max_depth: subdivision limit, ceil(log2 H) + 1 + max_depth <= 63;
 *   workspace/bytes: caller-owned device memory, cbt_workspace_bytes() long,
 *                    256-byte aligned;
 *   out: receives the state handle (host memory owned by the library).
 * Errors: CBT_EINVAL (malformed mesh), CBT_ECAPACITY, CBT_EDEPTH,
 * CBT_ENOMEM (workspace too small), CBT_ECUDA. Synchronous: the roots and
 * their CBT are built when it returns; the host arrays may then be freed. */
int cbt_create(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
               const int32_t* vert, const int32_t* face, int32_t V, const double* pos,
               int32_t D, int32_t max_depth, void* workspace, size_t bytes,
               cbt_stream_t stream, cbt_state** out);

/* Optional per-slot cache of the sphere form's camera-independent FP64
 * points (precision CBT_PREC_SPHERE with the LOD mode; Sec. 4 decodes planet
 * vertices in FP64 every frame). Classify keeps, per slot, the FP64 point
 * and radial scale of the four vertices its LOD tests read, tagged with the
 * heap ID and a generation that changes with the radius or the displacement.
 * A bisector whose tag matches then costs one FP64 fused multiply-add and one
 * conversion per coordinate; the results are the same floats as without the
 * cache. 144 bytes per pool slot: cbt_point_cache_bytes(D) returns
 * 144 * 2^D, or 0 for D outside 1..30. */
size_t cbt_point_cache_bytes(int32_t D);

/* Attaches a point cache to a state:
 *   memory/bytes: caller-owned device memory, 16-byte aligned, at least
 *                 cbt_point_cache_bytes(D) long; it must stay allocated and
 *                 unmoved until cbt_destroy (no detach).
 * The tags are cleared on `stream`, and the call synchronises it. Call it
 * while no frame of the state is in flight on another stream. Batches and
 * servers built afterwards include the cache; ones built before run the
 * state without it (still correct).
 * Errors: CBT_EINVAL (NULL state or memory, memory not 16-byte aligned, a
 * cache already attached), CBT_ENOMEM (bytes too small), CBT_ECUDA. */
int cbt_attach_point_cache(cbt_state* st, void* memory, size_t bytes, cbt_stream_t stream);

/* One frame of the update (Sec. 3.3, the update pipeline; Alg. 9):
 *   1. the live slots in ascending order (Alg. 7, CachePointers);
 *   2. classification on the frame-start state (GenerateCommands): split
 *      wish = visible and big and depth < max_depth; merge wish = no split
 *      wish, depth >= 1 and the parent is not (visible and big). "Big" means
 *      |v1 - v0|^2 q > |(v0 + v1) / 2|^2 with camera-relative FP32 vertices;
 *      "visible" means no plane has all three vertices on its negative side;
 *   3. the gate: a split costs its compatibility-chain allocation count (or
 *      3d + 4 with CBT_GATE_PAPER), a mergeable group its parent count at
 *      its smallest heap ID; merges then splits, each in ascending slot
 *      order, are granted while the running cost stays within the free slots;
 *   4. granted splits mark their chains, groups whose members all agree and
 *      carry no split merge (Alg. 4);
 *   5. new bisectors take the free slots of the frame-start CBT in that order
 *      (Alg. 8, ReserveBlocks); records and links are written (Table 1,
 *      Alg. 5/6; FillNewBlocks, UpdateNeighbors), the bitfield updated and
 *      the sum tree rebuilt (UpdateBitfield, SumReduction).
 * Deterministic: the result does not depend on thread scheduling.
 * Errors: CBT_EINVAL (NULL arguments or bad precision/mode), CBT_ECUDA.
 * Asynchronous. */
int cbt_update(cbt_state* st, const cbt_frame* frame, cbt_stream_t stream);

/* n plain updates in one call: cbt_update(states[b], frames + b, stream)
 * for b = 0 .. n-1 in order, each instance's frame launched on its own as
 * cbt_update does (no batching), from a host loop in the library. Stops at
 * the first error and returns it (the updates before it stay enqueued).
 * Errors: those of cbt_update; CBT_EINVAL for NULL arrays or n < 0.
 * Asynchronous. */
int cbt_update_many(cbt_state* const* states, const cbt_frame* frames, int32_t n, cbt_stream_t stream);

/* Device address of page-locked, mapped host memory (cudaHostAlloc'd or
 * registered; every pinned allocation is mapped under unified addressing),
 * for outputs that kernels write straight into host memory: e.g.
 * cbt_frame.vertices_out, so that the frame's vertex export lands in the
 * host buffer with no separate copy. CBT_EINVAL for other pointers. */
int cbt_host_device_pointer(void* h_ptr, void** d_ptr);

/* The frame's vertex export, moved to the host in one call: rows [0, N) of
 * d_vertices (float[N][3][3], as cbt_update's vertices_out wrote them for
 * the current live list; N = the live count, read on the device) are
 * copied into h_vertices by a kernel with 16-byte stores through the mapped
 * address of the pinned buffer, and N is stored at *h_count (also pinned),
 * so that one stream synchronisation covers the frame, the count and the
 * copy. At most cap rows are copied; CBT_ENOMEM when N > cap (*h_count
 * still holds N). CBT_EINVAL for NULL, misaligned or unpinned host
 * pointers.
 * Synchronous. */
int cbt_vertices_to_host(cbt_state* st, const float* d_vertices, float* h_vertices, uint32_t cap,
                         uint32_t* h_count, cbt_stream_t stream);

/* Rows [0, rows) of a frame's vertex export (float[rows][3][3] at
 * d_vertices, DEVICE memory) copied into h_vertices (page-locked HOST
 * memory, at least rows rows) by the copy engine on `stream`, nothing
 * synchronised: rows is the live count, e.g. from cbt_live_count_async once
 * the caller has waited for it. With two export buffers a frame's rows go
 * out while the next frame computes. CBT_EINVAL for NULL pointers, CBT_ECUDA
 * when the copy cannot be enqueued; rows = 0 enqueues nothing. */
int cbt_vertices_to_host_async(const float* d_vertices, float* h_vertices, uint32_t rows, cbt_stream_t stream);

/* Indexed export of the live bisectors, the input of a visibility buffer
 * (the paper exports its triangulation into one, Sec. 4). Corners that are
 * the same point of the subdivided surface share one vertex: a corner's
 * identity is its exact weight row (Eq. 1) in lowest terms over the global
 * mesh vertices and face centroids of its root, so shared corners match
 * across bisectors, roots and faces and the indexed mesh is watertight.
 * Corners at a mesh vertex or face centroid are matched by that global
 * point; the others lie inside a root edge or triangle, where the conforming
 * bisection (Sec. 2.3) puts the bisectors sharing the point in one fan,
 * walked through the neighbour links.
 * Vertices are numbered in order of first occurrence over (live index,
 * corner); triangle i is live bisector i (ascending slot, as cbt_leaves).
 *   d_tri_vertices: DEVICE float[N][3][3], the per-bisector vertices of the
 *           current live list (cbt_update's vertices_out or cbt_vertices);
 *           may be NULL when d_vertices is NULL;
 *   d_workspace: DEVICE scratch of cbt_index_workspace_bytes(st,
 *           triangles_cap) bytes at least (4 bytes per pool slot, per global
 *           point and, twice, per corner), caller-owned, 256-byte aligned;
 *   d_vertices: DEVICE float[vertices_cap][3] or NULL: each vertex's
 *           position, copied from its first occurrence;
 *   d_indices: DEVICE u32[triangles_cap][3];
 *   d_heap: DEVICE u64[triangles_cap] or NULL: the triangles' heap IDs (the
 *           visibility buffer's triangle payload);
 *   *h_nvertices / *h_ntriangles receive the counts (either may be NULL).
 * The live count N is read on the device: the launches are sized for
 * triangles_cap and the call synchronises once, at the end.
 * Errors: CBT_EINVAL (NULL state, workspace or indices; vertices without
 * d_tri_vertices; a workspace not 256-byte aligned or an output not aligned
 * to its element), CBT_ENOMEM (N > triangles_cap, workspace too small, or
 * more vertices than vertices_cap: the counts are still returned),
 * CBT_EDEVICE (a live bisector whose heap ID names no root of the mesh, or
 * neighbour links that do not close a fan: a link without its way back, a
 * fan that does not return to its start or passes 64 bisectors), CBT_ECUDA.
 * Five launches on `stream`; synchronous (returns the counts).
 * cbt_index_workspace_bytes returns 0 for a NULL state. */
size_t cbt_index_workspace_bytes(const cbt_state* st, uint32_t max_live);
int cbt_index(cbt_state* st, const float* d_tri_vertices, void* d_workspace, size_t bytes, float* d_vertices,
              uint32_t vertices_cap, uint32_t* d_indices, uint32_t triangles_cap, uint64_t* d_heap,
              uint32_t* h_nvertices, uint32_t* h_ntriangles, cbt_stream_t stream);

/* Number of live bisectors (CBT root). Synchronous. */
int cbt_live_count(cbt_state* st, uint32_t* h_count, cbt_stream_t stream);

/* The same count, enqueued on `stream` after the work already there: a
 * 4-byte copy into `count`, which is DEVICE memory or page-locked HOST memory
 * (4-byte aligned, caller-owned); nothing is synchronised, so the caller
 * waits on the stream or an event recorded after it before reading. With it
 * a frame's export can be copied to the host (its size known from the
 * count) while the next frame computes. CBT_EINVAL for NULL or misaligned
 * pointers, CBT_ECUDA when the copy cannot be enqueued. Section 3.1: the
 * count is the CBT's root. */
int cbt_live_count_async(cbt_state* st, uint32_t* count, cbt_stream_t stream);

/* Copies the live bisectors, ascending slot order, into caller device
 * buffers: d_slots[N], d_heap[N], d_links[N][3] as (Twin, Next, Prev).
 * Any output may be NULL. cap = capacity of the outputs in bisectors;
 * *h_count receives N. CBT_ENOMEM when N > cap. Synchronous. */
int cbt_leaves(cbt_state* st, uint32_t* d_slots, uint64_t* d_heap, uint32_t* d_links,
               uint32_t cap, uint32_t* h_count, cbt_stream_t stream);

/* Vertices of the live bisectors, ascending slot order, as FP32 [N][3][3]
 * relative to h_origin (Alg. 2 / Eq. 1 with exact integer weights; FP32,
 * fixed-point or FP64 evaluation as `precision`; FP64 is used on the device
 * only to subtract h_origin from the root vertices). d_out: caller device
 * memory of cap * 9 floats. *h_count receives N. CBT_ENOMEM when N > cap.
 * CBT_PREC_SPHERE is not taken here (CBT_EINVAL): sphere vertices come from
 * cbt_update's vertices_out, which carries the radius. Synchronous. */
int cbt_vertices(cbt_state* st, float* d_out, const double h_origin[3], uint32_t precision,
                 int32_t fixed_shift, uint32_t cap, uint32_t* h_count, cbt_stream_t stream);

/* The CBT: d_bitfield[max(1, 2^D / 32)] u32 words (bit s%32 of word s/32 is
 * slot s) and d_sums[2 * words] in heap order: d_sums[1] is the root (live
 * count), d_sums[words + w] = popcount(word w), d_sums[k] = d_sums[2k] +
 * d_sums[2k+1]. These equal the paper's CBT heap nodes 1 .. 2*words - 1
 * (Sec. 3.1). Either may be NULL. Asynchronous. */
int cbt_cbt(cbt_state* st, uint32_t* d_bitfield, uint32_t* d_sums, cbt_stream_t stream);

/* Counters of the last frame and the sticky device error word. Returns
 * CBT_EDEVICE when that word is non-zero. Synchronous. */
int cbt_stats(cbt_state* st, cbt_frame_stats* out, cbt_stream_t stream);

/* Releases the host handle; the workspace stays the caller's. */
void cbt_destroy(cbt_state* st);

/* Number of kernel launches the last cbt_update enqueued. */
uint32_t cbt_last_launch_count(const cbt_state* st);

/* Execution form of a frame (Alg. 9). Fused (the default): the whole frame is
 * one cooperative launch of a persistent kernel whose phases are separated by
 * grid-wide barriers; every block is resident, and every barrier wait is
 * bounded (a wait that runs out makes every instance of the launch report
 * CBT_DERR_TIMEOUT). Not fused: one launch per step (cbt_kernel_name). The
 * results are identical either way. cbt_set_fused(on) may re-upload the
 * word-tile prefixes on `stream` and waits for it; cbt_fused reads the form.
 * Host only. */
int cbt_set_fused(cbt_state* st, int on, cbt_stream_t stream);
int cbt_fused(const cbt_state* st);

/* Self-test of the bounded waits of the fused form, without a fault: a
 * cooperative launch of `blocks` blocks (1..64) meets a grid barrier that
 * expects one arrival more than there are blocks, so every wait runs out
 * after `limit` polls, sets the abort word and returns; the kernel ends
 * normally and the context stays usable. d_scratch: DEVICE, 256 bytes,
 * 256-byte aligned (cleared by the call). Returns CBT_ETIMEOUT when the
 * waits gave up (the expected outcome), CBT_OK if they did not, CBT_EINVAL,
 * CBT_ECUDA. Synchronous. */
int cbt_selftest_bounded_wait(void* d_scratch, int32_t blocks, int32_t limit, cbt_stream_t stream);

/* Timing of cbt_update (off by default). Per-step form: CUDA events recorded
 * on the update's stream between its kernels, one duration per kernel
 * (cbt_kernel_name). Fused form: the device's global timer read by block 0
 * at the phase boundaries, one duration per phase (cbt_phase_name).
 * cbt_kernel_times waits for the last frame and writes up to n durations in
 * ms, in order; it returns how many were written (0 when timing is off). */
int cbt_set_timing(cbt_state* st, int on);
uint32_t cbt_kernel_times(cbt_state* st, float* ms, uint32_t n);
const char* cbt_kernel_name(uint32_t k);
const char* cbt_phase_name(uint32_t k);
/* Name of phase k of the state's last timed fused frame. A single instance
 * whose pool has at most 2^22 slots runs a frame of fewer phases (prep,
 * classify, walks, gate, alloc, fill, final, vertices; gate lasts 0 when
 * every request of the frame fits the free slots and is granted without a
 * prefix, vertices when the export is computed in final); other fused
 * frames have the phases of cbt_phase_name. */
const char* cbt_state_phase_name(const cbt_state* st, uint32_t k);

/* Update through a CUDA graph (on: the frame's launches are captured once
 * and replayed; the frame parameters reach the device through a copy from
 * pinned host memory that the graph performs). A single instance in the
 * fused form is one launch with its parameters passed by value and is
 * launched directly either way (sooner than a graph starting with a copy).
 * Results are identical either way. Host only. */
int cbt_set_graph(cbt_state* st, int on);

/* ------------------------------------------------------------------ batches
 * Many independent instances updated together: every kernel of the frame is
 * launched once for the whole batch, whose work items are (instance, tile of
 * live bisectors) pairs laid out from a device-side prefix over the
 * instances' live counts. Each instance's result is exactly the one
 * cbt_update would give it. The states keep their own workspaces; the batch
 * needs a further caller-owned device workspace for its instance table,
 * per-instance frame parameters and scan descriptors. A state may belong to
 * several batches but must not be updated by two of them (or by cbt_update)
 * concurrently. */
typedef struct cbt_batch cbt_batch;

/* Bytes of device workspace for a batch of the given states (0 if invalid). */
size_t cbt_batch_workspace_bytes(cbt_state* const* states, int32_t n);

/* Builds a batch of n distinct states; workspace is caller-owned device
 * memory of cbt_batch_workspace_bytes(), 256-byte aligned, kept until
 * cbt_batch_destroy. Errors: CBT_EINVAL, CBT_ENOMEM, CBT_ECUDA. Synchronous. */
int cbt_batch_create(cbt_state* const* states, int32_t n, void* workspace, size_t bytes,
                     cbt_stream_t stream, cbt_batch** out);

/* One frame for every instance: frames[b] is instance b's cbt_frame (as for
 * cbt_update). Asynchronous, except that it waits for the previous frame's
 * parameter copy before reusing its pinned staging buffer. */
int cbt_batch_update(cbt_batch* b, const cbt_frame* frames, cbt_stream_t stream);

/* Replay the batch frame as a CUDA graph (see cbt_set_graph). Host only. */
int cbt_batch_set_graph(cbt_batch* b, int on);

/* Online autotuner: the next 10 * rounds frames try, one per frame, the 9
 * per-step configurations (reduction / rank-to-bit tile width of 64, 128 or
 * 256 words, times 4, 8 or 16 blocks per SM for the item kernels) and the
 * fused form, and then keep the one with the smallest median frame time per
 * live bisector (the candidates run on different frames; each waits for its
 * frame and reads the batch's live count). The configuration never changes
 * the results. cbt_batch_config reads the
 * current choice (tuning = 1 while trying); cbt_batch_set_config sets a
 * per-step configuration directly (and leaves the fused form). */
int cbt_batch_autotune(cbt_batch* b, uint32_t rounds);
int cbt_batch_config(const cbt_batch* b, uint32_t* tile_words, uint32_t* blocks_per_sm, int* tuning);
int cbt_batch_set_config(cbt_batch* b, uint32_t tile_words, uint32_t blocks_per_sm, cbt_stream_t stream);

/* Execution form of the batch frame (as cbt_set_fused / cbt_fused). */
int cbt_batch_set_fused(cbt_batch* b, int on, cbt_stream_t stream);
int cbt_batch_fused(const cbt_batch* b);

/* Timing of cbt_batch_update (as cbt_set_timing / cbt_kernel_times). */
int cbt_batch_set_timing(cbt_batch* b, int on);
uint32_t cbt_batch_kernel_times(cbt_batch* b, float* ms, uint32_t n);
uint32_t cbt_batch_last_launch_count(const cbt_batch* b);

/* Releases the batch handle; the workspaces stay the caller's. */
void cbt_batch_destroy(cbt_batch* b);

/* ------------------------------------------------------------------ serving
 * A set of resident instances served by ticks: each tick updates, with one
 * launch per kernel, the subset of instances named in it (each with its own
 * frame), so requests that arrive while other ticks are on the GPU start in
 * the next tick. Up to `inflight` ticks can be outstanding, each with its
 * own device region (so ticks on different streams overlap); an instance may
 * be in at most one outstanding tick, which keeps its frames in order, and
 * its result is exactly the one cbt_update would give. */
typedef struct cbt_server cbt_server;

/* Bytes of device workspace for a server over these states (0 if invalid);
 * 1 <= inflight <= 16. */
size_t cbt_server_workspace_bytes(cbt_state* const* states, int32_t n, int32_t inflight);

/* Builds a server; workspace is caller-owned device memory, 256-byte aligned,
 * kept until cbt_server_destroy. Errors: CBT_EINVAL, CBT_ENOMEM, CBT_ECUDA. */
int cbt_server_create(cbt_state* const* states, int32_t n, int32_t inflight, void* workspace,
                      size_t bytes, cbt_server** out);

/* Enqueues one tick on `stream`: instance idx[i] (an index into the server's
 * states) takes frames[i]. *ticket receives the tick's slot. CBT_EINVAL if an
 * instance is repeated or already in an outstanding tick, or if the next
 * slot's previous tick has not been polled yet. Asynchronous. */
int cbt_server_submit(cbt_server* sv, const int32_t* idx, const cbt_frame* frames, int32_t k,
                      cbt_stream_t stream, int32_t* ticket);

/* Completion of a tick: 1 when done (live_before[i], if given, receives the
 * live count of idx[i] at the start of its frame), 0 while pending (wait = 0),
 * a negative CBT_* code on error. wait != 0 blocks until done. */
int cbt_server_poll(cbt_server* sv, int32_t ticket, int wait, uint32_t* live_before);

/* 1 if the slot the next submit will use is free. */
int32_t cbt_server_next_slot_free(const cbt_server* sv);

/* Tick form. Not fused (the default): a tick is one launch per step, and a
 * tick submitted on another stream overlaps the running one on the device.
 * Fused: a tick is one cooperative launch of the whole frame (cbt_set_fused),
 * and each tick waits on the device for the previous one (two cooperative
 * launches are never in flight together); submission, admission and
 * polling still overlap the running tick. Switch only with no tick pending
 * (CBT_EINVAL otherwise). Results are identical either way. Host only. */
int cbt_server_set_fused(cbt_server* sv, int on);

/* Releases the server (waiting for outstanding ticks); workspaces stay the
 * caller's. */
void cbt_server_destroy(cbt_server* sv);

/* SumReduction (Sec. 3.1) alone over a caller's bitfield, as a streaming
 * kernel: the per-level uint32 sums above the bitfield words, in the layout
 * of cbt_cbt (sums[W + w] = popcount of word w, sums[n] = sums[2n] +
 * sums[2n+1], sums[1] = the number of set bits). This is the prior method's
 * bottleneck that the paper times at 2^27 slots (Sec. 4); the frame update
 * runs the same reduction inside its own launch.
 *   d_bitfield: DEVICE u32[2^D / 32], 16-byte aligned, read only;
 *   D: 5 <= D <= 28 (W = 2^(D-5) words);
 *   d_sums: DEVICE u32[2W], 16-byte aligned, caller-owned. Its unused word
 *           sums[0] counts the call's finished chunks: it must be 0 when the
 *           call starts (a zeroed buffer) and the call leaves it 0, so calls
 *           on one d_sums must not overlap on the GPU.
 * One launch on `stream` (chunks of 4096 words; the last chunk to finish
 * builds the levels above the chunk roots); allocates nothing. Errors:
 * CBT_EINVAL (NULL or misaligned pointer, D < 5), CBT_ECAPACITY (D > 28),
 * CBT_ECUDA. Asynchronous. */
int cbt_sum_reduce(const uint32_t* d_bitfield, int32_t D, uint32_t* d_sums, cbt_stream_t stream);

/* CachePointers (Alg. 7, OneToBitID for every index) alone over a caller's
 * bitfield: d_live[i] = the position of the i-th set bit (from 0), for every
 * i below the number of set bits; with cbt_sum_reduce, the prior method's
 * reduction plus compaction that the paper times at 2^27 slots (Sec. 4).
 *   d_bitfield: DEVICE u32[2^D / 32], read only;
 *   d_sums: DEVICE u32[2W], the sum tree of d_bitfield as cbt_sum_reduce
 *           wrote it (read only; its root sums[1] is the output count);
 *   D: 5 <= D <= 28;
 *   d_live: DEVICE u32[cap], caller-owned; positions at index >= cap are
 *           not written (read the count from sums[1]).
 * One launch on `stream`; allocates nothing. Errors: CBT_EINVAL (NULL or
 * misaligned pointer, D < 5), CBT_ECAPACITY (D > 28), CBT_ECUDA.
 * Asynchronous. */
int cbt_compact(const uint32_t* d_bitfield, const uint32_t* d_sums, int32_t D, uint32_t* d_live, uint32_t cap,
                cbt_stream_t stream);

/* The reduction and live-slot compaction step of cbt_update (the CBT sum
 * tree and the ascending list of set bits) over a caller's bitfield, for
 * callers that cannot allocate device memory: a real-time frame loop in which
 * cudaMalloc/cudaFree would synchronize the device and stall the frame, or a
 * host application whose device memory all comes from its own allocator or a
 * graphics interop pool. This entry point allocates nothing; its scratch (a
 * tile ticket, a finished-tile counter, an error word and the look-back
 * descriptors) is one static device array of 33,024 bytes in this library,
 * held by every GPU that loads the library until the process exits. The
 * paper has no counterpart to this entry point.
 *   d_bitfield: DEVICE u32[max(1, 2^D / 32)], bit s % 32 of word s / 32 is slot
 *               s (bits at or above 2^D are ignored);
 *   D: 1 <= D <= 27 (the static scratch covers 4096 tiles of 1024 words);
 *   d_sums: DEVICE u32[2 * words], written in the layout of cbt_cbt; its word
 *           d_sums[0], which that layout leaves unused, receives the call's
 *           device status: 0, or CBT_DERR_TIMEOUT when a bounded wait of the
 *           kernel's look-back gave up (the tiles' prefixes, and so the list,
 *           are then not to be trusted);
 *   d_live: DEVICE u32[2^D], receives the slots of the set bits, ascending;
 *   d_count: DEVICE u32, receives the number of set bits, or 0xFFFFFFFF when
 *           d_sums[0] reports a timeout.
 * Read d_sums[0] or d_count once the stream has reached the call.
 * The first call on a device looks up the scratch's device address (with
 * that device current); make that first call before any stream capture.
 * Every call clears the part of the scratch it uses before its kernel runs;
 * calls whose work overlaps on the GPU (other streams, other threads) share
 * the scratch and race. Errors: CBT_EINVAL (NULL pointer, D < 1),
 * CBT_ECAPACITY (D > 27), CBT_ECUDA. Asynchronous. */
int cbt_reduce_compact_static(const uint32_t* d_bitfield, int32_t D, uint32_t* d_sums,
                              uint32_t* d_live, uint32_t* d_count, cbt_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif
