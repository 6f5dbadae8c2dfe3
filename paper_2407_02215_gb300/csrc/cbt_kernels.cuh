// Kernels of one frame of the CBT bisection update (Sec. 3.3 pipeline),
// restructured for sm_103a: decoupled look-back scans in place of the
// paper's atomic allocation counter, gathers in place of its neighbour
// scatters, and the CBT reduction fused with the live-slot compaction. Each
// kernel is launched once for a batch of instances.
#pragma once
#include "cbt_device.cuh"

namespace cbtgpu {

// Launch entry points (defined in cbt_kernels.cu).
void launch_prep(const BatchDev& bt, bool frame_start, int grid, cudaStream_t s);
void launch_classify(const BatchDev& bt, int grid, cudaStream_t s);
void launch_walk(const BatchDev& bt, int grid, cudaStream_t s);
void launch_gate(const BatchDev& bt, int grid, cudaStream_t s);
void launch_scatter(const BatchDev& bt, int grid, cudaStream_t s);
void launch_alloc(const BatchDev& bt, int grid, cudaStream_t s);
void launch_free(const BatchDev& bt, int grid, cudaStream_t s);
void launch_fill(const BatchDev& bt, int grid, cudaStream_t s);
void launch_cbt(const BatchDev& bt, int grid, cudaStream_t s);
void launch_vertices(const BatchDev& bt, int grid, cudaStream_t s);
// Vertex rows into mapped host memory (cbt_index.cu).
int launch_rows_to_host(const uint32_t* count, const float* src, float* dst, uint32_t cap, uint32_t* h_count,
                        int sms, cudaStream_t s);
// Indexed export (cbt_index.cu).
size_t index_workspace_bytes(uint32_t max_live, uint32_t pool, uint32_t npts);
int launch_index(const Inst& I, const uint32_t* corner, uint32_t npts, uint32_t cap, void* workspace, size_t bytes,
                 const float* tri, float* verts, uint32_t vcap, uint32_t* idx, uint64_t* ids, int sms,
                 cudaStream_t s, uint32_t* h_cnt, uint32_t* h_nvert, uint32_t* h_ntri);
// The one-launch frame (cbt_fused.cu): blocks of it resident per SM, and its
// cooperative launch over `grid` blocks.
int frame_blocks_per_sm();
cudaError_t launch_frame(const BatchDev& bt, int grid, cudaStream_t s);
// The single-instance frame in fewer phases (cbt_fused.cu); tbits = log2 of
// the slots under one word tile's sum-tree node, min(2^D, 32 tile words).
// It holds its scan-tile and word-tile tables in shared memory, so it takes
// pools of at most kFrame1MaxCap slots with 64-word tiles.
constexpr uint32_t kFrame1MaxCap = 1u << 22;
constexpr uint32_t kFrame1TileWords = 64;
constexpr int kFrame1Phases = 8;
int frame1_blocks_per_sm();
cudaError_t launch_frame1(const BatchDev& bt, int grid, uint32_t tbits, cudaStream_t s);
cudaError_t launch_wait_selftest(BatchGlobals* bg, int blocks, int limit, cudaStream_t s);
void launch_init(const Inst& I, const int32_t* twin, const int32_t* next, const int32_t* prev,
                 const double* hpos, int grid, cudaStream_t s);
void launch_leaves(const Inst& I, uint32_t* slots, uint64_t* heap, uint32_t* links, int grid,
                   cudaStream_t s);

}  // namespace cbtgpu
