// Kernels of one frame of the CBT bisection update (Sec. 3.3 pipeline),
// restructured for sm_103a: decoupled look-back scans in place of the
// paper's atomic allocation counter, gathers in place of its neighbour
// scatters, and the CBT reduction fused with the live-slot compaction.
#pragma once
#include "cbt_device.cuh"

namespace cbtgpu {

// Launch entry points (defined in cbt_kernels.cu).
void launch_prep(const Inst& I, const FrameP& fp, bool frame_start, int grid, cudaStream_t s);
void launch_classify(const Inst& I, const FrameP& fp, int grid, cudaStream_t s);
void launch_gate(const Inst& I, const FrameP& fp, int grid, cudaStream_t s);
void launch_scatter(const Inst& I, int grid, cudaStream_t s);
void launch_alloc(const Inst& I, int grid, cudaStream_t s);
void launch_free(const Inst& I, int grid, cudaStream_t s);
void launch_fill(const Inst& I, int grid, cudaStream_t s);
void launch_cbt(const Inst& I, int grid, cudaStream_t s);
void launch_init(const Inst& I, const int32_t* twin, const int32_t* next, const int32_t* prev,
                 const int32_t* face, const double* hpos, int grid, cudaStream_t s);
void launch_leaves(const Inst& I, uint32_t* slots, uint64_t* heap, uint32_t* links, int grid,
                   cudaStream_t s);
void launch_vertices(const Inst& I, const FrameP& fp, float* out, uint32_t cap, int grid, cudaStream_t s);

}  // namespace cbtgpu
