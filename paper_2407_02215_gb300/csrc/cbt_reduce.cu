// SumReduction (Sec. 3.1) over a caller's bitfield, as a streaming kernel
// (and CachePointers over the same bitfield, further below):
// the per-level uint32 sums of the CBT above its bitfield words (the layout
// of cbt_cbt: sums[W + w] = popc(word w), sums[n] = sums[2n] + sums[2n+1],
// sums[1] = the number of set bits). One launch: each block reduces chunks
// of 4096 words (coalesced vector loads of the words; the levels in the
// thread, then across the warp by shuffles, then across the block's warps),
// and the last block to finish builds the levels above the chunk roots in
// shared memory.
// The unused word sums[0] counts the finished chunks and is left at 0.
#include <cstdint>

#include "cbt.h"
#include "cbt_device.cuh"

namespace {

constexpr int kRThreads = 256;
constexpr uint32_t kChunkWords = 4096;               // words per chunk: 8 warps of 512
constexpr uint32_t kMaxRoots = 2048;                 // chunk roots the last block reduces (D <= 28)

// Levels above the n nodes at s[n, 2n) of a shared heap-ordered array, each
// also stored to sums (block-wide).
__device__ __forceinline__ void top_levels(uint32_t* s, uint32_t n, uint32_t* sums) {
    for (uint32_t m = n >> 1; m >= 1u; m >>= 1) {
        for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) {
            const uint32_t p = m + k;
            const uint32_t v = s[2u * p] + s[2u * p + 1u];
            s[p] = v;
            sums[p] = v;
        }
        __syncthreads();
    }
}

// W >= kChunkWords. A warp covers 512 consecutive words (a level-9 node) as
// four rows of 128 words, each row one coalesced 512-byte load (lane x holds
// words 4x..4x+3 of the row): levels 1..2 stay in the thread, 3..7 across the
// lanes of a row (shuffles), 8..9 in lane 0 over the four rows, 10..12 across
// the 8 warps of the block.
__global__ void __launch_bounds__(kRThreads) k_sum_chunks(const uint32_t* __restrict__ bits, uint32_t W,
                                                          uint32_t* __restrict__ sums) {
    __shared__ uint32_t s_warp[kRThreads / 32];
    __shared__ uint32_t s_last;
    __shared__ uint32_t s_top[2 * kMaxRoots];
    const uint32_t nchunks = W / kChunkWords;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint32_t wbase = c * kChunkWords + (uint32_t)warp * 512u;  // the warp's first word
        uint4 a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = __ldcs(reinterpret_cast<const uint4*>(bits + wbase + 128u * r) + lane);
        uint32_t row[4];  // level 7 of each row, in lane 0
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t w = wbase + 128u * r + 4u * lane;  // this lane's first word
            const uint32_t p0 = __popc(a[r].x), p1 = __popc(a[r].y), p2 = __popc(a[r].z), p3 = __popc(a[r].w);
            __stcs(reinterpret_cast<uint4*>(sums + W + w), make_uint4(p0, p1, p2, p3));        // level 0
            const uint32_t q0 = p0 + p1, q1 = p2 + p3;
            __stcs(reinterpret_cast<uint2*>(sums + ((W + w) >> 1)), make_uint2(q0, q1));       // level 1
            uint32_t x = q0 + q1;
            uint32_t node = (W + w) >> 2;                                                      // level 2
            sums[node] = x;
#pragma unroll
            for (int k = 1; k <= 5; ++k) {  // levels 3..7
                x += __shfl_down_sync(0xFFFFFFFFu, x, 1 << (k - 1));
                node >>= 1;
                if ((lane & ((1 << k) - 1)) == 0) sums[node] = x;
            }
            row[r] = x;
        }
        uint32_t y = 0;
        if (lane == 0) {
            const uint32_t n8 = (W + wbase) >> 8;  // level 8: two nodes per warp
            sums[n8] = row[0] + row[1];
            sums[n8 + 1] = row[2] + row[3];
            y = row[0] + row[1] + row[2] + row[3];
            sums[n8 >> 1] = y;  // level 9
            s_warp[warp] = y;
        }
        __syncthreads();
        if (warp == 0) {  // levels 10..12
            uint32_t z = lane < kRThreads / 32 ? s_warp[lane] : 0u;
            uint32_t n = ((W + c * kChunkWords) >> 9) + (uint32_t)lane;
#pragma unroll
            for (int k = 1; k <= 3; ++k) {
                z += __shfl_down_sync(0xFFFFFFFFu, z, 1 << (k - 1));
                n >>= 1;
                if (lane < kRThreads / 32 && (lane & ((1 << k) - 1)) == 0) sums[n] = z;
            }
        }
        __syncthreads();
    }
    if (nchunks == 1u) return;  // the chunk root is the tree root
    // the last block to finish builds the levels above the chunk roots; the
    // roots it reads were all written by thread 0 of their blocks
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(sums, 1u) == gridDim.x - 1u ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (uint32_t k = threadIdx.x; k < nchunks; k += blockDim.x) s_top[nchunks + k] = __ldcg(sums + nchunks + k);
    __syncthreads();
    top_levels(s_top, nchunks, sums);
    if (threadIdx.x == 0) sums[0] = 0u;
}

// W < kChunkWords: the whole tree by one block.
__global__ void __launch_bounds__(1024) k_sum_small(const uint32_t* __restrict__ bits, uint32_t W,
                                                    uint32_t* __restrict__ sums) {
    __shared__ uint32_t s[2 * kChunkWords];
    for (uint32_t w = threadIdx.x; w < W; w += blockDim.x) {
        const uint32_t p = (uint32_t)__popc(bits[w]);
        s[W + w] = p;
        sums[W + w] = p;
    }
    __syncthreads();
    top_levels(s, W, sums);
}

// CachePointers (Alg. 7 for every index) over a caller's bitfield and the
// sum tree k_sum_chunks wrote for it: live[i] = the position of the i-th set
// bit. Every warp takes 128-word segments (level-7 nodes; small enough that
// the warps share them evenly) in turn, with no block-wide step: the
// segment's first output index is read off the tree (the left siblings along
// its node's path, one level per lane), its 4 rows of 32 words are loaded at
// once, and each row is compacted: every lane writes the
// positions of its word's set bits into the warp's staging row at its scan
// offset (two set bits per loop step), and the warp copies the row out with
// coalesced stores. Positions at
// index >= cap are dropped.
constexpr int kStage = 32 * 32;  // positions of 32 words, at most
constexpr uint32_t kSegLog = 7;
constexpr uint32_t kSegWords = 1u << kSegLog;
constexpr int kSegRows = (int)kSegWords / 32;
__global__ void __launch_bounds__(kRThreads) k_compact_segments(const uint32_t* __restrict__ bits,
                                                                const uint32_t* __restrict__ sums, uint32_t W,
                                                                uint32_t* __restrict__ live, uint32_t cap) {
    __shared__ uint32_t s_stage[kRThreads / 32][kStage];
    const uint32_t nseg = W / kSegWords;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* stage = s_stage[warp];
    const uint32_t nwarps = gridDim.x * (kRThreads / 32);
    for (uint32_t sg = blockIdx.x * (kRThreads / 32) + (uint32_t)warp; sg < nseg; sg += nwarps) {
        const uint32_t w0 = sg * kSegWords;
        uint32_t x[kSegRows];
#pragma unroll
        for (int r = 0; r < kSegRows; ++r) x[r] = __ldcs(bits + w0 + 32u * r + (uint32_t)lane);
        const uint32_t n = ((W + w0) >> kSegLog) >> lane;  // the segment's node, `lane` levels up
        uint32_t base = (n > 1u && (n & 1u)) ? __ldg(sums + n - 1u) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) base += __shfl_xor_sync(0xFFFFFFFFu, base, o);
#pragma unroll
        for (int r = 0; r < kSegRows; ++r) {
            const uint32_t w = w0 + 32u * r + (uint32_t)lane;
            uint32_t m = x[r];
            const uint32_t p = (uint32_t)__popc(m);
            uint32_t inc = p;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if (lane >= o) inc += y;
            }
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
            uint32_t k = inc - p;
            const uint32_t wb = w * 32u;
            while (m) {  // two set bits per step
                stage[k] = wb + (uint32_t)(__ffs(m) - 1);
                m &= m - 1u;
                if (m) {
                    stage[k + 1u] = wb + (uint32_t)(__ffs(m) - 1);
                    m &= m - 1u;
                }
                k += 2u;
            }
            __syncwarp();
            if (base + tot <= cap) {  // warp-uniform
                for (uint32_t q = (uint32_t)lane; q < tot; q += 32u) __stcs(live + base + q, stage[q]);
            } else {
                for (uint32_t q = (uint32_t)lane; q < tot; q += 32u)
                    if (base + q < cap) __stcs(live + base + q, stage[q]);
            }
            __syncwarp();
            base += tot;
        }
    }
}

// W < kSegWords: one warp walks the words 32 at a time.
__global__ void __launch_bounds__(32) k_compact_small(const uint32_t* __restrict__ bits, uint32_t W,
                                                      uint32_t* __restrict__ live, uint32_t cap) {
    __shared__ uint32_t stage[kStage];
    const int lane = threadIdx.x;
    uint32_t base = 0;
    for (uint32_t w0 = 0; w0 < W; w0 += 32u) {
        const uint32_t w = w0 + (uint32_t)lane;
        uint32_t x = w < W ? bits[w] : 0u;
        const uint32_t p = (uint32_t)__popc(x);
        uint32_t inc = p;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
        uint32_t k = inc - p;
        while (x) {
            stage[k++] = w * 32u + (uint32_t)(__ffs(x) - 1);
            x &= x - 1u;
        }
        __syncwarp();
        for (uint32_t q = (uint32_t)lane; q < tot; q += 32u)
            if (base + q < cap) live[base + q] = stage[q];
        __syncwarp();
        base += tot;
    }
}

}  // namespace

extern "C" int cbt_compact(const uint32_t* d_bitfield, const uint32_t* d_sums, int32_t D, uint32_t* d_live,
                           uint32_t cap, cbt_stream_t stream) {
    if (!d_bitfield || !d_sums || (!d_live && cap) || D < 5) return CBT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_bitfield) | reinterpret_cast<uintptr_t>(d_sums) |
         reinterpret_cast<uintptr_t>(d_live)) & 3u)
        return CBT_EINVAL;
    if (D > 28) return CBT_ECAPACITY;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t W = 1u << (D - 5);
    if (cap == 0) return CBT_OK;
    if (W < kSegWords) {
        k_compact_small<<<1, 32, 0, s>>>(d_bitfield, W, d_live, cap);
    } else {
        const uint32_t blocks = W / kSegWords / (kRThreads / 32);  // one segment per warp at most
        int dev = 0, sms = 1, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_compact_segments, kRThreads, 0);
        const uint32_t grid = static_cast<uint32_t>(sms) * static_cast<uint32_t>(per > 0 ? per : 1);
        const uint32_t g = blocks < 1u ? 1u : (blocks < grid ? blocks : grid);
        k_compact_segments<<<g, kRThreads, 0, s>>>(d_bitfield, d_sums, W, d_live, cap);
    }
    return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_sum_reduce(const uint32_t* d_bitfield, int32_t D, uint32_t* d_sums, cbt_stream_t stream) {
    if (!d_bitfield || !d_sums || D < 5) return CBT_EINVAL;
    if (D > 28) return CBT_ECAPACITY;  // at most kMaxRoots chunk roots for the last block
    if ((reinterpret_cast<uintptr_t>(d_bitfield) & 15u) || (reinterpret_cast<uintptr_t>(d_sums) & 15u))
        return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t W = 1u << (D - 5);
    if (W < kChunkWords) {
        k_sum_small<<<1, 1024, 0, s>>>(d_bitfield, W, d_sums);
    } else {
        const uint32_t nchunks = W / kChunkWords;
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint32_t cap = static_cast<uint32_t>(sms) * 8u;
        k_sum_chunks<<<nchunks < cap ? nchunks : cap, kRThreads, 0, s>>>(d_bitfield, W, d_sums);
    }
    return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA;
}
