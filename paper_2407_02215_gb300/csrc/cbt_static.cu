// CBT reduction and live-slot compaction over a caller's bitfield, with its
// scratch in a static device array instead of caller- or library-allocated
// memory (cbt_reduce_compact_static in cbt.h).
//
// The scratch is g_cbt_static_scratch below: 32 counter words (a tile ticket
// and a finished-tile counter) followed by one look-back descriptor per tile
// of 1024 bitfield words, for at most 4096 tiles, i.e. pools of up to 2^27
// slots (33,024 bytes in all). Every device that loads the library holds one
// copy until the process exits.
//
// Host code may not use the array's name as a device address (on the host it
// names a stand-in object), so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; the first call should therefore come before any stream capture.
// Every call clears the counters and the descriptors it will use before its
// kernel runs; calls whose work overlaps on the GPU share the array and race.
// A look-back wait that runs out sets the sticky error word in the scratch;
// the last tile to finish copies it into the caller's sums[0] (a word the
// sum-tree layout leaves unused) and then writes 0xFFFFFFFF as the count.
#include <cstdint>
#include <mutex>

#include "cbt.h"
#include "cbt_device.cuh"

namespace {

using namespace cbtgpu;

constexpr int32_t kStaticMaxD = 27;
constexpr uint32_t kStaticTileWords = 1024;
constexpr uint32_t kStaticMaxTiles = (1u << (kStaticMaxD - 5)) / kStaticTileWords;
constexpr uint32_t kCounterSlots = 32;  // 256 bytes of counters ahead of the descriptors
constexpr int kStaticSpinLimit = 1 << 22;

__device__ __align__(256) unsigned long long g_cbt_static_scratch[kCounterSlots + kStaticMaxTiles];

__device__ __forceinline__ unsigned long long ld_volatile_status(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile_status(unsigned long long* p, unsigned long long v) {
    *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
unsigned long long* g_scratch_ptr[kMaxDevices] = {};

// Exclusive block scan of one u32 per thread (256 threads); total via `total`.
__device__ uint32_t static_block_scan(uint32_t x, uint32_t& total, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < kThreads / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        __syncwarp();
        if (lane < kThreads / 32) s_warp[lane] = wi - w;
        if (lane == kThreads / 32 - 1) s_warp[kThreads / 32] = wi;
    }
    __syncthreads();
    const uint32_t r = s_warp[warp] + inc - x;
    total = s_warp[kThreads / 32];
    __syncthreads();
    return r;
}

// Publishes the tile's count, looks back over earlier tiles (bounded waits),
// returns the tile's exclusive prefix to every thread.
__device__ uint32_t static_tile_prefix(unsigned long long* status, uint32_t tile, uint32_t agg,
                                       unsigned int* err, uint32_t* s_excl) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        uint32_t ex = 0;
        if (tile == 0) {
            if (lane == 0) st_volatile_status(status, (kFlagIncl << 62) | agg);
        } else {
            if (lane == 0) st_volatile_status(status + tile, (kFlagAgg << 62) | agg);
            int p = (int)tile - 1;
            while (p >= 0) {
                const int idx = p - lane;
                unsigned long long s = idx >= 0 ? ld_volatile_status(status + idx) : (kFlagIncl << 62);
                int iters = 0;
                bool timed_out = false;
                while (!__all_sync(0xFFFFFFFFu, (s >> 62) != 0ull)) {
                    if (++iters > kStaticSpinLimit) {
                        timed_out = true;
                        break;
                    }
                    __nanosleep(32);
                    if ((s >> 62) == 0ull && idx >= 0) s = ld_volatile_status(status + idx);
                }
                if (timed_out) {
                    if (lane == 0) atomicOr(err, kErrTimeout);
                    break;
                }
                const unsigned incl = __ballot_sync(0xFFFFFFFFu, (s >> 62) == kFlagIncl);
                const int first = incl ? __ffs(incl) - 1 : 31;
                uint32_t v = lane <= first ? (uint32_t)(s & 0xFFFFFFFFull) : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                ex += v;
                if (incl) break;
                p -= 32;
            }
            if (lane == 0) st_volatile_status(status + tile, (kFlagIncl << 62) | (ex + agg));
        }
        if (lane == 0) *s_excl = ex;
    }
    __syncthreads();
    const uint32_t r = *s_excl;
    __syncthreads();
    return r;
}

// One tile of kStaticTileWords words per block iteration: popcounts, the
// tile's part of the sum tree, the live slots of its set bits in order
// (each warp's 128 words as four rows of 32, a row's positions staged in
// shared memory and stored coalesced); the last tile to finish builds the
// levels above the tiles, the count and the error word.
__global__ void __launch_bounds__(kThreads)
k_reduce_compact_static(const uint32_t* bits, uint32_t W, uint32_t TW, uint32_t ntiles, uint32_t valid_bits,
                        uint32_t* sums, uint32_t* live, uint32_t* count, unsigned long long* scratch) {
    __shared__ uint32_t s_tile, s_last, s_excl;
    __shared__ uint32_t s_warp[kThreads / 32 + 1];
    __shared__ uint32_t s_lvl[2][kThreads];
    __shared__ uint32_t s_rows[kThreads / 32][1024];
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
    unsigned int* done = reinterpret_cast<unsigned int*>(scratch + 1);
    unsigned int* err = reinterpret_cast<unsigned int*>(scratch + 2);
    unsigned long long* status = scratch + kCounterSlots;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if (tile >= ntiles) break;
        const uint32_t w0 = tile * TW + threadIdx.x * 4u;
        const bool mine = threadIdx.x * 4u < TW;
        uint32_t pc[4] = {0, 0, 0, 0};
        if (mine)
            for (uint32_t k = 0; k < 4u && threadIdx.x * 4u + k < TW; ++k) {
                uint32_t m = bits[w0 + k];
                if (valid_bits < 32u) m &= (1u << valid_bits) - 1u;
                pc[k] = __popc(m);
            }
        if (mine) {
            for (uint32_t k = 0; k < 4u && threadIdx.x * 4u + k < TW; ++k) sums[W + w0 + k] = pc[k];
            if (TW >= 2u) {
                sums[(W + w0) >> 1] = pc[0] + pc[1];
                if (TW >= 4u) {
                    sums[((W + w0) >> 1) + 1] = pc[2] + pc[3];
                    sums[(W + w0) >> 2] = pc[0] + pc[1] + pc[2] + pc[3];
                }
            }
        }
        const uint32_t tsum = pc[0] + pc[1] + pc[2] + pc[3];
        uint32_t cnt = TW >= 4u ? TW / 4u : 1u;
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
                sums[((W + tile * TW) >> lvl) + threadIdx.x] = v;
            }
            cur ^= 1;
            __syncthreads();
        }
        uint32_t tot;
        const uint32_t tex = static_block_scan(tsum, tot, s_warp);
        const uint32_t ex = static_tile_prefix(status, tile, tot, err, &s_excl);
        // the warp's words [wb, wb + 128) in rows of 32, lane l on word wb +
        // 32 k + l; its first output index is its first lane's prefix
        const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
        uint32_t out = ex + __shfl_sync(0xFFFFFFFFu, tex, 0);
        const uint32_t wb = tile * TW + warp * 128u;
        uint32_t* row = s_rows[warp];
#pragma unroll 1
        for (uint32_t k = 0; k < 4u; ++k) {
            const uint32_t wl = warp * 128u + k * 32u + lane;  // word within the tile
            uint32_t m = wl < TW ? bits[wb + k * 32u + lane] : 0u;
            if (valid_bits < 32u) m &= (1u << valid_bits) - 1u;
            const uint32_t pc = __popc(m);
            uint32_t inc = pc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                if ((int)lane >= o) inc += y;
            }
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
            uint32_t o = inc - pc;
            while (m) {
                row[o++] = (wb + k * 32u + lane) * 32u + (uint32_t)(__ffs(m) - 1);
                m &= m - 1u;
            }
            __syncwarp();
            for (uint32_t q = lane; q < total; q += 32u) live[out + q] = row[q];
            __syncwarp();
            out += total;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(done, 1u) == ntiles - 1u) ? 1u : 0u;
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (uint32_t n = ntiles >> 1; n >= 1u; n >>= 1) {
                for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
                    sums[n + k] = __ldcg(sums + 2u * (n + k)) + __ldcg(sums + 2u * (n + k) + 1u);
                __threadfence();
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                // every tile's look-back ended before its finish was counted
                const unsigned int e = atomicOr(err, 0u);
                sums[0] = e;
                *count = e ? 0xFFFFFFFFu : __ldcg(sums + 1);
            }
        }
    }
}

// Address of the static scratch on the current device, looked up once per
// device (with that device current) and cached.
int static_scratch(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CBT_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cbt_static_scratch) != cudaSuccess || !p) return CBT_ECUDA;
        g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CBT_OK;
}

}  // namespace

extern "C" int cbt_reduce_compact_static(const uint32_t* d_bitfield, int32_t D, uint32_t* d_sums,
                                         uint32_t* d_live, uint32_t* d_count, cbt_stream_t stream) {
    if (!d_bitfield || !d_sums || !d_live || !d_count || D < 1) return CBT_EINVAL;
    if (D > kStaticMaxD) return CBT_ECAPACITY;
    const uint32_t cap = 1u << D;
    const uint32_t W = cap >= 32u ? cap / 32u : 1u;
    const uint32_t TW = W < kStaticTileWords ? W : kStaticTileWords;
    const uint32_t ntiles = W / TW;
    if (ntiles > kStaticMaxTiles) return CBT_ECAPACITY;
    unsigned long long* scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (kCounterSlots + ntiles), s) != cudaSuccess)
        return CBT_ECUDA;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t grid = ntiles < 2u * (uint32_t)sms ? ntiles : 2u * (uint32_t)sms;
    k_reduce_compact_static<<<grid, kThreads, 0, s>>>(d_bitfield, W, TW, ntiles, cap < 32u ? cap : 32u,
                                                      d_sums, d_live, d_count, scratch);
    return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA;
}
