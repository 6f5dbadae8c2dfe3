// Indexed export of the live bisectors (the paper exports the triangulation
// into a visibility buffer, Sec. 4; R15 reading): corners that are the same
// point of the subdivided surface share one vertex, numbered in order of
// first occurrence over (live index, corner).
//
// A corner's identity is its exact weight row (Eq. 1, over 2^d) in lowest
// terms, each nonzero weight paired with the global point of its root corner
// (mesh vertex, or V + face for a face centroid), pairs in ascending point
// order. Five launches over the 3N corners ("occurrences" o = 3 i + c):
//   insert: the identity and a 64-bit hash of it; an open-addressing table
//           (linear probing, claimed by compare-and-swap of the hash, no
//           waiting) gives each distinct hash a slot, whose smallest
//           occurrence becomes the vertex's representative;
//   mark:   every occurrence compares its identity with its representative's
//           (a 64-bit hash collision between two identities is reported,
//           not merged) and flags itself when it is the representative;
//           flags are counted per tile of 2048 occurrences;
//   tiles:  one block scans the tile counts;
//   ids:    representatives get their vertex index (tile base + scan);
//   write:  index buffer, vertex buffer (the representative's per-bisector
//           vertex), heap IDs.
#include <cstdint>

#include "cbt.h"
#include "cbt_kernels.cuh"
#include "cbt_phases.cuh"

namespace cbtgpu {

namespace {

constexpr int kIThreads = 256;
constexpr uint32_t kITile = 2048;  // occurrences per tile of the vertex numbering: kIThreads * 8

struct VKey {
    unsigned long long a, b, c, e;  // ids 0 | 1; id 2 | d << 32 | n << 40; weights 0 and 1 (2 follows)
};

struct IndexWs {
    unsigned long long* tag;  // [T] hash | 1 of the slot's identity, 0 = empty
    uint32_t* rep;            // [T] smallest occurrence of the slot
    VKey* okey;               // [3N] identity per occurrence
    uint32_t* oslot;          // [3N] table slot per occurrence
    uint32_t* vid;            // [3N] first-occurrence flag, then vertex index of representatives
    uint32_t* tile;           // [ntiles + 1] flags per tile, then exclusive prefix
    uint32_t* cnt;            // [4] 0: collision flag, 1: vertex count
    uint32_t T;               // table size, a power of two > 3N
};

__device__ __forceinline__ bool same_key(const VKey& x, const VKey& y) {
    return x.a == y.a && x.b == y.b && x.c == y.c && x.e == y.e;
}

// Identity of corner v of a bisector with weights W (rows = corners) at
// depth d, root corners' global points p[3].
template <typename T>
__device__ __forceinline__ VKey corner_identity(const T W[9], int v, int d, const uint32_t p[3]) {
    unsigned long long w[3] = {(unsigned long long)W[3 * v], (unsigned long long)W[3 * v + 1],
                               (unsigned long long)W[3 * v + 2]};
    // lowest terms: strip the common factors of two (at most d of them)
    const unsigned long long any = w[0] | w[1] | w[2];
    const int tz = min(d, any ? __ffsll((long long)any) - 1 : d);
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] >>= tz;
    const uint32_t dd = (uint32_t)(d - tz);
    uint32_t id[3] = {kNull, kNull, kNull};
    unsigned long long ww[3] = {0, 0, 0};
    uint32_t n = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!w[k]) continue;
        // insertion keeping the points ascending
        uint32_t q = n;
        while (q > 0 && id[q - 1] > p[k]) {
            id[q] = id[q - 1];
            ww[q] = ww[q - 1];
            --q;
        }
        id[q] = p[k];
        ww[q] = w[k];
        ++n;
    }
    VKey key;
    key.a = (unsigned long long)id[0] | ((unsigned long long)id[1] << 32);
    key.b = (unsigned long long)id[2] | ((unsigned long long)dd << 32) | ((unsigned long long)n << 40);
    key.c = ww[0];
    key.e = ww[1];
    return key;
}

__device__ __forceinline__ unsigned long long key_hash(const VKey& k) {
    return splitmix64(k.a ^ splitmix64(k.b ^ splitmix64(k.c ^ splitmix64(k.e))));
}

template <typename T>
__device__ __forceinline__ void insert_corners(const Inst& I, const uint32_t* corner, IndexWs ws, uint32_t i,
                                               uint64_t j, int d, uint32_t h, const uint32_t* tab) {
    T W[9], Wp[9];
    decode_weights<T>(j, d, W, Wp, tab);
    const uint32_t p[3] = {corner[3 * h], corner[3 * h + 1], corner[3 * h + 2]};
#pragma unroll 1
    for (int v = 0; v < 3; ++v) {
        const uint32_t o = 3u * i + (uint32_t)v;
        const VKey key = corner_identity<T>(W, v, d, p);
        const unsigned long long hs = key_hash(key), t = hs | 1ull;
        uint32_t sl = (uint32_t)(hs >> 32) & (ws.T - 1u);
        bool placed = false;
        for (uint32_t probe = 0; probe < ws.T; ++probe) {
            unsigned long long cur = ws.tag[sl];
            if (cur == 0ull) cur = atomicCAS(ws.tag + sl, 0ull, t);
            if (cur == 0ull || cur == t) {
                placed = true;
                break;
            }
            sl = (sl + 1u) & (ws.T - 1u);
        }
        if (!placed) {  // cannot happen while T > 3N; reported, never waited on
            atomicOr(ws.cnt, 2u);
            sl = 0;
        }
        ws.okey[o] = key;
        ws.oslot[o] = sl;
        atomicMin(ws.rep + sl, o);
    }
}

// The live count N is read on the device (the CBT root); a count above the
// capacity the workspace was carved for is reported and nothing is done.
__device__ __forceinline__ uint32_t live_n(const Inst& I, uint32_t cap) {
    const uint32_t n = __ldg(I.sums + 1);
    return n <= cap ? n : 0u;
}

__global__ void __launch_bounds__(kIThreads) k_index_insert(Inst I, const uint32_t* corner, IndexWs ws,
                                                            uint32_t cap) {
    __shared__ __align__(16) uint32_t s_tab[kDecTabWords];
    load_dec6(s_tab);
    __syncthreads();
    const uint32_t N = live_n(I, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ws.cnt[2] = __ldg(I.sums + 1);
        if (ws.cnt[2] > cap) atomicOr(ws.cnt, 8u);
    }
    for (uint32_t i = blockIdx.x * kIThreads + threadIdx.x; i < N; i += gridDim.x * kIThreads) {
        const uint64_t j = I.heap[I.live[i]];
        const int d = depth_of(j, I.ch);
        const uint32_t h = (uint32_t)((j >> d) - (1ull << I.ch));
        if (d < 0 || h >= I.H) {
            atomicOr(ws.cnt, 4u);
            continue;
        }
        if (d <= 31)
            insert_corners<uint32_t>(I, corner, ws, i, j, d, h, s_tab);
        else
            insert_corners<unsigned long long>(I, corner, ws, i, j, d, h, s_tab);
    }
}

__global__ void __launch_bounds__(kIThreads) k_index_mark(Inst I, IndexWs ws, uint32_t cap) {
    __shared__ uint32_t s_cnt;
    const uint32_t n3 = 3u * live_n(I, cap);
    for (uint32_t t = blockIdx.x; t * kITile < n3; t += gridDim.x) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        uint32_t mine = 0;
        for (uint32_t k = threadIdx.x; k < kITile; k += kIThreads) {
            const uint32_t o = t * kITile + k;
            if (o >= n3) break;
            const uint32_t r = ws.rep[ws.oslot[o]];
            if (r >= n3 || !same_key(ws.okey[o], ws.okey[r])) atomicOr(ws.cnt, 1u);
            const uint32_t f = r == o ? 1u : 0u;
            ws.vid[o] = f;
            mine += f;
        }
        for (int s = 16; s > 0; s >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, s);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
        __syncthreads();
        if (threadIdx.x == 0) ws.tile[t] = s_cnt;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_index_tiles(Inst I, IndexWs ws, uint32_t cap) {
    __shared__ Pair s_warp[1024 / 32 + 1];
    const uint32_t ntiles = (3u * live_n(I, cap) + kITile - 1u) / kITile;
    uint32_t run = 0;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += blockDim.x) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t v = t < ntiles ? ws.tile[t] : 0u;
        Pair tot;
        const Pair ex = block_scan(Pair{v, 0u}, tot, s_warp);
        if (t < ntiles) ws.tile[t] = run + ex.a;
        run += tot.a;
    }
    if (threadIdx.x == 0) {
        ws.tile[ntiles] = run;
        ws.cnt[1] = run;
    }
}

__global__ void __launch_bounds__(kIThreads) k_index_ids(Inst I, IndexWs ws, uint32_t cap) {
    __shared__ Pair s_warp[kIThreads / 32 + 1];
    const uint32_t n3 = 3u * live_n(I, cap);
    constexpr uint32_t kPer = kITile / kIThreads;
    for (uint32_t t = blockIdx.x; t * kITile < n3; t += gridDim.x) {
        // thread k holds occurrences t kITile + k kPer .. + kPer - 1
        const uint32_t o0 = t * kITile + threadIdx.x * kPer;
        uint32_t f[kPer], c = 0;
#pragma unroll
        for (uint32_t q = 0; q < kPer; ++q) {
            f[q] = o0 + q < n3 ? ws.vid[o0 + q] : 0u;
            c += f[q];
        }
        Pair tot;
        uint32_t run = ws.tile[t] + block_scan(Pair{c, 0u}, tot, s_warp).a;
#pragma unroll
        for (uint32_t q = 0; q < kPer; ++q)
            if (f[q]) ws.vid[o0 + q] = run++;
    }
}

__global__ void __launch_bounds__(kIThreads) k_index_write(Inst I, IndexWs ws, uint32_t cap, const float* tri,
                                                           float* verts, uint32_t vcap, uint32_t* idx,
                                                           uint64_t* ids) {
    const uint32_t N = live_n(I, cap);
    for (uint32_t i = blockIdx.x * kIThreads + threadIdx.x; i < N; i += gridDim.x * kIThreads) {
#pragma unroll
        for (uint32_t v = 0; v < 3; ++v) {
            const uint32_t o = 3u * i + v;
            const uint32_t r = ws.rep[ws.oslot[o]];
            const uint32_t x = r < 3u * N ? ws.vid[r] : 0u;
            idx[o] = x;
            if (r == o && verts && tri && x < vcap) {
#pragma unroll
                for (int c = 0; c < 3; ++c) verts[3ull * x + c] = tri[3ull * o + c];
            }
        }
        if (ids) ids[i] = I.heap[I.live[i]];
    }
}

uint32_t table_size(uint32_t n) {
    uint64_t t = 64;
    while (t <= 3ull * n) t <<= 1;
    return static_cast<uint32_t>(t);
}

size_t align256(size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); }

// Workspace carved for up to n live bisectors; returns the bytes used.
size_t carve(uint32_t n, char* base, IndexWs* ws) {
    const uint32_t T = table_size(n);
    const size_t n3 = 3ull * n, ntiles = (n3 + kITile - 1u) / kITile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return base ? base + o : nullptr;
    };
    IndexWs w{};
    w.tag = reinterpret_cast<unsigned long long*>(take(8ull * T));
    w.rep = reinterpret_cast<uint32_t*>(take(4ull * T));
    w.okey = reinterpret_cast<VKey*>(take(sizeof(VKey) * n3));
    w.oslot = reinterpret_cast<uint32_t*>(take(4ull * n3));
    w.vid = reinterpret_cast<uint32_t*>(take(4ull * n3));
    w.tile = reinterpret_cast<uint32_t*>(take(4ull * (ntiles + 1u)));
    w.cnt = reinterpret_cast<uint32_t*>(take(16u));
    w.T = T;
    if (ws) *ws = w;
    return off;
}

// Rows [0, n) of 36-byte vertex records into mapped host memory, n = the
// live count read on the device (capped at cap rows): 16-byte vector loads
// and stores over the grid (aligned pointers), the tail words by block 0;
// thread 0 of block 0 also stores the live count at h_count.
__global__ void __launch_bounds__(kIThreads) k_rows_to_host(const uint32_t* count, const float* src, float* dst,
                                                            uint32_t cap, uint32_t* h_count, bool vec) {
    const uint32_t total = __ldg(count), n = min(total, cap);
    const size_t words = 9ull * n;
    const size_t q = vec ? words / 4u : 0u;
    const size_t stride = (size_t)gridDim.x * kIThreads;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (size_t k = (size_t)blockIdx.x * kIThreads + threadIdx.x; k < q; k += stride) d4[k] = __ldcs(s4 + k);
    if (blockIdx.x == 0) {
        for (size_t k = 4u * q + threadIdx.x; k < words; k += kIThreads) dst[k] = src[k];
        if (threadIdx.x == 0) *h_count = total;
    }
}

}  // namespace

int launch_rows_to_host(const uint32_t* count, const float* src, float* dst, uint32_t cap, uint32_t* h_count,
                        int sms, cudaStream_t s) {
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0u;
    k_rows_to_host<<<static_cast<unsigned>(sms) * 4u, kIThreads, 0, s>>>(count, src, dst, cap, h_count, vec);
    return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

size_t index_workspace_bytes(uint32_t n) { return carve(n, nullptr, nullptr); }

int launch_index(const Inst& I, const uint32_t* corner, uint32_t cap, void* workspace, size_t bytes,
                 const float* tri, float* verts, uint32_t vcap, uint32_t* idx, uint64_t* ids, int sms,
                 cudaStream_t s, uint32_t* h_nvert, uint32_t* h_ntri) {
    IndexWs ws;
    if (carve(cap, static_cast<char*>(workspace), &ws) > bytes) return CBT_ENOMEM;
    const uint32_t n3 = 3u * cap, ntiles = (n3 + kITile - 1u) / kITile;
    if (cudaMemsetAsync(ws.tag, 0, 8ull * ws.T, s) != cudaSuccess ||
        cudaMemsetAsync(ws.rep, 0xFF, 4ull * ws.T, s) != cudaSuccess ||
        cudaMemsetAsync(ws.cnt, 0, 16u, s) != cudaSuccess)
        return CBT_ECUDA;
    const uint32_t most = static_cast<uint32_t>(sms) * 8u;
    auto grid = [&](uint32_t work) { return work == 0 ? 1u : (work < most ? work : most); };
    // sized for the capacity; every kernel reads the live count on the device
    k_index_insert<<<grid((cap + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(I, corner, ws, cap);
    k_index_mark<<<grid(ntiles), kIThreads, 0, s>>>(I, ws, cap);
    k_index_tiles<<<1, 1024, 0, s>>>(I, ws, cap);
    k_index_ids<<<grid(ntiles), kIThreads, 0, s>>>(I, ws, cap);
    k_index_write<<<grid((cap + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(I, ws, cap, tri, verts, vcap,
                                                                                 idx, ids);
    if (cudaGetLastError() != cudaSuccess) return CBT_ECUDA;
    uint32_t cnt[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(cnt, ws.cnt, 16u, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CBT_ECUDA;
    if (h_nvert) *h_nvert = cnt[1];
    if (h_ntri) *h_ntri = cnt[2];
    if (cnt[0] & 8u) return CBT_ENOMEM;  // more live bisectors than the capacity
    if (cnt[0]) return CBT_EDEVICE;
    if (cnt[1] > vcap && verts) return CBT_ENOMEM;
    return CBT_OK;
}

}  // namespace cbtgpu
