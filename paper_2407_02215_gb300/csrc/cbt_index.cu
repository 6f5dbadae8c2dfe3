// Indexed export of the live bisectors (the paper exports the triangulation
// into a visibility buffer, Sec. 4; R15 reading): corners that are the same
// point of the subdivided surface share one vertex, numbered in order of
// first occurrence over (live index, corner), the "occurrences" o = 3 i + c.
//
// A corner's identity is its exact weight row (Eq. 1, over 2^d) in lowest
// terms over the global points of its root's corners. The points are of two
// kinds, and each is matched without forming the row:
//   root points: a row with one nonzero weight is a mesh vertex or a face
//     centroid, a global point p. Which corners these are follows from the
//     path bits: Eq. 1 makes a child's corners 0 and 1 its parent's corners
//     (0, 2) after a 0 bit and (2, 1) after a 1 bit, and its corner 2 new.
//     Corners at one global point are matched by p (the smallest occurrence
//     per point by atomicMin), whatever the mesh's connectivity there.
//   the others lie inside a root edge or a root triangle, where the surface
//     is a manifold. The bisection keeps the triangulation conforming (Sec.
//     2.3: an edge is shared whole by at most two bisectors), so the
//     bisectors having such a point as a corner form one fan, walked through
//     the neighbour links (fan_min). The fan's smallest (slot, corner) is
//     its first occurrence, the live list ascending by slot.
// Five launches: init (clears the counts, marks every root point unseen),
// roots (slot -> live index, root points' atomicMin), fans (every
// occurrence's representative; representatives flagged and counted per tile
// of 2048 occurrences; the last block to finish scans the tile counts), ids
// (representatives get their vertex index), write (index buffer, vertex
// buffer from the representative's per-bisector vertex, heap IDs; the
// counts into page-locked host memory).
#include <cstdint>

#include "cbt.h"
#include "cbt_kernels.cuh"
#include "cbt_phases.cuh"

namespace cbtgpu {

namespace {

constexpr int kIThreads = 256;
constexpr uint32_t kITile = 2048;  // occurrences per tile of the vertex numbering: kIThreads * 8
constexpr uint32_t kRootTag = 1u << 31;
constexpr int kFanGuard = 64;  // bisectors around one point, at most (a longer walk is a link error)

// Device error bits of the export (cnt[0]).
constexpr uint32_t kIxLink = 1u, kIxHeap = 4u, kIxCap = 8u;

struct IndexWs {
    uint32_t* cnt;        // [4] 0: error bits, 1: vertex count, 2: live count, 3: fans blocks done
    uint32_t* tile;       // [ntiles + 1] representatives per tile, then exclusive prefix (follows cnt)
    uint32_t* slot_live;  // [pool] live index of each live slot
    uint32_t* rootrep;    // [npts] smallest occurrence at each root point
    uint32_t* orep;       // [3N] kRootTag | p at a root point, else 0; then the representative occurrence
    uint32_t* vid;        // [3N] representative flag, then the vertex index of representatives
    uint32_t npts;
};

// Root corner (0, 1, 2) that corner v of bisector j at depth d >= 0 is, or
// -1 when the corner lies inside a root edge or triangle. The bit of depth k
// is bit d - k of j.
__device__ __forceinline__ int root_corner(uint64_t j, int d, int v) {
    if (d == 0) return v;
    if (v == 2) return -1;
    const uint64_t low = (1ull << (d - 1)) - 1ull;  // the bits of depths 2 .. d
    const uint64_t b = j & low;
    const bool first = ((j >> (d - 1)) & 1ull) != 0ull;  // the bit of depth 1
    if (v == 0) return b == 0ull ? (first ? 2 : 0) : -1;
    return b == low ? (first ? 1 : 2) : -1;
}

// The live count N is read on the device (the CBT root); a count above the
// capacity the workspace was carved for is reported and nothing is done.
__device__ __forceinline__ uint32_t live_n(const Inst& I, uint32_t cap) {
    const uint32_t n = __ldg(I.sums + 1);
    return n <= cap ? n : 0u;
}

// Counts and tile counts cleared, every root point's smallest occurrence
// set to none.
__global__ void __launch_bounds__(kIThreads) k_index_init(IndexWs ws, uint32_t words) {
    for (uint32_t k = blockIdx.x * kIThreads + threadIdx.x; k < words || k < ws.npts; k += gridDim.x * kIThreads) {
        if (k < words) ws.cnt[k] = 0u;
        if (k < ws.npts) ws.rootrep[k] = kNull;
    }
}

__global__ void __launch_bounds__(kIThreads) k_index_roots(Inst I, const uint32_t* corner, IndexWs ws,
                                                           uint32_t cap) {
    const uint32_t N = live_n(I, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ws.cnt[2] = __ldg(I.sums + 1);
        if (ws.cnt[2] > cap) atomicOr(ws.cnt, kIxCap);
    }
    for (uint32_t i = blockIdx.x * kIThreads + threadIdx.x; i < N; i += gridDim.x * kIThreads) {
        const uint32_t s = I.live[i];
        uint32_t pre[3] = {0u, 0u, 0u};
        if (s < I.cap) {
            ws.slot_live[s] = i;
            const uint64_t j = I.heap[s];
            const int d = depth_of(j, I.ch);
            const uint32_t h = d >= 0 ? (uint32_t)((j >> d) - (1ull << I.ch)) : I.H;
            if (h < I.H) {
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const int rc = root_corner(j, d, v);
                    if (rc < 0) continue;
                    const uint32_t p = __ldg(corner + 3u * h + (uint32_t)rc);
                    if (p >= ws.npts) {
                        atomicOr(ws.cnt, kIxHeap);
                        continue;
                    }
                    atomicMin(ws.rootrep + p, 3u * i + (uint32_t)v);
                    pre[v] = kRootTag | p;
                }
            } else {
                atomicOr(ws.cnt, kIxHeap);
            }
        } else {
            atomicOr(ws.cnt, kIxHeap);
        }
#pragma unroll
        for (int v = 0; v < 3; ++v) ws.orep[3u * i + v] = pre[v];
    }
}

// Smallest (slot << 2 | corner) of the fan around corner c0 of slot s0 (a
// point inside a root edge or triangle). A step leaves bisector s across
// edge x, one of its two edges at the point (corner q), and lands on edge e
// of the neighbour u (the reverse-link tag). Eq. 1 turns the vertex order
// over at every split (the children of (v0, v1, v2) are (v0, v2, m) and
// (v2, v1, m)), so the shared edge runs backwards in u's vertex order when
// the two depths have the same parity and forwards otherwise. The edge kinds
// give the parity: in the conforming bisection a refinement edge (Twin, edge
// 0) at depth d is shared with a refinement edge at depth d or with a Next
// or Prev edge at depth d - 1 (the children's refinement edges are their
// parent's other two edges), so the depths' parities agree exactly when x
// and e are both refinement edges or both not. That says which end of e is
// the point, and the walk goes on across u's other edge there: first across
// the edge leaving the point (x = c0) until it closes on the start, and at a
// border once more across the edge into it (x = c0 - 1). A link without its
// way back, a fan that does not close on its start or one longer than
// kFanGuard sets kIxLink.
__device__ uint32_t fan_min(const Inst& I, uint32_t* err, uint32_t s0, uint32_t c0) {
    const uint4 r0 = I.nb[s0];
    uint32_t best = (s0 << 2) | c0;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        uint4 rx = r0;
        uint32_t q = c0, x = pass == 0 ? c0 : (c0 == 0u ? 2u : c0 - 1u);
        int k = 0;
        for (; k < kFanGuard; ++k) {
            const uint32_t u = link_of(rx, (int)x);
            if (u == kNull) break;
            const uint32_t e = (rx.w >> (2u * x)) & 3u;
            if (u >= I.cap || e > 2u) {
                atomicOr(err, kIxLink);
                return best;
            }
            rx = I.nb[u];
            const bool same = (x == 0u) == (e == 0u);
            const bool from_start = q == x;  // the point is where edge x starts
            q = (from_start != same) ? e : (e == 2u ? 0u : e + 1u);
            x = e == q ? (q == 0u ? 2u : q - 1u) : q;
            if (u == s0) {
                if (pass == 1 || q != c0) atomicOr(err, kIxLink);
                return best;
            }
            best = min(best, (u << 2) | q);
        }
        if (k == kFanGuard) {
            atomicOr(err, kIxLink);
            return best;
        }
    }
    return best;
}

// One thread per occurrence: its representative (the root point's smallest
// occurrence, or the fan's first); representatives flagged and counted per
// tile.
__global__ void __launch_bounds__(kIThreads) k_index_fans(Inst I, IndexWs ws, uint32_t cap) {
    const uint32_t N = live_n(I, cap), n3 = 3u * N;
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = blockIdx.x * kIThreads; base < n3; base += gridDim.x * kIThreads) {
        const uint32_t o = base + threadIdx.x;
        bool rep = false;
        if (o < n3) {
            const uint32_t pre = ws.orep[o];
            uint32_t r;
            if (pre & kRootTag) {
                r = ws.rootrep[pre & ~kRootTag];
            } else {
                const uint32_t i = o / 3u, c = o - 3u * i;
                const uint32_t s = I.live[i];
                const uint32_t b = s < I.cap ? fan_min(I, ws.cnt, s, c) : kNull;
                const uint32_t li = (b >> 2) < I.cap ? ws.slot_live[b >> 2] : kNull;
                r = li < N ? 3u * li + (b & 3u) : kNull;
            }
            if (r >= n3) {
                atomicOr(ws.cnt, kIxLink);
                r = o;
            }
            ws.orep[o] = r;
            rep = r == o;
            ws.vid[o] = rep ? 1u : 0u;
        }
        // a warp's 32 occurrences lie in one tile (kITile is a multiple of 32)
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, rep);
        if (lane == 0u && m) atomicAdd(ws.tile + (base + (threadIdx.x & ~31u)) / kITile, __popc(m));
    }
    // The last block to finish turns the tile counts into exclusive prefixes
    // (the other blocks' counts are visible to it: each block fences before
    // it counts itself done).
    __shared__ bool s_last;
    __shared__ Pair s_warp[kIThreads / 32 + 1];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ws.cnt + 3, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t ntiles = (n3 + kITile - 1u) / kITile;
    uint32_t run = 0;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += kIThreads) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t v = t < ntiles ? __ldcg(ws.tile + t) : 0u;
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

// One thread per occurrence (coalesced orep and index words); the first N
// threads also write the heap IDs.
__global__ void __launch_bounds__(kIThreads) k_index_write(Inst I, IndexWs ws, uint32_t cap, const float* tri,
                                                           float* verts, uint32_t vcap, uint32_t* idx,
                                                           uint64_t* ids, uint32_t* h_cnt) {
    const uint32_t N = live_n(I, cap), n3 = 3u * N;
    // the earlier launches have set every count
    if (blockIdx.x == 0 && threadIdx.x < 3u)
        reinterpret_cast<volatile uint32_t*>(h_cnt)[threadIdx.x] = ws.cnt[threadIdx.x];
    for (uint32_t o = blockIdx.x * kIThreads + threadIdx.x; o < n3; o += gridDim.x * kIThreads) {
        const uint32_t r = ws.orep[o];
        const uint32_t x = r < n3 ? ws.vid[r] : 0u;
        idx[o] = x;
        if (r == o && verts && tri && x < vcap) {
#pragma unroll
            for (int c = 0; c < 3; ++c) verts[3ull * x + c] = tri[3ull * o + c];
        }
        if (ids && o < N) ids[o] = I.heap[I.live[o]];
    }
}

size_t align256(size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); }

// Workspace carved for up to n live bisectors of a pool of `pool` slots over
// npts global points; returns the bytes used.
size_t carve(uint32_t n, uint32_t pool, uint32_t npts, char* base, IndexWs* ws) {
    const size_t n3 = 3ull * n, ntiles = (n3 + kITile - 1u) / kITile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return base ? base + o : nullptr;
    };
    IndexWs w{};
    w.cnt = reinterpret_cast<uint32_t*>(take(16u + 4ull * (ntiles + 1u)));
    w.tile = w.cnt ? w.cnt + 4 : nullptr;
    w.slot_live = reinterpret_cast<uint32_t*>(take(4ull * pool));
    w.rootrep = reinterpret_cast<uint32_t*>(take(4ull * npts));
    w.orep = reinterpret_cast<uint32_t*>(take(4ull * n3));
    w.vid = reinterpret_cast<uint32_t*>(take(4ull * n3));
    w.npts = npts;
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

size_t index_workspace_bytes(uint32_t max_live, uint32_t pool, uint32_t npts) {
    return carve(max_live, pool, npts, nullptr, nullptr);
}

int launch_index(const Inst& I, const uint32_t* corner, uint32_t npts, uint32_t cap, void* workspace, size_t bytes,
                 const float* tri, float* verts, uint32_t vcap, uint32_t* idx, uint64_t* ids, int sms,
                 cudaStream_t s, uint32_t* h_cnt, uint32_t* h_nvert, uint32_t* h_ntri) {
    if (npts >= kRootTag) return CBT_EINVAL;  // the root-point tag takes the top bit
    IndexWs ws;
    if (carve(cap, I.cap, npts, static_cast<char*>(workspace), &ws) > bytes) return CBT_ENOMEM;
    uint32_t* d_cnt = nullptr;
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_cnt), h_cnt, 0) != cudaSuccess) return CBT_ECUDA;
    const uint32_t n3 = 3u * cap, ntiles = (n3 + kITile - 1u) / kITile;
    const uint32_t words = 4u + ntiles + 1u;
    const uint32_t most = static_cast<uint32_t>(sms) * 8u;
    auto grid = [&](uint32_t work) { return work == 0 ? 1u : (work < most ? work : most); };
    // sized for the capacity; every kernel reads the live count on the device
    k_index_init<<<grid(((words > npts ? words : npts) + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(ws, words);
    k_index_roots<<<grid((cap + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(I, corner, ws, cap);
    k_index_fans<<<grid((n3 + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(I, ws, cap);
    k_index_ids<<<grid(ntiles), kIThreads, 0, s>>>(I, ws, cap);
    k_index_write<<<grid((n3 + kIThreads - 1u) / kIThreads), kIThreads, 0, s>>>(I, ws, cap, tri, verts, vcap,
                                                                                idx, ids, d_cnt);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CBT_ECUDA;
    uint32_t cnt[3];
    for (int k = 0; k < 3; ++k) cnt[k] = reinterpret_cast<volatile uint32_t*>(h_cnt)[k];
    if (h_nvert) *h_nvert = cnt[1];
    if (h_ntri) *h_ntri = cnt[2];
    if (cnt[0] & kIxCap) return CBT_ENOMEM;  // more live bisectors than the capacity
    if (cnt[0]) return CBT_EDEVICE;
    if (cnt[1] > vcap && verts) return CBT_ENOMEM;
    return CBT_OK;
}

}  // namespace cbtgpu
