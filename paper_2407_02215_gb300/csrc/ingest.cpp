// Host-side halfedge ingest and validation (Sec. 2.1, halfedge figure).
#include <cstdint>
#include <unordered_map>
#include <vector>

#include "cbt.h"

extern "C" int cbt_halfedges_from_faces(int32_t F, const int32_t* face_sizes,
                                        const int32_t* face_verts, int32_t H, int32_t* twin,
                                        int32_t* next, int32_t* prev, int32_t* vert,
                                        int32_t* face) {
    if (F < 1 || H < 3 || !face_sizes || !face_verts || !twin || !next || !prev || !vert || !face)
        return CBT_EINVAL;
    int64_t total = 0;
    for (int32_t f = 0; f < F; ++f) {
        if (face_sizes[f] < 3) return CBT_EINVAL;
        total += face_sizes[f];
    }
    if (total != H) return CBT_EINVAL;
    // Halfedges of face f are consecutive, in the face's vertex order.
    int32_t h0 = 0;
    for (int32_t f = 0; f < F; ++f) {
        const int32_t n = face_sizes[f];
        for (int32_t i = 0; i < n; ++i) {
            vert[h0 + i] = face_verts[h0 + i];
            next[h0 + i] = h0 + (i + 1 == n ? 0 : i + 1);
            prev[h0 + i] = h0 + (i == 0 ? n - 1 : i - 1);
            face[h0 + i] = f;
        }
        h0 += n;
    }
    // Twin: the halfedge running from Vert(Next h) to Vert(h).
    auto key = [](int32_t a, int32_t b) {
        return (static_cast<uint64_t>(static_cast<uint32_t>(a)) << 32) | static_cast<uint32_t>(b);
    };
    std::unordered_map<uint64_t, int32_t> directed;
    directed.reserve(static_cast<size_t>(H) * 2);
    for (int32_t h = 0; h < H; ++h) {
        if (!directed.emplace(key(vert[h], vert[next[h]]), h).second) return CBT_EINVAL;
    }
    for (int32_t h = 0; h < H; ++h) {
        const auto it = directed.find(key(vert[next[h]], vert[h]));
        twin[h] = it == directed.end() ? -1 : it->second;
    }
    return CBT_OK;
}

namespace cbtgpu {

// Checks the halfedge operators' invariants: Next/Prev inverse and within a
// face, Twin an involution without fixed points running the other way.
int validate_halfedges(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                       const int32_t* vert, const int32_t* face, int32_t V) {
    if (H < 3 || V < 1 || !twin || !next || !prev || !vert || !face) return CBT_EINVAL;
    for (int32_t h = 0; h < H; ++h) {
        const int32_t n = next[h], p = prev[h], t = twin[h];
        if (n < 0 || n >= H || p < 0 || p >= H) return CBT_EINVAL;
        if (prev[n] != h || next[p] != h) return CBT_EINVAL;
        if (face[h] < 0 || face[h] >= H || face[n] != face[h]) return CBT_EINVAL;
        if (vert[h] < 0 || vert[h] >= V) return CBT_EINVAL;
        if (t != -1) {
            if (t < 0 || t >= H || t == h || twin[t] != h) return CBT_EINVAL;
            if (vert[t] != vert[n] || vert[next[t]] != vert[h]) return CBT_EINVAL;
        }
    }
    // Every face cycle must close within H steps.
    std::vector<uint8_t> seen(static_cast<size_t>(H), 0);
    for (int32_t h = 0; h < H; ++h) {
        if (seen[h]) continue;
        int32_t x = h, steps = 0;
        do {
            seen[x] = 1;
            x = next[x];
            if (++steps > H) return CBT_EINVAL;
        } while (x != h);
        if (steps < 3) return CBT_EINVAL;
    }
    return CBT_OK;
}

}  // namespace cbtgpu
