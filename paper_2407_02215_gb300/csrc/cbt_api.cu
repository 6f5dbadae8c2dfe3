// C ABI of the CBT bisection library (declared in include/cbt.h).
#include <algorithm>
#include <cstring>
#include <vector>

#include "cbt.h"
#include "cbt_kernels.cuh"

namespace cbtgpu {
int validate_halfedges(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                       const int32_t* vert, const int32_t* face, int32_t V);
}

using namespace cbtgpu;

constexpr int kMaxKernels = 10;
const char* const kKernelNames[kMaxKernels] = {"prep", "classify", "gate", "scatter", "alloc",
                                                "free", "fill", "cbt", "vertices", ""};

struct cbt_state {
    Inst inst;
    void* workspace;
    size_t bytes;
    int sms;
    uint32_t frame;
    uint32_t launches;
    bool timing;
    uint32_t timed;  // kernels timed in the last frame
    cudaEvent_t ev[kMaxKernels + 1];
};

namespace {

struct Layout {
    size_t globals, heap, nb, cd, bits, sums, live, freel, scan, status, root64, rel, total;
    uint32_t cap, W, ntiles_items, ntiles_words, tile_words, ch;
};

uint32_t ceil_log2(uint32_t x) {
    uint32_t c = 0;
    while ((1ull << c) < static_cast<uint64_t>(x)) ++c;
    return c;
}

bool make_layout(int32_t H, int32_t D, Layout& L) {
    if (H < 3 || D < 1 || D > 30) return false;
    L.ch = ceil_log2(static_cast<uint32_t>(H));
    if (static_cast<uint32_t>(D) < L.ch) return false;
    L.cap = 1u << D;
    L.W = std::max(1u, L.cap / 32u);
    L.tile_words = std::min(L.W, kTileWords);
    L.ntiles_words = L.W / L.tile_words;
    L.ntiles_items = (L.cap + kTileItems - 1u) / kTileItems;
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off = (off + n + 255u) & ~static_cast<size_t>(255u);
        return o;
    };
    const size_t cap = L.cap, h = static_cast<size_t>(H);
    L.globals = take(sizeof(Globals));
    L.heap = take(8u * cap);
    L.nb = take(16u * cap);
    L.cd = take(8u * cap);
    L.bits = take(4u * L.W);
    L.sums = take(8u * L.W);
    L.live = take(4u * cap);
    L.freel = take(4u * cap);
    L.scan = take(4u * cap);
    L.status = take(8u * (3u * static_cast<size_t>(L.ntiles_items) + L.ntiles_words));
    L.root64 = take(72u * h);
    L.rel = take(72u * h);
    L.total = off;
    return true;
}

int grid_items(const cbt_state* st) {
    const uint32_t want = (st->inst.cap + kThreads - 1u) / kThreads;
    return static_cast<int>(std::max(1u, std::min<uint32_t>(want, static_cast<uint32_t>(st->sms) * 8u)));
}
int grid_tiles(const cbt_state* st) {
    return static_cast<int>(std::max(1u, std::min<uint32_t>(st->inst.ntiles_items, static_cast<uint32_t>(st->sms) * 2u)));
}
int grid_words(const cbt_state* st) {
    return static_cast<int>(std::max(1u, std::min<uint32_t>(st->inst.ntiles_words, static_cast<uint32_t>(st->sms) * 2u)));
}
int grid_prep(const cbt_state* st, bool frame_start) {
    uint32_t n = 9u * st->inst.H;
    if (frame_start) n = std::max(n, 3u * st->inst.ntiles_items + st->inst.ntiles_words);
    const uint32_t want = (n + kThreads - 1u) / kThreads;
    return static_cast<int>(std::max(1u, std::min<uint32_t>(want, static_cast<uint32_t>(st->sms) * 4u)));
}

int check_launch() { return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA; }

bool frame_from_api(const cbt_frame* f, uint32_t frame, FrameP& fp) {
    if (!f || f->precision > 2u || f->mode > 4u || f->nplanes > 5u || f->gate > 1u) return false;
    if (f->fixed_shift < 0 || f->fixed_shift > 62) return false;
    if (f->mode == CBT_MODE_LIST && ((f->n_split && !f->split_list) || (f->n_merge && !f->merge_list)))
        return false;
    std::memset(&fp, 0, sizeof(fp));
    for (int c = 0; c < 3; ++c) fp.eye[c] = f->eye[c];
    for (int p = 0; p < 5; ++p)
        for (int c = 0; c < 3; ++c) fp.planes[3 * p + c] = f->planes[p][c];
    fp.q = f->q;
    fp.nplanes = f->nplanes;
    fp.mode = f->mode;
    fp.seed = f->seed;
    fp.precision = f->precision;
    fp.shift = f->fixed_shift;
    fp.gate = f->gate;
    fp.split_list = f->split_list;
    fp.n_split = f->n_split;
    fp.merge_list = f->merge_list;
    fp.n_merge = f->n_merge;
    fp.frame = frame;
    if (f->vertices_out && f->vertices_cap == 0) return false;
    return true;
}

}  // namespace

extern "C" size_t cbt_workspace_bytes(int32_t H, int32_t D) {
    Layout L;
    return make_layout(H, D, L) ? L.total : 0u;
}

extern "C" int cbt_create(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                          const int32_t* vert, const int32_t* face, int32_t V, const double* pos,
                          int32_t D, int32_t max_depth, void* workspace, size_t bytes,
                          cbt_stream_t stream, cbt_state** out) {
    if (!out) return CBT_EINVAL;
    *out = nullptr;
    if (!pos || !workspace) return CBT_EINVAL;
    int rc = validate_halfedges(H, twin, next, prev, vert, face, V);
    if (rc) return rc;
    const uint32_t ch = ceil_log2(static_cast<uint32_t>(H));
    if (D < 1 || D > 30 || static_cast<uint32_t>(D) < ch) return CBT_ECAPACITY;
    if (max_depth < 0 || ch + 1u + static_cast<uint32_t>(max_depth) > 63u) return CBT_EDEPTH;
    Layout L;
    if (!make_layout(H, D, L)) return CBT_EINVAL;
    if (bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return CBT_ENOMEM;

    cbt_state* st = new cbt_state();
    st->workspace = workspace;
    st->bytes = bytes;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&st->sms, cudaDevAttrMultiProcessorCount, dev);
    if (st->sms <= 0) st->sms = 1;
    char* b = static_cast<char*>(workspace);
    Inst& I = st->inst;
    I.g = reinterpret_cast<Globals*>(b + L.globals);
    I.heap = reinterpret_cast<uint64_t*>(b + L.heap);
    I.nb = reinterpret_cast<uint4*>(b + L.nb);
    I.cd = reinterpret_cast<uint2*>(b + L.cd);
    I.bits = reinterpret_cast<uint32_t*>(b + L.bits);
    I.sums = reinterpret_cast<uint32_t*>(b + L.sums);
    I.live = reinterpret_cast<uint32_t*>(b + L.live);
    I.freel = reinterpret_cast<uint32_t*>(b + L.freel);
    I.scan = reinterpret_cast<uint32_t*>(b + L.scan);
    I.status = reinterpret_cast<unsigned long long*>(b + L.status);
    I.root64 = reinterpret_cast<double*>(b + L.root64);
    I.rel = b + L.rel;
    I.cap = L.cap;
    I.W = L.W;
    I.D = static_cast<uint32_t>(D);
    I.H = static_cast<uint32_t>(H);
    I.ch = ch;
    I.max_depth = static_cast<uint32_t>(max_depth);
    I.ntiles_items = L.ntiles_items;
    I.ntiles_words = L.ntiles_words;
    I.tile_words = L.tile_words;

    // Stage the halfedge operators and the position of Vert(h) per halfedge
    // in the (not yet used) relative-vertex region.
    const size_t h = static_cast<size_t>(H);
    std::vector<int32_t> ints(4u * h);
    std::vector<double> hpos(3u * h);
    for (size_t k = 0; k < h; ++k) {
        ints[k] = twin[k];
        ints[h + k] = next[k];
        ints[2u * h + k] = prev[k];
        ints[3u * h + k] = face[k];
        for (int c = 0; c < 3; ++c) hpos[3u * k + c] = pos[3u * static_cast<size_t>(vert[k]) + c];
    }
    int32_t* d_ints = reinterpret_cast<int32_t*>(b + L.rel);
    double* d_hpos = reinterpret_cast<double*>(b + L.rel + 16u * h);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(I.g, 0, sizeof(Globals), s);
    cudaMemsetAsync(I.status, 0, 8u * (3u * static_cast<size_t>(L.ntiles_items) + L.ntiles_words), s);
    cudaMemcpyAsync(d_ints, ints.data(), 16u * h, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_hpos, hpos.data(), 24u * h, cudaMemcpyHostToDevice, s);
    const int grid = static_cast<int>(std::min<uint32_t>((std::max(L.W, static_cast<uint32_t>(H)) + 255u) / 256u,
                                                         static_cast<uint32_t>(st->sms) * 4u));
    launch_init(I, d_ints, d_ints + h, d_ints + 2u * h, d_ints + 3u * h, d_hpos, std::max(1, grid), s);
    launch_cbt(I, grid_words(st), s);
    rc = check_launch();
    if (rc == CBT_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = CBT_ECUDA;
    if (rc) {
        delete st;
        return rc;
    }
    *out = st;
    return CBT_OK;
}

extern "C" int cbt_update(cbt_state* st, const cbt_frame* frame, cbt_stream_t stream) {
    if (!st) return CBT_EINVAL;
    FrameP fp;
    if (!frame_from_api(frame, st->frame, fp)) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const Inst& I = st->inst;
    uint32_t k = 0;
    auto mark = [&]() {
        if (st->timing) cudaEventRecord(st->ev[k], s);
        ++k;
    };
    mark();
    launch_prep(I, fp, true, grid_prep(st, true), s);
    mark();
    launch_classify(I, fp, grid_items(st), s);
    mark();
    launch_gate(I, fp, grid_tiles(st), s);
    mark();
    launch_scatter(I, grid_items(st), s);
    mark();
    launch_alloc(I, grid_tiles(st), s);
    mark();
    launch_free(I, grid_words(st), s);
    mark();
    launch_fill(I, grid_items(st), s);
    mark();
    launch_cbt(I, grid_words(st), s);
    mark();
    if (frame->vertices_out) {
        launch_vertices(I, fp, frame->vertices_out, frame->vertices_cap, grid_items(st), s);
        mark();
    }
    st->launches = k - 1u;
    st->timed = st->timing ? k - 1u : 0u;
    st->frame += 1u;
    return check_launch();
}

extern "C" int cbt_live_count(cbt_state* st, uint32_t* h_count, cbt_stream_t stream) {
    if (!st || !h_count) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h_count, st->inst.sums + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CBT_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_leaves(cbt_state* st, uint32_t* d_slots, uint64_t* d_heap, uint32_t* d_links,
                          uint32_t cap, uint32_t* h_count, cbt_stream_t stream) {
    uint32_t n = 0;
    int rc = cbt_live_count(st, &n, stream);
    if (rc) return rc;
    if (h_count) *h_count = n;
    if (n > cap) return CBT_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    launch_leaves(st->inst, d_slots, d_heap, d_links, grid_items(st), s);
    rc = check_launch();
    if (rc) return rc;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_vertices(cbt_state* st, float* d_out, const double h_origin[3], uint32_t precision,
                            int32_t fixed_shift, uint32_t cap, uint32_t* h_count, cbt_stream_t stream) {
    if (!st || !d_out || !h_origin || precision > 2u || fixed_shift < 0 || fixed_shift > 62)
        return CBT_EINVAL;
    uint32_t n = 0;
    int rc = cbt_live_count(st, &n, stream);
    if (rc) return rc;
    if (h_count) *h_count = n;
    if (n > cap) return CBT_ENOMEM;
    FrameP fp;
    std::memset(&fp, 0, sizeof(fp));
    for (int c = 0; c < 3; ++c) fp.eye[c] = h_origin[c];
    fp.precision = precision;
    fp.shift = fixed_shift;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    launch_prep(st->inst, fp, false, grid_prep(st, false), s);
    launch_vertices(st->inst, fp, d_out, cap, grid_items(st), s);
    rc = check_launch();
    if (rc) return rc;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_cbt(cbt_state* st, uint32_t* d_bitfield, uint32_t* d_sums, cbt_stream_t stream) {
    if (!st) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (d_bitfield && cudaMemcpyAsync(d_bitfield, st->inst.bits, 4u * st->inst.W,
                                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return CBT_ECUDA;
    if (d_sums && cudaMemcpyAsync(d_sums, st->inst.sums, 8u * st->inst.W, cudaMemcpyDeviceToDevice, s) !=
                      cudaSuccess)
        return CBT_ECUDA;
    return CBT_OK;
}

extern "C" int cbt_stats(cbt_state* st, cbt_frame_stats* out, cbt_stream_t stream) {
    if (!st || !out) return CBT_EINVAL;
    Globals g;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&g, st->inst.g, sizeof(Globals), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CBT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CBT_ECUDA;
    out->live_before = g.stats[kStLiveBefore];
    out->live_after = g.stats[kStLiveAfter];
    out->free_before = g.stats[kStFreeBefore];
    out->split_wishes = g.stats[kStSplitWishes];
    out->merge_candidates = g.stats[kStMergeCand];
    out->split_granted = g.stats[kStSplitGranted];
    out->merge_granted = g.stats[kStMergeGranted];
    out->split_bisectors = g.stats[kStSplitBis];
    out->merged_bisectors = g.stats[kStMergedBis];
    out->merge_groups = g.stats[kStMergeGroups];
    out->allocated = g.stats[kStAllocated];
    out->relinked = g.stats[kStRelinked];
    out->frame = st->frame;
    out->error = g.err;
    return g.err ? CBT_EDEVICE : CBT_OK;
}

extern "C" void cbt_destroy(cbt_state* st) {
    if (!st) return;
    if (st->timing)
        for (auto& e : st->ev) cudaEventDestroy(e);
    delete st;
}

extern "C" int cbt_set_timing(cbt_state* st, int on) {
    if (!st) return CBT_EINVAL;
    if (on && !st->timing) {
        for (auto& e : st->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return CBT_ECUDA;
        st->timing = true;
    } else if (!on && st->timing) {
        for (auto& e : st->ev) cudaEventDestroy(e);
        st->timing = false;
        st->timed = 0;
    }
    return CBT_OK;
}

extern "C" uint32_t cbt_kernel_times(cbt_state* st, float* ms, uint32_t n) {
    if (!st || !st->timing || st->timed == 0 || !ms) return 0u;
    if (cudaEventSynchronize(st->ev[st->timed]) != cudaSuccess) return 0u;
    const uint32_t m = std::min(n, st->timed);
    for (uint32_t k = 0; k < m; ++k) {
        ms[k] = 0.0f;
        cudaEventElapsedTime(&ms[k], st->ev[k], st->ev[k + 1]);
    }
    return m;
}

extern "C" const char* cbt_kernel_name(uint32_t k) { return k < kMaxKernels ? kKernelNames[k] : ""; }

extern "C" uint32_t cbt_last_launch_count(const cbt_state* st) { return st ? st->launches : 0u; }
