// C ABI of the CBT bisection library (declared in include/cbt.h).
//
// A single instance is updated as a batch of one: its workspace holds, after
// its own arrays, a small batch region (instance table, frame parameters,
// tile prefixes, look-back descriptors). cbt_batch_* build the same region
// for many instances in a caller-provided workspace, so that one launch per
// kernel updates them all.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cbt.h"
#include "cbt_kernels.cuh"

namespace cbtgpu {
int validate_halfedges(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                       const int32_t* vert, const int32_t* face, int32_t V);
}

using namespace cbtgpu;

namespace {

constexpr int kNumKernels = 10;
const char* const kKernelNames[kNumKernels] = {"prep", "classify", "walk", "gate", "scatter", "alloc",
                                               "free", "fill", "cbt", "vertices"};
// launches per entry of kKernelNames ("cbt" is the reduction plus the compaction)
constexpr uint32_t kLaunchesPerStep[kNumKernels] = {1, 1, 1, 1, 1, 1, 1, 1, 2, 1};
// phases of the one-launch frame
const char* const kPhaseNames[kFramePhases] = {"prep",  "classify", "gate_sum", "gate",    "alloc_sum",
                                               "alloc", "fill",     "reduce",   "compact", "vertices"};
// phases of the single-instance frame (k_frame1)
const char* const kPhaseNames1[kFrame1Phases] = {"prep",  "classify", "walks", "gate",
                                                 "alloc", "fill",     "final", "vertices"};
constexpr uint32_t kFusedTileWords = 64;
constexpr uint32_t kFusedMaxTileWords = 128;

size_t align256(size_t x) { return (x + 255u) & ~static_cast<size_t>(255u); }

uint32_t ceil_log2(uint32_t x) {
    uint32_t c = 0;
    while ((1ull << c) < static_cast<uint64_t>(x)) ++c;
    return c;
}

uint32_t word_tiles(uint32_t W, uint32_t tw) { return W / std::min(W, tw); }
uint32_t item_tiles(uint32_t cap) { return (cap + kTileItems - 1u) / kTileItems; }

// Per-instance arrays.
struct Layout {
    size_t globals, heap, nb, cd, bits, sums, live, freel, scan, grp, chg, chgr, vc, root64, rel, corner, rbnd, batch,
        total;
    uint32_t cap, W, ch;
};

// A batch region for instances with the given pool sizes and halfedge counts.
struct BatchLayout {
    size_t inst, fps, bg, tile_base, ctile_base, stile_base, wtile_base, vtile_base, rel_base, status, tpre, total;
    uint32_t Titems, TwordsMax, Trel;
};

BatchLayout batch_layout(uint32_t n, const uint32_t* cap, const uint32_t* W, const uint32_t* H) {
    BatchLayout L{};
    for (uint32_t b = 0; b < n; ++b) {
        L.Titems += item_tiles(cap[b]);
        L.TwordsMax += word_tiles(W[b], kMinTileWords);
        L.Trel += 9u * H[b];
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.inst = take(sizeof(Inst) * n);
    L.fps = take(sizeof(FrameP) * n);
    L.bg = take(sizeof(BatchGlobals));
    L.tile_base = take(4u * (n + 1u));
    L.ctile_base = take(4u * (n + 1u));
    L.stile_base = take(4u * (n + 1u));
    L.wtile_base = take(4u * (n + 1u));
    L.vtile_base = take(4u * (n + 1u));
    L.rel_base = take(4u * (n + 1u));
    L.status = take(8u * (2u * static_cast<size_t>(L.Titems) + L.TwordsMax));
    L.tpre = take(4u * 2u * static_cast<size_t>(L.TwordsMax));
    L.total = off;
    return L;
}

bool make_layout(int32_t H, int32_t D, Layout& L) {
    if (H < 3 || D < 1 || D > 30) return false;
    L.ch = ceil_log2(static_cast<uint32_t>(H));
    if (static_cast<uint32_t>(D) < L.ch) return false;
    L.cap = 1u << D;
    L.W = std::max(1u, L.cap / 32u);
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t o = off;
        off = align256(off + n);
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
    L.grp = take(16u * cap);
    L.chg = take(4u * cap);
    L.chgr = take(16u * cap);
    L.vc = take(36u * cap);
    L.root64 = take(72u * h);
    L.rel = take(72u * h);
    L.corner = take(12u * h);
    L.rbnd = take(4u * ((h + 31u) / 32u));
    const uint32_t Hh = static_cast<uint32_t>(H);
    const BatchLayout B = batch_layout(1, &L.cap, &L.W, &Hh);
    L.batch = take(B.total);
    L.total = off;
    return true;
}

int check_launch() { return cudaGetLastError() == cudaSuccess ? CBT_OK : CBT_ECUDA; }

bool frame_from_api(const cbt_frame* f, uint32_t frame, FrameP& fp) {
    if (!f || f->precision > 3u || f->mode > 4u || f->nplanes > 5u || f->gate > 1u) return false;
    if (f->precision == 3u && !(f->sphere_radius > 0.0 && f->sphere_radius < 1e300)) return false;
    if (f->fixed_shift < 0 || f->fixed_shift > 62) return false;
    if (f->mode == CBT_MODE_LIST && ((f->n_split && !f->split_list) || (f->n_merge && !f->merge_list)))
        return false;
    if (f->vertices_out && (f->vertices_cap == 0 || (reinterpret_cast<uintptr_t>(f->vertices_out) & 3u))) return false;
    if (f->disp_amplitude != 0.0f &&
        !(std::isfinite(f->disp_amplitude) && std::isfinite(f->disp_frequency) && f->disp_frequency > 0.0f &&
          f->disp_octaves >= 1u && f->disp_octaves <= 8u && (f->precision == 0u || f->precision == 3u)))
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
    fp.radius = f->sphere_radius;
    fp.shift = f->fixed_shift;
    fp.gate = f->gate;
    fp.split_list = f->split_list;
    fp.n_split = f->n_split;
    fp.merge_list = f->merge_list;
    fp.n_merge = f->n_merge;
    fp.frame = frame;
    fp.vout = f->vertices_out;
    fp.vcap = f->vertices_cap;
    if (f->disp_amplitude != 0.0f) {
        fp.damp = f->disp_amplitude;
        fp.dfreq = f->disp_frequency;
        fp.doct = f->disp_octaves;
        fp.dseed = f->disp_seed;
    }
    return true;
}

}  // namespace

// Host side of a batch (also the batch of one inside every state).
struct cbt_batch {
    std::vector<cbt_state*> st;
    uint32_t n = 0;
    int sms = 1;
    char* region = nullptr;
    BatchLayout L{};
    BatchDev dev{};
    std::vector<uint32_t> cap, W, H;
    FrameP* h_fps = nullptr;  // pinned staging for the per-instance frame parameters
    cudaEvent_t staged = nullptr;
    bool staged_pending = false;
    uint32_t tw = kFusedTileWords;
    uint32_t grid_mult = 8;
    bool fused = true;   // one cooperative launch per frame (else one launch per step)
    int fused_grid = 1;  // its blocks: resident blocks per SM x SMs, at most the tiles
    int fused_grid1 = 0; // the same for the single-instance frame (0: not available)
    bool last_frame1 = false;  // the last fused frame ran the single-instance kernel
    bool use_graph = false;
    cudaGraphExec_t exec = nullptr;
    uint32_t exec_tw = 0, exec_mult = 0;
    bool exec_vertices = false, exec_fused = false;
    bool timing = false;
    cudaEvent_t ev[kNumKernels + 1] = {};
    uint32_t timed = 0, launches = 0;
    // online autotuner over (tile words, blocks per SM)
    bool tuning = false;
    uint32_t tune_k = 0, tune_rounds = 0;
    std::vector<float> tune_ms;
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    bool tune_pending = false;
    uint32_t tune_cfg = 0;
};

struct cbt_state {
    Inst inst;
    uint32_t* corner;  // [H][3] global points of the root corners: vert[h], vert[next h], V + face[h]
    uint32_t npts;     // global points: 1 + the largest in corner
    uint32_t* h_ix = nullptr;  // pinned counts of the last cbt_index (made by its first call)
    void* workspace;
    size_t bytes;
    int sms;
    uint32_t frame;
    cbt_batch* self;
};

namespace {

const uint32_t kTuneTw[3] = {64, 128, 256};
const uint32_t kTuneMult[3] = {4, 8, 16};

// Word tile of the one-launch frame: 64 words, unless the batch's bitfields
// make more than four tiles per resident block, where each tile's setup
// (instance lookup, block synchronisations) would dominate: then 128, the
// most its compaction can stage (32 positions per word in a 4096-word
// shared buffer).
uint32_t fused_tile_words(const cbt_batch* B) {
    uint64_t tiles = 0;
    for (uint32_t b = 0; b < B->n; ++b) tiles += word_tiles(B->W[b], kFusedTileWords);
    const uint64_t grid = static_cast<uint64_t>(B->sms) * static_cast<uint64_t>(frame_blocks_per_sm());
    return tiles > 4u * grid ? kFusedMaxTileWords : kFusedTileWords;
}

int upload_static_prefixes(cbt_batch* B, cudaStream_t s) {
    std::vector<uint32_t> w(B->n + 1), v(B->n + 1), r(B->n + 1);
    w[0] = v[0] = r[0] = 0;
    for (uint32_t b = 0; b < B->n; ++b) {
        w[b + 1] = w[b] + word_tiles(B->W[b], B->tw);
        v[b + 1] = v[b] + item_tiles(B->cap[b]);
        r[b + 1] = r[b] + 9u * B->H[b];
    }
    B->dev.Twords = w[B->n];
    B->dev.Titems = v[B->n];
    B->dev.Trel = r[B->n];
    B->dev.tw = B->tw;
    const size_t bytes = 4u * (B->n + 1u);
    if (cudaMemcpyAsync(const_cast<uint32_t*>(B->dev.wtile_base), w.data(), bytes, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(const_cast<uint32_t*>(B->dev.vtile_base), v.data(), bytes, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(const_cast<uint32_t*>(B->dev.rel_base), r.data(), bytes, cudaMemcpyHostToDevice, s))
        return CBT_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

// Builds a batch over `n` states in `region` (L.total bytes of device memory).
int batch_build(cbt_state* const* states, uint32_t n, char* region, cudaStream_t s, cbt_batch** out) {
    cbt_batch* B = new cbt_batch();
    B->n = n;
    B->st.assign(states, states + n);
    B->sms = states[0]->sms;
    for (uint32_t b = 0; b < n; ++b) {
        B->cap.push_back(states[b]->inst.cap);
        B->W.push_back(states[b]->inst.W);
        B->H.push_back(states[b]->inst.H);
    }
    B->L = batch_layout(n, B->cap.data(), B->W.data(), B->H.data());
    B->region = region;
    BatchDev& d = B->dev;
    d.inst = reinterpret_cast<const Inst*>(region + B->L.inst);
    d.fps = nullptr;
    d.B = n;
    d.tile_base = reinterpret_cast<uint32_t*>(region + B->L.tile_base);
    d.ctile_base = reinterpret_cast<uint32_t*>(region + B->L.ctile_base);
    d.stile_base = reinterpret_cast<uint32_t*>(region + B->L.stile_base);
    d.wtile_base = reinterpret_cast<const uint32_t*>(region + B->L.wtile_base);
    d.vtile_base = reinterpret_cast<const uint32_t*>(region + B->L.vtile_base);
    d.rel_base = reinterpret_cast<const uint32_t*>(region + B->L.rel_base);
    d.bg = reinterpret_cast<BatchGlobals*>(region + B->L.bg);
    d.status = reinterpret_cast<unsigned long long*>(region + B->L.status);
    d.tpre = reinterpret_cast<uint32_t*>(region + B->L.tpre);
    std::vector<Inst> insts(n);
    for (uint32_t b = 0; b < n; ++b) insts[b] = states[b]->inst;
    std::memset(&d.inst0, 0, sizeof(Inst));
    if (n == 1) d.inst0 = insts[0];
    int rc = CBT_OK;
    if (cudaMemcpyAsync(region + B->L.inst, insts.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(d.bg, 0, sizeof(BatchGlobals), s) ||
        cudaMallocHost(reinterpret_cast<void**>(&B->h_fps), sizeof(FrameP) * n) ||
        cudaEventCreateWithFlags(&B->staged, cudaEventDisableTiming))
        rc = CBT_ECUDA;
    B->tw = fused_tile_words(B);  // the one-launch frame is the default form
    if (!rc) rc = upload_static_prefixes(B, s);
    if (!rc) {
        const int per_sm = frame_blocks_per_sm();
        if (per_sm <= 0) rc = CBT_ECUDA;
        const uint32_t work = std::max({B->dev.Titems, B->dev.Twords, (B->dev.Trel + 255u) / 256u, 1u});
        B->fused_grid = static_cast<int>(std::min<uint32_t>(work, static_cast<uint32_t>(per_sm * B->sms)));
        // the single-instance frame spreads classify, the walks and the rows
        // of its export over the whole grid, so a small instance also gets
        // every SM
        const int per_sm1 = n == 1 ? frame1_blocks_per_sm() : 0;
        if (per_sm1 > 0) B->fused_grid1 = per_sm1 * B->sms;
    }
    if (rc) {
        if (B->h_fps) cudaFreeHost(B->h_fps);
        delete B;
        return rc;
    }
    *out = B;
    return CBT_OK;
}

void batch_free(cbt_batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->timing)
        for (auto& e : B->ev) cudaEventDestroy(e);
    for (auto& e : B->tune_ev)
        if (e) cudaEventDestroy(e);
    if (B->staged) cudaEventDestroy(B->staged);
    if (B->h_fps) cudaFreeHost(B->h_fps);
    delete B;
}

int grid_prep(const cbt_batch* B) {
    const uint32_t n = std::max(B->dev.Trel, 2u * B->dev.Titems + B->dev.Twords);
    const uint32_t want = (n + kThreads - 1u) / kThreads;
    return static_cast<int>(std::max(1u, std::min<uint32_t>(want, static_cast<uint32_t>(B->sms) * 4u)));
}

// The kernels of one frame of a batch descriptor; ev (optional) receives an
// event before and after every kernel. Returns the number of launches.
uint32_t enqueue_kernels(const BatchDev& bt, int sms, uint32_t grid_mult, bool vertices, cudaStream_t s,
                         cudaEvent_t* ev) {
    const uint32_t prep_n = std::max(bt.Trel, 2u * bt.Titems + bt.Twords);
    const int prep = static_cast<int>(std::max(1u, std::min<uint32_t>((prep_n + kThreads - 1u) / kThreads,
                                                                     static_cast<uint32_t>(sms) * 4u)));
    const int items = std::max(1, static_cast<int>(std::min<uint32_t>(bt.Titems, static_cast<uint32_t>(sms) * grid_mult)));
    const int scans = std::max(1, static_cast<int>(std::min<uint32_t>(bt.Titems, static_cast<uint32_t>(sms) * 4u)));
    const int words = std::max(1, static_cast<int>(std::min<uint32_t>(bt.Twords, static_cast<uint32_t>(sms) * 4u)));
    uint32_t k = 0;
    auto mark = [&]() {
        if (ev) cudaEventRecord(ev[k], s);
        ++k;
    };
    mark();
    launch_prep(bt, true, prep, s);
    mark();
    launch_classify(bt, items, s);
    mark();
    launch_walk(bt, items, s);
    mark();
    launch_gate(bt, scans, s);
    mark();
    launch_scatter(bt, items, s);
    mark();
    launch_alloc(bt, scans, s);
    mark();
    launch_free(bt, words, s);
    mark();
    launch_fill(bt, items, s);
    mark();
    launch_cbt(bt, words, s);
    mark();
    if (vertices) {
        launch_vertices(bt, items, s);
        mark();
    }
    uint32_t launches = 0;
    for (uint32_t q = 0; q + 1u < k; ++q) launches += kLaunchesPerStep[q];
    return launches;
}

// The kernels of one frame. `timed`: record events between the kernels (the
// one-launch frame records its phase boundaries on the device instead).
// A single instance whose pool and word tiles fit the single-instance
// frame's shared tables runs that kernel.
bool use_frame1(const cbt_batch* B) {
    return B->n == 1 && B->fused_grid1 > 0 && B->cap[0] <= kFrame1MaxCap && B->tw == kFrame1TileWords;
}

void enqueue_frame(cbt_batch* B, cudaStream_t s, bool vertices, bool timed) {
    if (B->fused) {
        BatchDev bt = B->dev;
        bt.timing = timed ? 1u : 0u;
        B->launches = 1;
        if (use_frame1(B)) {
            const uint32_t span = std::min<uint32_t>(B->cap[0], 32u * B->tw);
            launch_frame1(bt, B->fused_grid1, ceil_log2(span), s);
            B->last_frame1 = true;
            B->timed = timed ? static_cast<uint32_t>(kFrame1Phases) : 0u;
            return;
        }
        B->last_frame1 = false;
        launch_frame(bt, B->fused_grid, s);
        // a batch exports vertices within its compaction phase
        B->timed = timed ? static_cast<uint32_t>(B->n == 1 ? kFramePhases : kFramePhases - 1) : 0u;
        return;
    }
    B->launches = enqueue_kernels(B->dev, B->sms, B->grid_mult, vertices, s, timed ? B->ev : nullptr);
    B->timed = timed ? (vertices ? 10u : 9u) : 0u;
}

int apply_config(cbt_batch* B, uint32_t tw, uint32_t mult, cudaStream_t s) {
    B->grid_mult = mult;
    B->fused = false;
    if (tw == B->tw) return CBT_OK;
    B->tw = tw;
    return upload_static_prefixes(B, s);
}

int set_fused(cbt_batch* B, bool on, cudaStream_t s) {
    if (!on) {
        B->fused = false;
        return CBT_OK;
    }
    const uint32_t tw = fused_tile_words(B);
    if (B->tw != tw) {
        B->tw = tw;
        const int rc = upload_static_prefixes(B, s);
        if (rc) return rc;
    }
    B->fused = true;
    return CBT_OK;
}

int batch_update(cbt_batch* B, const cbt_frame* frames, cudaStream_t s) {
    const uint32_t n = B->n;
    std::vector<FrameP> fps(n);
    bool vertices = false;
    for (uint32_t b = 0; b < n; ++b) {
        if (!frame_from_api(frames + b, B->st[b]->frame, fps[b])) return CBT_EINVAL;
        vertices = vertices || fps[b].vout != nullptr;
    }
    // online autotuner: one candidate configuration per frame, round robin,
    // then the fastest by median time per live bisector (results do not depend on it)
    if (B->tuning) {
        if (B->tune_pending) {
            // candidates run on different frames, whose work differs: compare
            // time per live bisector of the batch
            float ms = 0.0f;
            uint32_t live = 0;
            cudaEventSynchronize(B->tune_ev[1]);
            cudaEventElapsedTime(&ms, B->tune_ev[0], B->tune_ev[1]);
            if (cudaMemcpy(&live, &B->dev.bg->live_total, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                return CBT_ECUDA;
            B->tune_ms.push_back(ms / static_cast<float>(std::max(live, 1u)));
            B->tune_pending = false;
        }
        const uint32_t ncfg = 10;  // 3 x 3 per-step configurations, then the one-launch frame
        auto apply = [&](uint32_t c) {
            return c == 9 ? set_fused(B, true, s) : apply_config(B, kTuneTw[c / 3], kTuneMult[c % 3], s);
        };
        if (B->tune_ms.size() >= ncfg * B->tune_rounds) {
            uint32_t best = 0;
            float best_ms = 1e30f;
            for (uint32_t c = 0; c < ncfg; ++c) {
                std::vector<float> v;
                for (size_t k = c; k < B->tune_ms.size(); k += ncfg) v.push_back(B->tune_ms[k]);
                std::sort(v.begin(), v.end());
                const float med = v[v.size() / 2];
                if (med < best_ms) {
                    best_ms = med;
                    best = c;
                }
            }
            B->tuning = false;
            B->tune_cfg = best;
            int rc = apply(best);
            if (rc) return rc;
        } else {
            int rc = apply(static_cast<uint32_t>(B->tune_ms.size()) % ncfg);
            if (rc) return rc;
        }
    }
    const bool tune_now = B->tuning;
    if (tune_now) cudaEventRecord(B->tune_ev[0], s);
    // A single instance in the fused form is one launch whose parameters
    // travel by value: launched directly, it starts sooner than a graph
    // whose first node copies the parameters.
    const bool direct = B->fused && n == 1;
    if (B->use_graph && !direct) {
        // the graph copies the frame parameters from pinned staging
        if (B->staged_pending) cudaEventSynchronize(B->staged);
        std::memcpy(B->h_fps, fps.data(), sizeof(FrameP) * n);
        if (!B->exec || B->exec_tw != B->tw || B->exec_mult != B->grid_mult || B->exec_vertices != vertices ||
            B->exec_fused != B->fused) {
            if (B->exec) {
                cudaGraphExecDestroy(B->exec);
                B->exec = nullptr;
            }
            cudaStream_t cs;
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) return CBT_ECUDA;
            cudaGraph_t g = nullptr;
            B->dev.fps = reinterpret_cast<const FrameP*>(B->region + B->L.fps);
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            cudaMemcpyAsync(B->region + B->L.fps, B->h_fps, sizeof(FrameP) * n, cudaMemcpyHostToDevice, cs);
            enqueue_frame(B, cs, vertices, false);
            const cudaError_t e1 = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (e1 != cudaSuccess || !g) return CBT_ECUDA;
            const cudaError_t e2 = cudaGraphInstantiate(&B->exec, g, 0);
            cudaGraphDestroy(g);
            if (e2 != cudaSuccess) return CBT_ECUDA;
            B->exec_tw = B->tw;
            B->exec_mult = B->grid_mult;
            B->exec_vertices = vertices;
            B->exec_fused = B->fused;
        }
        if (cudaGraphLaunch(B->exec, s) != cudaSuccess) return CBT_ECUDA;
        cudaEventRecord(B->staged, s);
        B->staged_pending = true;
        B->timed = 0;
    } else if (n == 1) {
        B->dev.fps = nullptr;
        B->dev.fp0 = fps[0];
        enqueue_frame(B, s, vertices, B->timing);
    } else {
        if (B->staged_pending) cudaEventSynchronize(B->staged);
        std::memcpy(B->h_fps, fps.data(), sizeof(FrameP) * n);
        if (cudaMemcpyAsync(B->region + B->L.fps, B->h_fps, sizeof(FrameP) * n, cudaMemcpyHostToDevice, s))
            return CBT_ECUDA;
        cudaEventRecord(B->staged, s);
        B->staged_pending = true;
        B->dev.fps = reinterpret_cast<const FrameP*>(B->region + B->L.fps);
        enqueue_frame(B, s, vertices, B->timing);
    }
    if (tune_now) {
        cudaEventRecord(B->tune_ev[1], s);
        B->tune_pending = true;
    }
    for (uint32_t b = 0; b < n; ++b) B->st[b]->frame += 1u;
    return check_launch();
}

}  // namespace

extern "C" size_t cbt_workspace_bytes(int32_t H, int32_t D) {
    Layout L;
    return make_layout(H, D, L) ? L.total : 0u;
}

extern "C" size_t cbt_point_cache_bytes(int32_t D) {
    if (D < 1 || D > 30) return 0;
    return 144u * (static_cast<size_t>(1) << D);
}

extern "C" int cbt_attach_point_cache(cbt_state* st, void* memory, size_t bytes, cbt_stream_t stream) {
    if (!st || !memory || (reinterpret_cast<uintptr_t>(memory) & 15u) || st->inst.pc) return CBT_EINVAL;
    const size_t cap = st->inst.cap;
    if (bytes < 144u * cap) return CBT_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(memory);
    Inst I = st->inst;
    I.pc = reinterpret_cast<double*>(b);                // [16][cap]
    I.pct = reinterpret_cast<ulonglong2*>(b + 128u * cap);  // [cap], cleared: heap ID 0 is never live
    if (cudaMemsetAsync(I.pct, 0, 16u * cap, s) != cudaSuccess ||
        cudaMemcpyAsync(const_cast<Inst*>(st->self->dev.inst), &I, sizeof(Inst), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CBT_ECUDA;
    st->inst = I;
    st->self->dev.inst0 = I;
    return CBT_OK;
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
    st->frame = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&st->sms, cudaDevAttrMultiProcessorCount, dev);
    if (st->sms <= 0) st->sms = 1;
    char* b = static_cast<char*>(workspace);
    Inst& I = st->inst;
    std::memset(&I, 0, sizeof(I));
    I.g = reinterpret_cast<Globals*>(b + L.globals);
    I.heap = reinterpret_cast<uint64_t*>(b + L.heap);
    I.nb = reinterpret_cast<uint4*>(b + L.nb);
    I.cd = reinterpret_cast<uint2*>(b + L.cd);
    I.bits = reinterpret_cast<uint32_t*>(b + L.bits);
    I.sums = reinterpret_cast<uint32_t*>(b + L.sums);
    I.live = reinterpret_cast<uint32_t*>(b + L.live);
    I.freel = reinterpret_cast<uint32_t*>(b + L.freel);
    I.scan = reinterpret_cast<uint32_t*>(b + L.scan);
    I.grp = reinterpret_cast<uint4*>(b + L.grp);
    I.chg = reinterpret_cast<uint32_t*>(b + L.chg);
    I.chgr = reinterpret_cast<uint4*>(b + L.chgr);
    I.vc = reinterpret_cast<float*>(b + L.vc);
    I.pc = nullptr;  // no point cache until cbt_attach_point_cache
    I.pct = nullptr;
    I.root64 = reinterpret_cast<double*>(b + L.root64);
    I.rel = b + L.rel;
    I.cap = L.cap;
    I.W = L.W;
    I.D = static_cast<uint32_t>(D);
    I.H = static_cast<uint32_t>(H);
    I.ch = ch;
    I.max_depth = static_cast<uint32_t>(max_depth);
    I.ntiles_items = item_tiles(L.cap);

    // Stage the halfedge operators and the position of Vert(h) per halfedge
    // in the (not yet used) relative-vertex region.
    const size_t h = static_cast<size_t>(H);
    std::vector<int32_t> ints(3u * h);
    std::vector<double> hpos(3u * h);
    std::vector<uint32_t> corner(3u * h);
    std::vector<uint32_t> rbnd((h + 31u) / 32u, 0u);
    for (size_t k = 0; k < h; ++k) {
        if (twin[k] < 0) rbnd[k >> 5] |= 1u << (k & 31u);
        ints[k] = twin[k];
        ints[h + k] = next[k];
        ints[2u * h + k] = prev[k];
        for (int c = 0; c < 3; ++c) hpos[3u * k + c] = pos[3u * static_cast<size_t>(vert[k]) + c];
        corner[3u * k] = static_cast<uint32_t>(vert[k]);
        corner[3u * k + 1u] = static_cast<uint32_t>(vert[next[k]]);
        corner[3u * k + 2u] = static_cast<uint32_t>(V) + static_cast<uint32_t>(face[k]);
    }
    st->corner = reinterpret_cast<uint32_t*>(b + L.corner);
    st->npts = h ? 1u + *std::max_element(corner.begin(), corner.end()) : 0u;
    int32_t* d_ints = reinterpret_cast<int32_t*>(b + L.rel);
    double* d_hpos = reinterpret_cast<double*>(b + L.rel + align256(12u * h));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaMemsetAsync(I.g, 0, sizeof(Globals), s);
    cudaMemcpyAsync(d_ints, ints.data(), 12u * h, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_hpos, hpos.data(), 24u * h, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(st->corner, corner.data(), 12u * h, cudaMemcpyHostToDevice, s);
    I.rbnd = reinterpret_cast<const uint32_t*>(b + L.rbnd);
    cudaMemcpyAsync(const_cast<uint32_t*>(I.rbnd), rbnd.data(), 4u * rbnd.size(), cudaMemcpyHostToDevice, s);
    const int grid = static_cast<int>(std::min<uint32_t>((std::max(L.W, static_cast<uint32_t>(H)) + 255u) / 256u,
                                                         static_cast<uint32_t>(st->sms) * 4u));
    launch_init(I, d_ints, d_ints + h, d_ints + 2u * h, d_hpos, std::max(1, grid), s);
    rc = check_launch();
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = CBT_ECUDA;
    if (!rc) {
        cbt_state* self[1] = {st};
        rc = batch_build(self, 1, b + L.batch, s, &st->self);
    }
    if (!rc) {
        // the reduction and live list of the roots
        cbt_batch* B = st->self;
        cudaMemsetAsync(B->dev.status, 0, 8u * (2u * static_cast<size_t>(B->dev.Titems) + B->dev.Twords), s);
        cudaMemsetAsync(B->dev.bg, 0, sizeof(BatchGlobals), s);
        B->dev.fps = nullptr;
        std::memset(&B->dev.fp0, 0, sizeof(FrameP));
        launch_cbt(B->dev, std::max(1, static_cast<int>(std::min<uint32_t>(B->dev.Twords, static_cast<uint32_t>(st->sms) * 4u))), s);
        rc = check_launch();
        if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = CBT_ECUDA;
    }
    if (rc) {
        batch_free(st->self);
        delete st;
        return rc;
    }
    *out = st;
    return CBT_OK;
}

extern "C" int cbt_update(cbt_state* st, const cbt_frame* frame, cbt_stream_t stream) {
    if (!st || !frame) return CBT_EINVAL;
    return batch_update(st->self, frame, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cbt_update_many(cbt_state* const* states, const cbt_frame* frames, int32_t n, cbt_stream_t stream) {
    if (!states || !frames || n < 0) return CBT_EINVAL;
    for (int32_t b = 0; b < n; ++b) {
        const int rc = cbt_update(states[b], frames + b, stream);
        if (rc) return rc;
    }
    return CBT_OK;
}

extern "C" int cbt_live_count(cbt_state* st, uint32_t* h_count, cbt_stream_t stream) {
    if (!st || !h_count) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h_count, st->inst.sums + 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CBT_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_live_count_async(cbt_state* st, uint32_t* count, cbt_stream_t stream) {
    if (!st || !count || (reinterpret_cast<uintptr_t>(count) & 3u)) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return cudaMemcpyAsync(count, st->inst.sums + 1, 4, cudaMemcpyDefault, s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_leaves(cbt_state* st, uint32_t* d_slots, uint64_t* d_heap, uint32_t* d_links,
                          uint32_t cap, uint32_t* h_count, cbt_stream_t stream) {
    uint32_t n = 0;
    int rc = cbt_live_count(st, &n, stream);
    if (rc) return rc;
    if (h_count) *h_count = n;
    if (n > cap) return CBT_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = static_cast<int>(std::max(1u, std::min<uint32_t>((n + 255u) / 256u, static_cast<uint32_t>(st->sms) * 8u)));
    launch_leaves(st->inst, d_slots, d_heap, d_links, grid, s);
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
    cbt_batch* B = st->self;
    FrameP fp;
    std::memset(&fp, 0, sizeof(fp));
    for (int c = 0; c < 3; ++c) fp.eye[c] = h_origin[c];
    fp.precision = precision;
    fp.shift = fixed_shift;
    fp.vout = d_out;
    fp.vcap = cap;
    BatchDev bt = B->dev;
    bt.fps = nullptr;
    bt.fp0 = fp;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    launch_prep(bt, false, grid_prep(B), s);
    launch_vertices(bt, std::max(1, static_cast<int>(std::min<uint32_t>(bt.Titems, static_cast<uint32_t>(st->sms) * 8u))), s);
    rc = check_launch();
    if (rc) return rc;
    return cudaStreamSynchronize(s) == cudaSuccess ? CBT_OK : CBT_ECUDA;
}

extern "C" int cbt_host_device_pointer(void* h_ptr, void** d_ptr) {
    if (!h_ptr || !d_ptr) return CBT_EINVAL;
    *d_ptr = nullptr;
    if (cudaHostGetDevicePointer(d_ptr, h_ptr, 0) != cudaSuccess) {
        cudaGetLastError();  // not page-locked and mapped: clear the error
        return CBT_EINVAL;
    }
    return CBT_OK;
}

extern "C" int cbt_vertices_to_host(cbt_state* st, const float* d_vertices, float* h_vertices, uint32_t cap,
                                    uint32_t* h_count, cbt_stream_t stream) {
    if (!st || !d_vertices || !h_vertices || !h_count) return CBT_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_vertices) | reinterpret_cast<uintptr_t>(h_vertices) |
         reinterpret_cast<uintptr_t>(h_count)) & 3u)
        return CBT_EINVAL;
    void* dv = nullptr;
    void* dc = nullptr;
    if (cbt_host_device_pointer(h_vertices, &dv) || cbt_host_device_pointer(h_count, &dc)) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int rc = launch_rows_to_host(st->inst.sums + 1, d_vertices, static_cast<float*>(dv), cap,
                                       static_cast<uint32_t*>(dc), st->sms, s);
    if (rc) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CBT_ECUDA;
    return *h_count > cap ? CBT_ENOMEM : CBT_OK;
}

extern "C" int cbt_vertices_to_host_async(const float* d_vertices, float* h_vertices, uint32_t rows,
                                          cbt_stream_t stream) {
    if (!d_vertices || !h_vertices) return CBT_EINVAL;
    if (rows == 0u) return CBT_OK;
    return cudaMemcpyAsync(h_vertices, d_vertices, 36ull * rows, cudaMemcpyDeviceToHost,
                           reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? CBT_OK
               : CBT_ECUDA;
}

extern "C" size_t cbt_index_workspace_bytes(const cbt_state* st, uint32_t max_live) {
    return st ? index_workspace_bytes(max_live, st->inst.cap, st->npts) : 0u;
}

extern "C" int cbt_index(cbt_state* st, const float* d_tri_vertices, void* d_workspace, size_t bytes,
                         float* d_vertices, uint32_t vertices_cap, uint32_t* d_indices, uint32_t triangles_cap,
                         uint64_t* d_heap, uint32_t* h_nvertices, uint32_t* h_ntriangles, cbt_stream_t stream) {
    if (!st || !d_workspace || !d_indices || (d_vertices && !d_tri_vertices)) return CBT_EINVAL;
    // the workspace is carved in 256-byte aligned arrays; the outputs are aligned to their element types
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255u) || (reinterpret_cast<uintptr_t>(d_indices) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_heap) & 7u) || (reinterpret_cast<uintptr_t>(d_vertices) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_tri_vertices) & 3u))
        return CBT_EINVAL;
    if (!st->h_ix && cudaMallocHost(reinterpret_cast<void**>(&st->h_ix), 16u) != cudaSuccess) {
        st->h_ix = nullptr;
        return CBT_ECUDA;
    }
    return launch_index(st->inst, st->corner, st->npts, triangles_cap, d_workspace, bytes, d_tri_vertices, d_vertices,
                        vertices_cap, d_indices, d_heap, st->sms, reinterpret_cast<cudaStream_t>(stream), st->h_ix,
                        h_nvertices, h_ntriangles);
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
    if (st->h_ix) cudaFreeHost(st->h_ix);
    batch_free(st->self);
    delete st;
}

extern "C" uint32_t cbt_last_launch_count(const cbt_state* st) { return st ? st->self->launches : 0u; }

namespace {
int set_timing(cbt_batch* B, int on) {
    if (on && !B->timing) {
        for (auto& e : B->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return CBT_ECUDA;
        B->timing = true;
    } else if (!on && B->timing) {
        for (auto& e : B->ev) cudaEventDestroy(e);
        B->timing = false;
        B->timed = 0;
    }
    return CBT_OK;
}
uint32_t kernel_times(cbt_batch* B, float* ms, uint32_t n) {
    if (!B->timing || B->timed == 0 || !ms) return 0u;
    if (B->fused) {
        unsigned long long t[kFramePhases + 1];
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(t, B->dev.bg->t, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return 0u;
        // t[k] opens phase k; the last phase ends at t[kFramePhases] (the
        // latest block end)
        const uint32_t m = std::min(n, B->timed);
        for (uint32_t k = 0; k < m; ++k) {
            const unsigned long long end = k + 1 == B->timed ? t[kFramePhases] : t[k + 1];
            ms[k] = end > t[k] ? static_cast<float>(end - t[k]) * 1e-6f : 0.0f;
        }
        return m;
    }
    if (cudaEventSynchronize(B->ev[B->timed]) != cudaSuccess) return 0u;
    const uint32_t m = std::min(n, B->timed);
    for (uint32_t k = 0; k < m; ++k) {
        ms[k] = 0.0f;
        cudaEventElapsedTime(&ms[k], B->ev[k], B->ev[k + 1]);
    }
    return m;
}
}  // namespace

extern "C" int cbt_set_timing(cbt_state* st, int on) { return st ? set_timing(st->self, on) : CBT_EINVAL; }

extern "C" uint32_t cbt_kernel_times(cbt_state* st, float* ms, uint32_t n) {
    return st ? kernel_times(st->self, ms, n) : 0u;
}

extern "C" const char* cbt_kernel_name(uint32_t k) { return k < kNumKernels ? kKernelNames[k] : ""; }

extern "C" const char* cbt_phase_name(uint32_t k) {
    return k < static_cast<uint32_t>(kFramePhases) ? kPhaseNames[k] : "";
}

extern "C" const char* cbt_state_phase_name(const cbt_state* st, uint32_t k) {
    if (st && st->self->last_frame1) return k < static_cast<uint32_t>(kFrame1Phases) ? kPhaseNames1[k] : "";
    return cbt_phase_name(k);
}

extern "C" int cbt_selftest_bounded_wait(void* d_scratch, int32_t blocks, int32_t limit, cbt_stream_t stream) {
    if (!d_scratch || blocks < 1 || blocks > 64 || limit < 1) return CBT_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_scratch) & 255u) return CBT_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    BatchGlobals* bg = static_cast<BatchGlobals*>(d_scratch);
    if (cudaMemsetAsync(bg, 0, sizeof(BatchGlobals), s) != cudaSuccess) return CBT_ECUDA;
    if (launch_wait_selftest(bg, blocks, limit, s) != cudaSuccess) return CBT_ECUDA;
    uint32_t abort_word = 0;
    if (cudaMemcpyAsync(&abort_word, &bg->abort, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CBT_ECUDA;
    return abort_word ? CBT_ETIMEOUT : CBT_OK;
}

extern "C" int cbt_set_fused(cbt_state* st, int on, cbt_stream_t stream) {
    if (!st) return CBT_EINVAL;
    return set_fused(st->self, on != 0, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cbt_fused(const cbt_state* st) { return st && st->self->fused ? 1 : 0; }

extern "C" int cbt_set_graph(cbt_state* st, int on) {
    if (!st) return CBT_EINVAL;
    st->self->use_graph = on != 0;
    return CBT_OK;
}

// ------------------------------------------------------------------ batches

extern "C" size_t cbt_batch_workspace_bytes(cbt_state* const* states, int32_t n) {
    if (!states || n < 1) return 0u;
    std::vector<uint32_t> cap(n), W(n), H(n);
    for (int32_t b = 0; b < n; ++b) {
        if (!states[b]) return 0u;
        cap[b] = states[b]->inst.cap;
        W[b] = states[b]->inst.W;
        H[b] = states[b]->inst.H;
    }
    return batch_layout(static_cast<uint32_t>(n), cap.data(), W.data(), H.data()).total;
}

extern "C" int cbt_batch_create(cbt_state* const* states, int32_t n, void* workspace, size_t bytes,
                                cbt_stream_t stream, cbt_batch** out) {
    if (!out || !states || n < 1 || !workspace) return CBT_EINVAL;
    *out = nullptr;
    for (int32_t b = 0; b < n; ++b) {
        if (!states[b]) return CBT_EINVAL;
        for (int32_t c = 0; c < b; ++c)
            if (states[c] == states[b]) return CBT_EINVAL;
    }
    if (bytes < cbt_batch_workspace_bytes(states, n) || (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return CBT_ENOMEM;
    return batch_build(states, static_cast<uint32_t>(n), static_cast<char*>(workspace),
                       reinterpret_cast<cudaStream_t>(stream), out);
}

extern "C" int cbt_batch_update(cbt_batch* b, const cbt_frame* frames, cbt_stream_t stream) {
    if (!b || !frames) return CBT_EINVAL;
    return batch_update(b, frames, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cbt_batch_set_graph(cbt_batch* b, int on) {
    if (!b) return CBT_EINVAL;
    b->use_graph = on != 0;
    return CBT_OK;
}

extern "C" int cbt_batch_autotune(cbt_batch* b, uint32_t rounds) {
    if (!b || rounds == 0) return CBT_EINVAL;
    for (auto& e : b->tune_ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) return CBT_ECUDA;
    b->tuning = true;
    b->tune_rounds = rounds;
    b->tune_ms.clear();
    b->tune_pending = false;
    return CBT_OK;
}

extern "C" int cbt_batch_config(const cbt_batch* b, uint32_t* tile_words, uint32_t* blocks_per_sm,
                                int* tuning) {
    if (!b) return CBT_EINVAL;
    if (tile_words) *tile_words = b->tw;
    if (blocks_per_sm) *blocks_per_sm = b->grid_mult;
    if (tuning) *tuning = b->tuning ? 1 : 0;
    return CBT_OK;
}

extern "C" int cbt_batch_set_config(cbt_batch* b, uint32_t tile_words, uint32_t blocks_per_sm,
                                    cbt_stream_t stream) {
    if (!b || (tile_words != 64 && tile_words != 128 && tile_words != 256) || blocks_per_sm < 1 ||
        blocks_per_sm > 64)
        return CBT_EINVAL;
    return apply_config(b, tile_words, blocks_per_sm, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cbt_batch_set_timing(cbt_batch* b, int on) { return b ? set_timing(b, on) : CBT_EINVAL; }

extern "C" int cbt_batch_set_fused(cbt_batch* b, int on, cbt_stream_t stream) {
    if (!b) return CBT_EINVAL;
    return set_fused(b, on != 0, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int cbt_batch_fused(const cbt_batch* b) { return b && b->fused ? 1 : 0; }

extern "C" uint32_t cbt_batch_kernel_times(cbt_batch* b, float* ms, uint32_t n) {
    return b ? kernel_times(b, ms, n) : 0u;
}

extern "C" uint32_t cbt_batch_last_launch_count(const cbt_batch* b) { return b ? b->launches : 0u; }

extern "C" void cbt_batch_destroy(cbt_batch* b) { batch_free(b); }

// ------------------------------------------------------------------ server

namespace {

// One in-flight tick: a device region holding the tick's packed instance
// table, frame parameters and prefixes, the launch counters, the tile
// prefix, live-count output and look-back descriptors; its pinned host twin.
struct ServerSlot {
    char* dev = nullptr;
    char* host = nullptr;  // pinned: packed tick block, then live counts
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<int32_t> idx;
};

struct TickLayout {
    size_t inst, fps, wbase, vbase, rbase, block;         // packed block (copied per tick)
    size_t bg, tile_base, ctile_base, stile_base, nout, status, total;  // rest of the device region
};

TickLayout tick_layout(uint32_t k, uint32_t n_max, uint32_t status_words) {
    TickLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.inst = take(sizeof(Inst) * k);
    L.fps = take(sizeof(FrameP) * k);
    L.wbase = take(4u * (k + 1u));
    L.vbase = take(4u * (k + 1u));
    L.rbase = take(4u * (k + 1u));
    L.block = off;
    // the fixed part is laid out for the largest tick so that its offsets
    // do not move between ticks
    size_t moff = 0;
    auto mtake = [&](size_t bytes) {
        const size_t o = moff;
        moff = align256(moff + bytes);
        return o;
    };
    mtake(sizeof(Inst) * n_max);
    mtake(sizeof(FrameP) * n_max);
    mtake(4u * (n_max + 1u));
    mtake(4u * (n_max + 1u));
    mtake(4u * (n_max + 1u));
    L.bg = mtake(sizeof(BatchGlobals));
    L.tile_base = mtake(4u * (n_max + 1u));
    L.ctile_base = mtake(4u * (n_max + 1u));
    L.stile_base = mtake(4u * (n_max + 1u));
    L.nout = mtake(4u * n_max);
    L.status = mtake(8u * static_cast<size_t>(status_words));
    L.total = moff;
    return L;
}

}  // namespace

struct cbt_server {
    std::vector<cbt_state*> st;
    std::vector<int32_t> inflight;  // slot of each instance's pending tick, or -1
    uint32_t n = 0;
    int sms = 1;
    uint32_t status_words = 0;
    size_t slot_bytes = 0;
    uint32_t tw = 256, grid_mult = 8;
    bool fused = false;  // ticks as one cooperative launch each, one at a time on the device
    int frame_per_sm = 0;
    std::vector<ServerSlot> slots;
    uint32_t next = 0;
    bool any_tick = false;
};

extern "C" size_t cbt_server_workspace_bytes(cbt_state* const* states, int32_t n, int32_t inflight) {
    if (!states || n < 1 || inflight < 1 || inflight > 16) return 0u;
    uint64_t titems = 0, twords = 0;
    for (int32_t b = 0; b < n; ++b) {
        if (!states[b]) return 0u;
        titems += item_tiles(states[b]->inst.cap);
        twords += word_tiles(states[b]->inst.W, kMinTileWords);
    }
    const TickLayout L = tick_layout(static_cast<uint32_t>(n), static_cast<uint32_t>(n),
                                     static_cast<uint32_t>(2u * titems + twords));
    return L.total * static_cast<size_t>(inflight);
}

extern "C" int cbt_server_create(cbt_state* const* states, int32_t n, int32_t inflight, void* workspace,
                                 size_t bytes, cbt_server** out) {
    if (!out || !states || n < 1 || inflight < 1 || inflight > 16 || !workspace) return CBT_EINVAL;
    *out = nullptr;
    const size_t need = cbt_server_workspace_bytes(states, n, inflight);
    if (need == 0u) return CBT_EINVAL;
    if (bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return CBT_ENOMEM;
    cbt_server* sv = new cbt_server();
    sv->st.assign(states, states + n);
    sv->inflight.assign(static_cast<size_t>(n), -1);
    sv->n = static_cast<uint32_t>(n);
    sv->sms = states[0]->sms;
    uint64_t titems = 0, twords = 0;
    for (int32_t b = 0; b < n; ++b) {
        titems += item_tiles(states[b]->inst.cap);
        twords += word_tiles(states[b]->inst.W, kMinTileWords);
    }
    sv->status_words = static_cast<uint32_t>(2u * titems + twords);
    const TickLayout L = tick_layout(sv->n, sv->n, sv->status_words);
    sv->slot_bytes = L.total;
    sv->slots.resize(static_cast<size_t>(inflight));
    int rc = CBT_OK;
    for (int32_t r = 0; r < inflight && !rc; ++r) {
        ServerSlot& S = sv->slots[r];
        S.dev = static_cast<char*>(workspace) + L.total * static_cast<size_t>(r);
        if (cudaMallocHost(reinterpret_cast<void**>(&S.host), L.block + 4u * sv->n) != cudaSuccess ||
            cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMemset(S.dev + L.bg, 0, sizeof(BatchGlobals)) != cudaSuccess)  // grid-barrier counters
            rc = CBT_ECUDA;
    }
    sv->frame_per_sm = frame_blocks_per_sm();
    if (!rc && sv->frame_per_sm <= 0) rc = CBT_ECUDA;
    if (rc) {
        for (auto& S : sv->slots) {
            if (S.host) cudaFreeHost(S.host);
            if (S.done) cudaEventDestroy(S.done);
        }
        delete sv;
        return rc;
    }
    *out = sv;
    return CBT_OK;
}

extern "C" int cbt_server_submit(cbt_server* sv, const int32_t* idx, const cbt_frame* frames, int32_t k,
                                 cbt_stream_t stream, int32_t* ticket) {
    if (!sv || !idx || !frames || k < 1 || static_cast<uint32_t>(k) > sv->n || !ticket) return CBT_EINVAL;
    for (int32_t i = 0; i < k; ++i) {
        if (idx[i] < 0 || static_cast<uint32_t>(idx[i]) >= sv->n) return CBT_EINVAL;
        if (sv->inflight[idx[i]] >= 0) return CBT_EINVAL;  // one pending tick per instance
        for (int32_t j = 0; j < i; ++j)
            if (idx[j] == idx[i]) return CBT_EINVAL;
    }
    const uint32_t r = sv->next;
    ServerSlot& S = sv->slots[r];
    if (S.busy) return CBT_EINVAL;  // poll the slot's previous ticket first
    const uint32_t kk = static_cast<uint32_t>(k);
    const TickLayout L = tick_layout(kk, sv->n, sv->status_words);
    Inst* hi = reinterpret_cast<Inst*>(S.host + L.inst);
    FrameP* hf = reinterpret_cast<FrameP*>(S.host + L.fps);
    uint32_t* hw = reinterpret_cast<uint32_t*>(S.host + L.wbase);
    uint32_t* hv = reinterpret_cast<uint32_t*>(S.host + L.vbase);
    uint32_t* hr = reinterpret_cast<uint32_t*>(S.host + L.rbase);
    hw[0] = hv[0] = hr[0] = 0;
    bool vertices = false;
    for (uint32_t i = 0; i < kk; ++i) {
        cbt_state* st = sv->st[idx[i]];
        hi[i] = st->inst;
        if (!frame_from_api(frames + i, st->frame, hf[i])) return CBT_EINVAL;
        vertices = vertices || hf[i].vout != nullptr;
        hw[i + 1] = hw[i] + word_tiles(st->inst.W, sv->tw);
        hv[i + 1] = hv[i] + item_tiles(st->inst.cap);
        hr[i + 1] = hr[i] + 9u * st->inst.H;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // a fused tick starts after the previous tick (two cooperative launches
    // are never in flight together)
    if (sv->fused && sv->any_tick) {
        const uint32_t prev = (r + static_cast<uint32_t>(sv->slots.size()) - 1u) % static_cast<uint32_t>(sv->slots.size());
        if (cudaStreamWaitEvent(s, sv->slots[prev].done, 0) != cudaSuccess) return CBT_ECUDA;
    }
    if (cudaMemcpyAsync(S.dev, S.host, L.block, cudaMemcpyHostToDevice, s) != cudaSuccess) return CBT_ECUDA;
    BatchDev bt{};
    bt.inst = reinterpret_cast<const Inst*>(S.dev + L.inst);
    bt.fps = reinterpret_cast<const FrameP*>(S.dev + L.fps);
    bt.B = kk;
    bt.tw = sv->tw;
    bt.tile_base = reinterpret_cast<uint32_t*>(S.dev + L.tile_base);
    bt.ctile_base = reinterpret_cast<uint32_t*>(S.dev + L.ctile_base);
    bt.stile_base = reinterpret_cast<uint32_t*>(S.dev + L.stile_base);
    bt.wtile_base = reinterpret_cast<const uint32_t*>(S.dev + L.wbase);
    bt.vtile_base = reinterpret_cast<const uint32_t*>(S.dev + L.vbase);
    bt.rel_base = reinterpret_cast<const uint32_t*>(S.dev + L.rbase);
    bt.bg = reinterpret_cast<BatchGlobals*>(S.dev + L.bg);
    bt.status = reinterpret_cast<unsigned long long*>(S.dev + L.status);
    bt.Titems = hv[kk];
    bt.Twords = hw[kk];
    bt.Trel = hr[kk];
    bt.nout = reinterpret_cast<uint32_t*>(S.dev + L.nout);
    if (sv->fused) {
        const uint32_t work = std::max({bt.Titems, bt.Twords, (bt.Trel + 255u) / 256u, 1u});
        const uint32_t grid = std::min(work, static_cast<uint32_t>(sv->frame_per_sm * sv->sms));
        if (launch_frame(bt, static_cast<int>(grid), s) != cudaSuccess) return CBT_ECUDA;
    } else {
        enqueue_kernels(bt, sv->sms, sv->grid_mult, vertices, s, nullptr);
    }
    cudaMemcpyAsync(S.host + L.block, bt.nout, 4u * kk, cudaMemcpyDeviceToHost, s);
    if (cudaEventRecord(S.done, s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return CBT_ECUDA;
    S.busy = true;
    S.idx.assign(idx, idx + k);
    for (uint32_t i = 0; i < kk; ++i) {
        sv->inflight[idx[i]] = static_cast<int32_t>(r);
        sv->st[idx[i]]->frame += 1u;
    }
    sv->next = (r + 1u) % static_cast<uint32_t>(sv->slots.size());
    sv->any_tick = true;
    *ticket = static_cast<int32_t>(r);
    return CBT_OK;
}

extern "C" int cbt_server_set_fused(cbt_server* sv, int on) {
    if (!sv) return CBT_EINVAL;
    for (const auto& S : sv->slots)
        if (S.busy) return CBT_EINVAL;  // switch between ticks only
    sv->fused = on != 0;
    sv->tw = sv->fused ? kFusedTileWords : 256u;
    return CBT_OK;
}

extern "C" int cbt_server_poll(cbt_server* sv, int32_t ticket, int wait, uint32_t* live_before) {
    if (!sv || ticket < 0 || static_cast<size_t>(ticket) >= sv->slots.size()) return -CBT_EINVAL;
    ServerSlot& S = sv->slots[ticket];
    if (!S.busy) return -CBT_EINVAL;
    const cudaError_t e = wait ? cudaEventSynchronize(S.done) : cudaEventQuery(S.done);
    if (e == cudaErrorNotReady) return 0;
    if (e != cudaSuccess) return -CBT_ECUDA;
    const TickLayout L = tick_layout(static_cast<uint32_t>(S.idx.size()), sv->n, sv->status_words);
    if (live_before) std::memcpy(live_before, S.host + L.block, 4u * S.idx.size());
    for (int32_t b : S.idx) sv->inflight[b] = -1;
    S.idx.clear();
    S.busy = false;
    return 1;
}

extern "C" int32_t cbt_server_next_slot_free(const cbt_server* sv) {
    return sv && !sv->slots[sv->next].busy ? 1 : 0;
}

extern "C" void cbt_server_destroy(cbt_server* sv) {
    if (!sv) return;
    for (auto& S : sv->slots) {
        if (S.busy) cudaEventSynchronize(S.done);
        if (S.host) cudaFreeHost(S.host);
        if (S.done) cudaEventDestroy(S.done);
    }
    delete sv;
}
