// api.cu -- libhgm host runtime behind the C ABI of include/hgm.h.
//
// Handles keep models and scenes resident in device memory (Sec. 3.6: data
// stays on the GPU across launches), stably sorted by frame with the minnode
// table of Sec. 3.4. A match call plans units (model, scene, offset), orders
// them by decreasing model size (longest-processing-time first, so that the
// persistent recursion kernel ends with short units), and runs
//   (a) unary table -> candidate selection -> (b) recursion -> (c) backtrack
// per chunk of units whose argmin tables fit the workspace budget. Nothing
// crosses the host/device boundary between the kernels; the paper's host
// loop over i (Alg. 2) is inside kernel (b).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hgm_internal.cuh"
#include "prop.cuh"

namespace hgm {
namespace {

constexpr uint32_t kDeadMagic = 0xdeadbeefu;

thread_local std::string g_err;
std::mutex g_mu;

hgm_status fail(hgm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

hgm_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(HGM_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(HGM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copies n elements from a host-or-device pointer into a host vector.
template <typename T>
hgm_status fetch(const T *src, size_t n, std::vector<T> &dst, cudaStream_t st)
{
    dst.resize(n);
    if (n == 0) return HGM_OK;
    if (is_device_ptr(src)) {
        CK(cudaMemcpyAsync(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, st), "copy input to host");
        CK(cudaStreamSynchronize(st), "synchronise input copy");
    } else {
        std::memcpy(dst.data(), src, n * sizeof(T));
    }
    return HGM_OK;
}

template <typename T>
hgm_status upload(T **dptr, const std::vector<T> &h, cudaStream_t st)
{
    size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
    CK(cudaMalloc((void **)dptr, bytes), "cudaMalloc");
    if (!h.empty()) CK(cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
    return HGM_OK;
}

int round_up4(int v) { return (v + 3) & ~3; }


// ---- profiling --------------------------------------------------------------
struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
};
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
std::vector<cudaEvent_t> g_prof_free;
double g_prof_ms[kProfCount];
int64_t g_prof_n[kProfCount];
std::mutex g_prof_mu;
ProfRec g_prof_open[kProfCount];
bool g_prof_is_open[kProfCount];

cudaEvent_t prof_event()
{
    if (!g_prof_free.empty()) {
        cudaEvent_t e = g_prof_free.back();
        g_prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// ---- workspace ------------------------------------------------------------------
bool g_capturing = false;   // a plan's launch sequence is being recorded: no allocation, no events

struct Buffer {
    void *p = nullptr;
    size_t bytes = 0;
    Buffer() = default;
    Buffer(const Buffer &) = delete;
    Buffer &operator=(const Buffer &) = delete;
    ~Buffer() { if (p) cudaFree(p); }
    cudaError_t ensure(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        if (g_capturing) return cudaErrorStreamCaptureUnsupported;   // sizes were fixed by the sizing pass
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t sz = std::max<size_t>(need, 256);
        cudaError_t e = cudaMalloc(&p, sz);
        if (e == cudaSuccess) bytes = sz;
        return e;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

struct Workspace {
    Buffer modelcat, U, cand_idx, cand_u, cand_cnt, beta, units, res, mrec, srec, counter, out_e, out_a, evaluated;
    Buffer mnorm, snorm, status;
    Buffer stage, perm_stage, flag;   // inputs of hgm_create_model / hgm_create_scene
    Buffer P, Pb, Q, Qb, modelxy, cand2_idx, cand2_u, cand2_cnt, units2, beta2, fb_units, fb_count, beta_fb, scores;
    Buffer fb_total;   // fallback units since the last hgm_prune_counters reset (device counter)
    Buffer chain_e, chain_a, chain_tab, chain_oe, chain_oa;   // independent-chains variant
    Buffer rf_e, rf_a;        // refinement of the pruned form: device outputs when the caller's are on the host
    Buffer ubf;               // precision mode: BF16 copies of the unary table's operands (TMA-staged kernel)
    Buffer beta_dummy;        // per-CTA argmin tables of the dummy-assignment recursion
};

// Buffers of the whole-block form: band tables, model rows, unary table, argmin tables, records, outputs.
struct BlockBufs {
    Buffer tab, cellb, dir, model, mrec, U, beta, scratch, oe, oa;
    int R = 0;                  // model rows gathered into `model` (prep_block_models)
    std::vector<int> urow;
    bool own_pinned = false;    // stream objects: upload the tables from a pinned staging buffer
    void *pinned = nullptr;
    size_t pinned_bytes = 0;
    cudaEvent_t upload_done = nullptr;   // the last upload from `pinned` (it is rewritten after this)
    ~BlockBufs()
    {
        if (pinned) cudaFreeHost(pinned);
        if (upload_done) cudaEventDestroy(upload_done);
    }
};
Workspace g_ws;
BlockBufs g_blk;

// Calls on different streams share g_ws / g_blk: each call's work waits for the previous call's (on whatever
// stream it ran), so a call with device outputs may return before its work finishes without racing the next.
cudaEvent_t g_ws_event = nullptr;
struct WsGuard {
    cudaStream_t st;
    explicit WsGuard(cudaStream_t s) : st(s)
    {
        if (g_ws_event) cudaStreamWaitEvent(st, g_ws_event, 0);
    }
    ~WsGuard()
    {
        if (!g_ws_event && cudaEventCreateWithFlags(&g_ws_event, cudaEventDisableTiming) != cudaSuccess) {
            g_ws_event = nullptr;
            return;
        }
        cudaEventRecord(g_ws_event, st);
    }
};
}  // namespace
}  // namespace hgm

// A stream of scene blocks matched against fixed models (hgm_stream_*).
struct hgm_stream {
    uint32_t magic;
    std::vector<const hgm_model *> models;
    hgm_params params;
    int32_t block_frames, F_user, Fp;
    int32_t max_points;                // capacity: points of one block (every buffer is sized for it at creation)
    hgm::BlockBufs bb;
    hgm::Buffer sc_buf, raw;           // the block's sorted points (xy | t | perm | minnode), raw descriptors
    hgm::Buffer f;                     // sorted, padded descriptors
    hgm::Buffer flag;
    hgm::Buffer dev_e, dev_a;     // results before the read-back (host outputs)
    void *pin_out = nullptr;      // pinned read-back of energies, assignments and the flag
    size_t pin_out_bytes = 0;
    void *pinned = nullptr;       // host staging of the uploads
    size_t pinned_bytes = 0;
    hgm_scene view;               // the current block as a scene (device arrays owned by this object)
};

namespace hgm {
namespace {
constexpr uint32_t kStreamMagic = 0x5354524du;   // "STRM"

bool valid_stream(const hgm_stream *s) { return s && s->magic == kStreamMagic; }

void free_stream(hgm_stream *s)
{
    if (s->pinned) cudaFreeHost(s->pinned);
    s->pinned = nullptr;
    if (s->pin_out) cudaFreeHost(s->pin_out);
    s->pin_out = nullptr;
}

bool g_count_mode = false;   // hgm_profile_enable(2): batch runs use the accounting recursion variant
size_t g_budget_override = 0;   // hgm_set_workspace_budget: bytes for the unary table and for a chunk (0 = auto)
int64_t g_pruned_units = 0;
int64_t g_refined_units = 0;   // units solved again by the refinement of the pruned form

// How run_batch issues its work: on the shared workspace (ordinary calls), or for a plan on the plan's own
// workspace, first as a sizing pass (grows the workspace, keeps a pinned copy of every host upload) and then
// as the recorded pass (no allocation, no host synchronisation, uploads from those pinned copies).
struct Exec {
    enum Mode { kNormal, kSizing, kCapture } mode = kNormal;
    Workspace *ws = &g_ws;
    size_t budget = 0;                                    // workspace budget fixed by the sizing pass
    std::vector<std::pair<void *, size_t>> *pinned = nullptr;
    size_t pin_next = 0;
    int64_t pruned_units = 0;                             // units of the pruned pass issued
    bool tensor = false;                                  // a tensor-core kernel ran (status flag is live)
    const std::vector<uint8_t> *select = nullptr;         // if set: only the units whose energy index is marked
    int64_t refined_units = 0;                            // units solved again by the refinement
};

hgm_status h2d(Exec &ex, void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!bytes) return HGM_OK;
    if (ex.mode == Exec::kSizing) {
        void *h = nullptr;
        CK(cudaMallocHost(&h, bytes), "pinned staging");
        ex.pinned->emplace_back(h, bytes);
    }
    if (ex.mode != Exec::kNormal) {
        if (ex.pin_next >= ex.pinned->size() || (*ex.pinned)[ex.pin_next].second != bytes)
            return fail(HGM_ECUDA, "plan: upload sequence differs between the sizing and the recorded pass");
        void *h = (*ex.pinned)[ex.pin_next++].first;
        std::memcpy(h, src, bytes);
        src = h;
    }
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "upload");
    return HGM_OK;
}

// dst[k][c] = src[perm[k]][c] for c < F, 0 for F <= c < Fp; flags a non-finite component.
__global__ void gather_rows_kernel(const float *__restrict__ src, int F, const int32_t *__restrict__ perm, int64_t n,
                                   int Fp, float *__restrict__ dst, int *__restrict__ bad)
{
    const int64_t total = n * Fp;
    int nonfinite = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / Fp;
        const int c = (int)(e - k * Fp);
        float v = 0.0f;
        if (c < F) {
            v = src[(int64_t)perm[k] * F + c];
            nonfinite |= !isfinite(v);
        }
        dst[e] = v;
    }
    if (nonfinite) atomicOr(bad, 1);
}

// Sorted, padded device copy of a descriptor array (host or device, n x F row-major): the raw rows go to the
// device in one copy (none for device input), then a gather kernel applies the permutation. Returns
// HGM_EINVAL on a non-finite component. Synchronous on st.
hgm_status upload_sorted_rows(const float *src, int64_t n, int F, int Fp, const std::vector<int32_t> &perm,
                              float **dst, const char *what, cudaStream_t st)
{
    const size_t bytes = (size_t)std::max<int64_t>(n * Fp, 1) * sizeof(float);
    CK(cudaMalloc((void **)dst, bytes), "cudaMalloc");
    if (n == 0) return HGM_OK;
    const float *dsrc = src;
    if (!is_device_ptr(src)) {
        CK(g_ws.stage.ensure((size_t)n * F * sizeof(float)), "workspace (input staging)");
        CK(cudaMemcpyAsync(g_ws.stage.p, src, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice, st),
           "upload descriptors");
        dsrc = g_ws.stage.as<float>();
    }
    CK(g_ws.perm_stage.ensure((size_t)n * sizeof(int32_t)), "workspace (input staging)");
    CK(cudaMemcpyAsync(g_ws.perm_stage.p, perm.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st),
       "upload permutation");
    CK(g_ws.flag.ensure(sizeof(int)), "workspace");
    CK(cudaMemsetAsync(g_ws.flag.p, 0, sizeof(int), st), "memset");
    const int64_t blocks = std::min<int64_t>((n * Fp + 255) / 256, 65536);
    gather_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(dsrc, F, g_ws.perm_stage.as<int32_t>(), n, Fp, *dst,
                                                         g_ws.flag.as<int>());
    CK(cudaGetLastError(), "gather kernel");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, g_ws.flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
    CK(cudaStreamSynchronize(st), "synchronise");
    if (bad) return fail(HGM_EINVAL, "non-finite %s descriptor", what);
    return HGM_OK;
}

}  // namespace

// Profiling hooks used by the kernel launchers.
// NVTX ranges (host-side launch spans) of the pipeline stages, for timeline tools
static const char *const kStageNames[kProfCount] = {"hgm: unary", "hgm: select", "hgm: recursion",
                                                    "hgm: backtrack", "hgm: pruning"};

void prof_begin(int kernel, cudaStream_t st)
{
    nvtxRangePushA(kStageNames[kernel]);
    if (!g_prof_on || g_capturing) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{kernel, prof_event(), prof_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    g_prof_open[kernel] = r;
    g_prof_is_open[kernel] = true;
}

void prof_end(int kernel, cudaStream_t st)
{
    nvtxRangePop();
    if (!g_prof_on || g_capturing) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_is_open[kernel]) return;
    ProfRec r = g_prof_open[kernel];
    g_prof_is_open[kernel] = false;
    cudaEventRecord(r.b, st);
    g_prof_pending.push_back(r);
}

}  // namespace hgm

using namespace hgm;

namespace hgm {
// Error reporting for other translation units of the library.
hgm_status set_error(hgm_status s, const char *msg)
{
    g_err = msg;
    return s;
}
bool valid_model(const hgm_model *m) { return m && m->magic == kModelMagic; }
bool valid_scene(const hgm_scene *s) { return s && s->magic == kSceneMagic; }
}  // namespace hgm

namespace {

hgm_status check_params(const hgm_params *p)
{
    if (!p) return fail(HGM_EINVAL, "params is NULL");
    if (!(std::isfinite(p->lambda1) && std::isfinite(p->lambda2) && std::isfinite(p->lambda3)) ||
        p->lambda1 < 0 || p->lambda2 < 0 || p->lambda3 < 0)
        return fail(HGM_EINVAL, "lambdas must be finite and >= 0");
    if (p->window < 0) return fail(HGM_EINVAL, "window must be >= 0");
    if (p->K < 1 || p->K > 255) return fail(HGM_EINVAL, "K must be in 1..255 (got %d)", p->K);
    if (p->K > kMaxK) return fail(HGM_EUNSUPPORTED, "K > %d is not supported by this library", kMaxK);
    if (p->precision != 0 && p->precision != 1)
        return fail(HGM_EUNSUPPORTED, "precision %d not available (0 = FP32 exact, 1 = BF16 + FP32 re-score)",
                    p->precision);
    if (p->offset_lo > p->offset_hi) return fail(HGM_EINVAL, "offset_lo > offset_hi");
    if (std::isnan(p->dummy_cost) || std::isinf(p->dummy_cost))
        return fail(HGM_EINVAL, "dummy_cost must be finite (< 0 for none)");
    if (p->dummy_cost >= 0 && p->prune)
        return fail(HGM_EUNSUPPORTED, "the dummy assignment is not available with pruning");
    if (p->prune) {
        if (p->prune->magic != kPropMagic) return fail(HGM_EINVAL, "prune is not a proposal-network handle");
        if (p->keep < 1 || p->keep > p->K) return fail(HGM_EINVAL, "keep must be in 1..K (got %d)", p->keep);
        if (p->refine < 0 || p->refine > 65535)
            return fail(HGM_EINVAL, "refine must be in 0..65535 (got %d)", p->refine);
    }
    return HGM_OK;
}

Params to_params(const hgm_params *p)
{
    Params q;
    q.lambda1 = p->lambda1;
    q.lambda2 = p->lambda2;
    q.lambda3 = p->lambda3;
    q.T = p->T;
    q.window = p->window;
    q.K = p->K;
    q.rescore = p->precision == 1 ? kRescore : 0;
    q.dummy = p->dummy_cost >= 0 ? p->dummy_cost : -1.0f;
    return q;
}

// Offset range of a pair: o in [-t_1, F_s-1-t_M] intersected with [offset_lo, offset_hi].
void pair_offsets(const hgm_model *m, const hgm_scene *s, const hgm_params *p, int32_t *n, int32_t *first)
{
    int64_t t1 = m->span_t1, tM = m->span_tM;
    int64_t lo = -t1, hi = (int64_t)s->d.n_frames - 1 - tM;
    lo = std::max<int64_t>(lo, p->offset_lo);
    hi = std::min<int64_t>(hi, p->offset_hi);
    *first = (int32_t)lo;
    *n = hi >= lo ? (int32_t)(hi - lo + 1) : 0;
}

hgm_status sort_points(const std::vector<int32_t> &t, std::vector<int32_t> &perm)
{
    perm.resize(t.size());
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return t[a] < t[b]; });
    return HGM_OK;
}

void free_model(hgm_model *m)
{
    for (hgm_model *c : m->chains) {
        free_model(c);
        delete c;
    }
    m->chains.clear();
    m->chain_n = 0;
    cudaFree(m->d.xy);
    cudaFree(m->d.t);
    cudaFree(m->d.f);
    cudaFree(m->d.perm);
    cudaFree(m->d.geo);
}

void free_scene(hgm_scene *s)
{
    cudaFree(s->d.xy);
    cudaFree(s->d.t);
    cudaFree(s->d.f);
    cudaFree(s->d.frame_start);
    cudaFree(s->d.perm);
}

// Staged inputs of one batch call.
struct Plan {
    std::vector<ModelRec> mrec;
    std::vector<SceneRec> srec;
    std::vector<int32_t> first;       // per pair
    std::vector<int64_t> e_start;     // per pair + 1
    std::vector<int64_t> a_start;     // per pair + 1
    int R = 0;                        // model rows in the unary table
    int max_M = 0;
};

hgm_status build_plan(const hgm_model *const *models, int nm, const hgm_scene *const *scenes, int ns,
                      const hgm_params *p, Plan &pl)
{
    pl.first.assign((size_t)nm * ns, 0);
    pl.e_start.assign((size_t)nm * ns + 1, 0);
    pl.a_start.assign((size_t)nm * ns + 1, 0);
    int F = -1;
    for (int m = 0; m < nm; ++m) {
        if (!valid_model(models[m])) return fail(HGM_EINVAL, "models[%d] is not a model handle", m);
        if (F < 0) F = models[m]->F_user;
        if (models[m]->F_user != F) return fail(HGM_EINVAL, "descriptor widths differ across models");
    }
    for (int s = 0; s < ns; ++s) {
        if (!valid_scene(scenes[s])) return fail(HGM_EINVAL, "scenes[%d] is not a scene handle", s);
        if (F >= 0 && scenes[s]->F_user != F) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    }
    for (int m = 0; m < nm; ++m)
        for (int s = 0; s < ns; ++s) {
            size_t q = (size_t)m * ns + s;
            int32_t n, first;
            pair_offsets(models[m], scenes[s], p, &n, &first);
            pl.first[q] = first;
            pl.e_start[q + 1] = pl.e_start[q] + n;
            pl.a_start[q + 1] = pl.a_start[q] + (int64_t)n * models[m]->d.M;
        }
    return HGM_OK;
}

// Runs a list of units (one segment group): chunks bounded by the budget for candidate lists and
// argmin tables; per chunk selection -> (pruning ->) recursion -> backtrack (-> fallback).
hgm_status run_units(Exec &ex, const hgm_model *const *models, std::vector<Unit> &all, int max_M, int K, int keep,
                     bool pruning, const Params &p, const PropInfer &pi, cudaStream_t st, float *d_energy,
                     int32_t *d_assign, size_t budget)
{
    Workspace &ws = *ex.ws;
    const int64_t n_units = (int64_t)all.size();
    hgm_status rc;
    int64_t begin = 0;
    while (begin < n_units) {
        int64_t cand_e = 0, beta_b = 0, end = begin;
        while (end < n_units) {
            const int M = models[all[(size_t)end].model]->d.M;
            int64_t ce = (int64_t)M * K, bb = (int64_t)(M - 2) * K * K;
            const int64_t bb_need = pruning ? (int64_t)(M - 2) * keep * keep : bb;
            const int64_t need = (cand_e + ce) * (int64_t)(sizeof(int32_t) * 2) + (cand_e + ce) / K * 4 +
                                 (beta_b + bb) / (K * K) * (bb_need / std::max<int64_t>(M - 2, 1));
            if (end > begin && (size_t)need > budget) break;
            all[(size_t)end].cand = cand_e;
            all[(size_t)end].beta = beta_b;
            cand_e += ce;
            beta_b += bb;
            ++end;
        }
        const int64_t n = end - begin;
        CK(ws.cand_idx.ensure((size_t)cand_e * sizeof(int32_t)), "workspace (candidates)");
        CK(ws.cand_u.ensure((size_t)cand_e * sizeof(float)), "workspace (candidates)");
        CK(ws.cand_cnt.ensure((size_t)(cand_e / K) * sizeof(int32_t)), "workspace (candidates)");
        if (!pruning && p.dummy < 0) CK(ws.beta.ensure((size_t)beta_b), "workspace (argmin tables)");
        CK(ws.units.ensure((size_t)n * sizeof(Unit)), "workspace (units)");
        CK(ws.res.ensure((size_t)n * sizeof(UnitResult)), "workspace (results)");
        CK(ws.counter.ensure(sizeof(int)), "workspace");
        if ((rc = h2d(ex, ws.units.p, all.data() + begin, (size_t)n * sizeof(Unit), st))) return rc;
        const Unit *du = ws.units.as<Unit>();
        const ModelRec *dm = ws.mrec.as<ModelRec>();
        const SceneRec *ds = ws.srec.as<SceneRec>();
        CK(launch_select(du, n, dm, ds, p, max_M, ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(),
                         ws.cand_cnt.as<int32_t>(), st),
           "select kernel");
        if (pruning) {
            const int64_t n_lists = cand_e / K;
            CK(ws.cand2_idx.ensure((size_t)n_lists * keep * sizeof(int32_t)), "workspace (pruned lists)");
            CK(ws.cand2_u.ensure((size_t)n_lists * keep * sizeof(float)), "workspace (pruned lists)");
            CK(ws.cand2_cnt.ensure((size_t)n_lists * sizeof(int32_t)), "workspace (pruned lists)");
            CK(ws.units2.ensure((size_t)n * sizeof(Unit)), "workspace (units)");
            CK(ws.beta2.ensure((size_t)(beta_b / ((int64_t)K * K) * keep * keep) + 1), "workspace (argmin tables)");
            CK(ws.scores.ensure((size_t)cand_e * sizeof(float)), "workspace (scores)");
            CK(launch_prop_prune(du, n, dm, ds, p, pi, ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(),
                                 ws.cand_cnt.as<int32_t>(), ws.scores.as<float>(), ws.cand2_idx.as<int32_t>(),
                                 ws.cand2_u.as<float>(), ws.cand2_cnt.as<int32_t>(), ws.status.as<int>(), st),
               "pruning kernels");
            CK(launch_derive_units(du, n, K, keep, ws.units2.as<Unit>(), st), "derive units");
            Params pk = p;
            pk.K = keep;
            pk.rescore = 0;
            const Unit *du2 = ws.units2.as<Unit>();
            CK(launch_recurse(du2, n, dm, ds, pk, ws.cand2_idx.as<int32_t>(), ws.cand2_u.as<float>(),
                              ws.cand2_cnt.as<int32_t>(), ws.beta2.as<uint8_t>(), ws.res.as<UnitResult>(),
                              ws.counter.as<int>(), st),
               "recursion kernel (pruned lists)");
            CK(launch_backtrack(du2, n, dm, ds, pk, ws.cand2_idx.as<int32_t>(), ws.beta2.as<uint8_t>(),
                                ws.res.as<UnitResult>(), d_energy, d_assign, st),
               "backtrack kernel (pruned lists)");
            // fallback: units whose pruned optimum is infeasible are solved again on the full lists, by the
            // fused recursion + backtrack reading their number on the device (no host round trip)
            CK(ws.fb_units.ensure((size_t)n * sizeof(Unit)), "workspace (fallback)");
            CK(ws.fb_count.ensure(sizeof(int)), "workspace");
            CK(cudaMemsetAsync(ws.fb_count.p, 0, sizeof(int), st), "memset");
            CK(launch_collect_infeasible(ws.res.as<UnitResult>(), du, n, ws.fb_units.as<Unit>(),
                                         ws.fb_count.as<int>(), g_ws.fb_total.as<unsigned long long>(), st),
               "collect infeasible");
            const int64_t scratch = recurse_fused_scratch(K, max_M);
            if (scratch < 0) return fail(HGM_ECUDA, "device query failed");
            CK(ws.beta_fb.ensure((size_t)scratch), "workspace (fallback)");
            if (pi.rescore)   // precision mode: the fallback solves full lists, their costs in FP32
                CK(launch_rescore_units(ws.fb_units.as<Unit>(), n, ws.fb_count.as<int>(), dm, ds, p,
                                        ws.cand_idx.as<int32_t>(), ws.cand_cnt.as<int32_t>(), ws.cand_u.as<float>(),
                                        st),
                   "re-score kernel (fallback)");
            CK(launch_recurse_fused(ws.fb_units.as<Unit>(), n, ws.fb_count.as<int>(), dm, ds, p,
                                    ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(), ws.cand_cnt.as<int32_t>(),
                                    ws.beta_fb.as<uint8_t>(), max_M, d_energy, d_assign, ws.counter.as<int>(), st),
               "recursion kernel (fallback)");
            ex.pruned_units += n;
            begin = end;
            continue;
        }
        if (p.dummy >= 0) {
            // the dummy assignment: its own recursion kernel, which also backtracks
            const int grid = dummy_grid();
            if (grid <= 0) return fail(HGM_ECUDA, "device query failed");
            CK(ws.beta_dummy.ensure((size_t)dummy_scratch_bytes(K, max_M, grid)), "workspace (argmin tables)");
            unsigned long long *ev = nullptr;
            if (g_count_mode && ex.mode == Exec::kNormal) {
                CK(ws.evaluated.ensure(sizeof(unsigned long long)), "workspace");
                ev = ws.evaluated.as<unsigned long long>();
            }
            CK(launch_recurse_dummy(du, n, dm, ds, p, p.dummy, ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(),
                                    ws.cand_cnt.as<int32_t>(), ws.beta_dummy.as<uint8_t>(), max_M, grid, d_energy,
                                    d_assign, ev, st),
               "recursion kernel (dummy)");
            begin = end;
            continue;
        }
        if (g_count_mode && ex.mode == Exec::kNormal) {
            CK(ws.evaluated.ensure(sizeof(unsigned long long)), "workspace");
            CK(launch_recurse_count(du, n, dm, ds, p, ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(),
                                    ws.cand_cnt.as<int32_t>(), ws.beta.as<uint8_t>(), ws.res.as<UnitResult>(),
                                    ws.counter.as<int>(), ws.evaluated.as<unsigned long long>(), st),
               "recursion kernel (accounting)");
        } else {
            CK(launch_recurse(du, n, dm, ds, p, ws.cand_idx.as<int32_t>(), ws.cand_u.as<float>(),
                              ws.cand_cnt.as<int32_t>(), ws.beta.as<uint8_t>(), ws.res.as<UnitResult>(),
                              ws.counter.as<int>(), st),
               "recursion kernel");
        }
        CK(launch_backtrack(du, n, dm, ds, p, ws.cand_idx.as<int32_t>(), ws.beta.as<uint8_t>(),
                            ws.res.as<UnitResult>(), d_energy, d_assign, st),
           "backtrack kernel");
        begin = end;
    }
    return HGM_OK;
}

// A scene segment: offsets [oa, ob) of scene s; its unary-table block covers the
// sorted points [j0, j1) of the frames every model's windows can reach from them.
struct Segment {
    int s;
    int32_t oa, ob;
    int64_t j0, j1;
};

hgm_status run_batch(Exec &ex, const hgm_model *const *models, int nm, const hgm_scene *const *scenes, int ns,
                     const hgm_params *hp, cudaStream_t st, float *energy, int32_t *assign)
{
    Workspace &ws = *ex.ws;
    hgm_status rc = check_params(hp);
    if (rc) return rc;
    Plan pl;
    rc = build_plan(models, nm, scenes, ns, hp, pl);
    if (rc) return rc;
    Params p = to_params(hp);
    const int64_t n_out = pl.e_start.back();
    const int64_t n_assign = pl.a_start.back();
    if (n_out == 0 || nm == 0 || ns == 0) return HGM_OK;
    const int K = p.K;
    const int F = models[0]->d.F;
    p.F = F;
    p.max_window = 0;
    for (int s = 0; s < ns; ++s) p.max_window = std::max(p.max_window, typical_window_points(scenes[s], p.window));

    // model rows of the unary table (all models of the batch)
    int R = 0, max_M = 0, tmin_all = INT32_MAX, tmax_all = INT32_MIN;
    std::vector<int> urow(nm);
    for (int m = 0; m < nm; ++m) {
        urow[m] = R;
        R += models[m]->d.M;
        max_M = std::max(max_M, models[m]->d.M);
        tmin_all = std::min(tmin_all, models[m]->t_sorted.front());
        tmax_all = std::max(tmax_all, models[m]->t_sorted.back());
    }
    CK(ws.modelcat.ensure((size_t)R * F * sizeof(float)), "workspace (models)");
    for (int m = 0; m < nm; ++m)
        CK(cudaMemcpyAsync(ws.modelcat.as<float>() + (size_t)urow[m] * F, models[m]->d.f,
                           (size_t)models[m]->d.M * F * sizeof(float), cudaMemcpyDeviceToDevice, st),
           "gather model descriptors");
    std::vector<ModelRec> mrec(nm);
    for (int m = 0; m < nm; ++m)
        mrec[m] = ModelRec{models[m]->d.xy, models[m]->d.t, models[m]->d.perm, models[m]->d.M, urow[m],
                           models[m]->d.f, models[m]->d.geo};
    CK(ws.mrec.ensure(nm * sizeof(ModelRec)), "workspace");
    if ((rc = h2d(ex, ws.mrec.p, mrec.data(), nm * sizeof(ModelRec), st))) return rc;
    CK(ws.status.ensure(sizeof(int)), "workspace");
    CK(cudaMemsetAsync(ws.status.p, 0, sizeof(int), st), "memset");

    // proposal network: first-layer projections of the model points (the scene points' per segment)
    const hgm_prop *prop = hp->prune;
    const bool pruning = prop != nullptr;
    const int keep = pruning ? hp->keep : K;
    const int Fu = models[0]->F_user;
    PropInfer pi{};
    if (pruning) {
        if (prop->L.F != Fu) return fail(HGM_EINVAL, "proposal network built for F = %d, descriptors have F = %d",
                                         prop->L.F, Fu);
        const float *th = prop->theta;
        CK(ws.P.ensure((size_t)R * kPropHidden * sizeof(float)), "workspace (projections)");
        CK(launch_rowdot_plain(ws.modelcat.as<float>(), R, F, th + prop->L.o_W1, kPropHidden, prop->L.dp, Fu,
                               th + prop->L.o_b1, ws.P.as<float>(), kPropHidden, ws.status.as<int>(), st),
           "projection kernel");
        // position terms of the model points folded into P (the scene points' into Q)
        CK(ws.modelxy.ensure((size_t)R * 2 * sizeof(float)), "workspace (models)");
        for (int m = 0; m < nm; ++m)
            CK(cudaMemcpyAsync(ws.modelxy.as<float>() + (size_t)urow[m] * 2, models[m]->d.xy,
                               (size_t)models[m]->d.M * 2 * sizeof(float), cudaMemcpyDeviceToDevice, st),
               "gather model positions");
        CK(ws.Pb.ensure((size_t)R * kPropHidden * sizeof(__nv_bfloat16)), "workspace (projections)");
        CK(launch_prop_fold_xy(ws.P.as<float>(), R, ws.modelxy.as<float>(), th + prop->L.o_W1 + 2 * Fu,
                               prop->L.dp, -1.0f, ws.Pb.as<__nv_bfloat16>(), st),
           "projection kernel");
        pi.Pb = ws.Pb.as<__nv_bfloat16>();
        pi.W2 = th + prop->L.o_W2;
        pi.b2 = th + prop->L.o_b2;
        pi.w3 = th + prop->L.o_w3;
        pi.b3 = th + prop->L.o_b3;
        pi.w1c = th + prop->L.o_W1 + 2 * Fu;
        pi.dp = prop->L.dp;
        pi.inv_window = 1.0f / (float)std::max(hp->window, 1);
        pi.keep = keep;
        pi.rescore = hp->precision == 1 ? 1 : 0;   // the kept candidates are re-scored by the pruning pass,
        p.rescore = 0;                              // the fallback units' full lists by the fallback pass
        if (!g_ws.fb_total.p) {
            if (ex.mode == Exec::kCapture) return fail(HGM_ECUDA, "plan: fallback counter missing");
            CK(g_ws.fb_total.ensure(sizeof(unsigned long long)), "workspace");
            CK(cudaMemsetAsync(g_ws.fb_total.p, 0, sizeof(unsigned long long), st), "memset");
        }
    }
    ex.tensor = pruning || hp->precision == 1;
    if (hp->precision == 1) {
        CK(ws.mnorm.ensure((size_t)R * sizeof(float)), "workspace (norms)");
        CK(launch_sqnorm_bf16(ws.modelcat.as<float>(), R, F, F, ws.mnorm.as<float>(), st), "norm kernel");
    }

    // outputs: device pointers are written in place, host ones through staging
    const bool e_dev = energy && is_device_ptr(energy);
    const bool a_dev = assign && is_device_ptr(assign);
    float *d_energy = nullptr;
    int32_t *d_assign = nullptr;
    if (energy) {
        if (e_dev) d_energy = energy;
        else {
            CK(ws.out_e.ensure((size_t)n_out * sizeof(float)), "workspace (energy)");
            d_energy = ws.out_e.as<float>();
        }
    }
    if (assign) {
        if (a_dev) d_assign = assign;
        else {
            CK(ws.out_a.ensure((size_t)n_assign * sizeof(int32_t)), "workspace (assign)");
            d_assign = ws.out_a.as<int32_t>();
        }
    }

    // budgets: unary table (+ projections) per segment group, and candidate lists + argmin tables per chunk
    size_t budget = ex.budget;
    if (ex.mode != Exec::kCapture) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        budget = g_budget_override ? g_budget_override
                                   : std::max<size_t>((size_t)256 << 20, std::min<size_t>((size_t)24 << 30, free_b / 3));
        ex.budget = budget;
    }
    const int64_t per_point = (int64_t)R * 4 + (pruning ? (int64_t)kPropHidden * 6 : 0);
    const int64_t max_points = std::max<int64_t>(1, (int64_t)budget / per_point);

    // segments: per scene, runs of offsets whose reachable frames hold at most max_points points
    std::vector<Segment> segs;
    for (int s = 0; s < ns; ++s) {
        int64_t o_lo = INT64_MAX, o_hi = INT64_MIN;
        for (int m = 0; m < nm; ++m) {
            const size_t q = (size_t)m * ns + s;
            const int64_t n = pl.e_start[q + 1] - pl.e_start[q];
            for (int64_t k = 0; k < n; ++k) {
                if (ex.select && !(*ex.select)[(size_t)(pl.e_start[q] + k)]) continue;
                o_lo = std::min<int64_t>(o_lo, pl.first[q] + k);
                o_hi = std::max<int64_t>(o_hi, pl.first[q] + k);
                if (!ex.select) {
                    o_hi = std::max<int64_t>(o_hi, (int64_t)pl.first[q] + n - 1);
                    break;
                }
            }
        }
        if (o_lo > o_hi) continue;
        const std::vector<int32_t> &fs = scenes[s]->fs_host;
        const int nf = scenes[s]->d.n_frames;
        auto frame_lo = [&](int64_t oa) { return (int)std::max<int64_t>(0, oa + tmin_all - hp->window); };
        auto frame_hi = [&](int64_t ob) { return (int)std::min<int64_t>(nf - 1, ob - 1 + tmax_all + hp->window); };
        int64_t oa = o_lo;
        while (oa <= o_hi) {
            int64_t ob = oa + 1;
            const int64_t j0 = fs[(size_t)frame_lo(oa)];
            while (ob <= o_hi && fs[(size_t)frame_hi(ob + 1) + 1] - j0 <= max_points) ++ob;
            segs.push_back(Segment{s, (int32_t)oa, (int32_t)ob, j0, (int64_t)fs[(size_t)frame_hi(ob) + 1]});
            oa = ob;
        }
    }

    size_t gbegin = 0;
    while (gbegin < segs.size()) {
        // a group of consecutive segments whose unary tables fit together
        size_t gend = gbegin;
        int64_t gpoints = 0;
        while (gend < segs.size()) {
            const int64_t pts = round_up4((int)std::max<int64_t>(segs[gend].j1 - segs[gend].j0, 1));
            if (gend > gbegin && gpoints + pts > max_points) break;
            gpoints += pts;
            ++gend;
        }
        const int ng = (int)(gend - gbegin);
        CK(ws.U.ensure((size_t)R * gpoints * sizeof(float)), "workspace (unary table)");
        if (pruning) {
            CK(ws.Q.ensure((size_t)gpoints * kPropHidden * sizeof(float)), "workspace (projections)");
            CK(ws.Qb.ensure((size_t)gpoints * kPropHidden * sizeof(__nv_bfloat16)), "workspace (projections)");
        }
        std::vector<SceneRec> srec((size_t)ng);
        int64_t off = 0, smax = 0;
        for (int g = 0; g < ng; ++g) {
            const Segment &sg = segs[gbegin + g];
            const SceneDev &d = scenes[sg.s]->d;
            const int64_t pts = sg.j1 - sg.j0, pitch = round_up4((int)std::max<int64_t>(pts, 1));
            SceneRec r{d.xy, d.t, d.frame_start, d.perm, ws.U.as<float>() + (size_t)R * off, pitch, d.S, d.n_frames,
                       d.f};
            r.ucol0 = sg.j0;
            if (pruning) r.pq = ws.Qb.as<__nv_bfloat16>() + (size_t)off * kPropHidden;
            srec[(size_t)g] = r;
            off += pitch;
            smax = std::max(smax, pts);
        }
        CK(ws.srec.ensure((size_t)ng * sizeof(SceneRec)), "workspace");
        if ((rc = h2d(ex, ws.srec.p, srec.data(), (size_t)ng * sizeof(SceneRec), st))) return rc;
        if (hp->precision == 1) {
            CK(ws.snorm.ensure((size_t)std::max<int64_t>(smax, 1) * sizeof(float)), "workspace");
            CK(ws.ubf.ensure(unary_bf16_scratch_bytes(R, smax, F)), "workspace (BF16 operands)");
        }
        for (int g = 0; g < ng; ++g) {
            const Segment &sg = segs[gbegin + g];
            const SceneDev &d = scenes[sg.s]->d;
            const float *segf = d.f + (size_t)sg.j0 * F;
            const int pts = (int)(sg.j1 - sg.j0);
            float *U = const_cast<float *>(srec[(size_t)g].U);
            if (hp->precision == 1) {
                CK(launch_sqnorm_bf16(segf, pts, F, F, ws.snorm.as<float>(), st), "norm kernel");
                CK(launch_unary_bf16(ws.modelcat.as<float>(), R, segf, pts, F, F, ws.mnorm.as<float>(),
                                     ws.snorm.as<float>(), p.lambda1, U, srec[(size_t)g].upitch,
                                     ws.status.as<int>(), ws.ubf.p, ws.ubf.bytes, st),
                   "BF16 unary kernel");
            } else {
                CK(launch_unary(ws.modelcat.as<float>(), R, segf, pts, F, p.lambda1, U, (int)srec[(size_t)g].upitch,
                                st),
                   "unary kernel");
            }
            if (pruning) {
                const float *th = prop->theta;
                // FP32 projection of the segment's points (scratch), then position terms folded in and one
                // rounding to the BF16 rows the scoring kernel gathers
                float *qf = ws.Q.as<float>();
                CK(launch_rowdot_plain(segf, pts, F, th + prop->L.o_W1 + Fu, kPropHidden, prop->L.dp, Fu, nullptr, qf,
                                       kPropHidden, ws.status.as<int>(), st),
                   "projection kernel");
                CK(launch_prop_fold_xy(qf, pts, reinterpret_cast<const float *>(d.xy) + (size_t)sg.j0 * 2,
                                       th + prop->L.o_W1 + 2 * Fu, prop->L.dp, 1.0f,
                                       const_cast<__nv_bfloat16 *>(srec[(size_t)g].pq), st),
                   "projection kernel");
            }
        }

        // units of the group, longest first (counting sort by model size, stable)
        std::vector<int64_t> bucket((size_t)max_M + 2, 0);
        auto span = [&](int m, int g, int64_t &lo, int64_t &hi) {
            const Segment &sg = segs[gbegin + g];
            const size_t q = (size_t)m * ns + sg.s;
            const int64_t n = pl.e_start[q + 1] - pl.e_start[q];
            lo = std::max<int64_t>(sg.oa, pl.first[q]);
            hi = std::min<int64_t>(sg.ob, (int64_t)pl.first[q] + n);
        };
        int64_t n_units = 0;
        for (int m = 0; m < nm; ++m)
            for (int g = 0; g < ng; ++g) {
                int64_t lo, hi;
                span(m, g, lo, hi);
                if (hi <= lo) continue;
                int64_t cnt = hi - lo;
                if (ex.select) {
                    const size_t q = (size_t)m * ns + segs[gbegin + g].s;
                    cnt = 0;
                    for (int64_t o = lo; o < hi; ++o) cnt += (*ex.select)[(size_t)(pl.e_start[q] + (o - pl.first[q]))];
                }
                bucket[(size_t)(max_M - models[m]->d.M)] += cnt;
                n_units += cnt;
            }
        std::vector<int64_t> pos(bucket.size() + 1, 0);
        for (size_t k = 0; k < bucket.size(); ++k) pos[k + 1] = pos[k] + bucket[k];
        std::vector<Unit> all((size_t)n_units);
        for (int m = 0; m < nm; ++m)
            for (int g = 0; g < ng; ++g) {
                int64_t lo, hi;
                span(m, g, lo, hi);
                const Segment &sg = segs[gbegin + g];
                const size_t q = (size_t)m * ns + sg.s;
                const int M = models[m]->d.M;
                int64_t &w = pos[(size_t)(max_M - M)];
                for (int64_t o = lo; o < hi; ++o) {
                    if (ex.select && !(*ex.select)[(size_t)(pl.e_start[q] + (o - pl.first[q]))]) continue;
                    Unit u{};
                    u.model = m;
                    u.scene = g;
                    u.offset = (int32_t)o;
                    u.out_e = pl.e_start[q] + (o - pl.first[q]);
                    u.out_a = pl.a_start[q] + (o - pl.first[q]) * M;
                    all[(size_t)w++] = u;
                }
            }
        rc = run_units(ex, models, all, max_M, K, keep, pruning, p, pi, st, d_energy, d_assign, budget);
        if (rc) return rc;
        gbegin = gend;
    }
    if (energy && !e_dev)
        CK(cudaMemcpyAsync(energy, d_energy, (size_t)n_out * sizeof(float), cudaMemcpyDeviceToHost, st), "energy D2H");
    if (assign && !a_dev)
        CK(cudaMemcpyAsync(assign, d_assign, (size_t)n_assign * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
           "assign D2H");
    if (ex.mode == Exec::kCapture) return HGM_OK;
    // host outputs, or a tensor-core kernel whose bounded waits report through the status flag: wait here
    if ((energy && !e_dev) || (assign && !a_dev) || ex.tensor) {
        int status = 0;
        if (ex.tensor) CK(cudaMemcpyAsync(&status, ws.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
        CK(cudaStreamSynchronize(st), "synchronise outputs");
        if (status) return fail(HGM_ETIMEOUT, "a bounded tensor-core wait gave up");
    } else {
        CK(cudaGetLastError(), "launch");
    }
    return HGM_OK;
}

// run_batch, followed, for the pruned form with params->refine > 0, by the refinement: per (model, scene)
// pair the `refine` offsets of lowest pruned energy (finite; ties to the lower offset) are solved again
// without pruning, in the same precision mode, over the pruned results.
hgm_status run_matching(Exec &ex, const hgm_model *const *models, int nm, const hgm_scene *const *scenes, int ns,
                        const hgm_params *hp, cudaStream_t st, float *energy, int32_t *assign)
{
    if (!hp || !hp->prune || hp->refine <= 0 || (!energy && !assign))
        return run_batch(ex, models, nm, scenes, ns, hp, st, energy, assign);
    hgm_status rc = check_params(hp);
    if (rc) return rc;
    Plan pl;
    if ((rc = build_plan(models, nm, scenes, ns, hp, pl))) return rc;
    const int64_t n_out = pl.e_start.back(), n_assign = pl.a_start.back();
    if (n_out == 0) return HGM_OK;
    const bool e_dev = energy && is_device_ptr(energy), a_dev = assign && is_device_ptr(assign);
    float *de = energy;
    int32_t *da = assign;
    if (!e_dev) {
        CK(g_ws.rf_e.ensure((size_t)n_out * sizeof(float)), "workspace (refinement)");
        de = g_ws.rf_e.as<float>();
    }
    if (assign && !a_dev) {
        CK(g_ws.rf_a.ensure((size_t)n_assign * sizeof(int32_t)), "workspace (refinement)");
        da = g_ws.rf_a.as<int32_t>();
    }
    if ((rc = run_batch(ex, models, nm, scenes, ns, hp, st, de, da))) return rc;
    std::vector<float> eh((size_t)n_out);
    CK(cudaMemcpyAsync(eh.data(), de, (size_t)n_out * sizeof(float), cudaMemcpyDeviceToHost, st), "energy D2H");
    CK(cudaStreamSynchronize(st), "synchronise");
    std::vector<uint8_t> sel((size_t)n_out, 0);
    std::vector<int64_t> idx;
    int64_t n_sel = 0;
    for (size_t q = 0; q + 1 < pl.e_start.size(); ++q) {
        idx.clear();
        for (int64_t k = pl.e_start[q]; k < pl.e_start[q + 1]; ++k)
            if (eh[(size_t)k] < INFINITY) idx.push_back(k);
        const size_t r = std::min<size_t>((size_t)hp->refine, idx.size());
        std::partial_sort(idx.begin(), idx.begin() + (std::ptrdiff_t)r, idx.end(), [&](int64_t x, int64_t y) {
            return eh[(size_t)x] < eh[(size_t)y] || (eh[(size_t)x] == eh[(size_t)y] && x < y);
        });
        for (size_t k = 0; k < r; ++k) sel[(size_t)idx[k]] = 1;
        n_sel += (int64_t)r;
    }
    if (n_sel > 0) {
        hgm_params pe = *hp;
        pe.prune = nullptr;
        pe.refine = 0;
        Exec ex2;
        ex2.select = &sel;
        if ((rc = run_batch(ex2, models, nm, scenes, ns, &pe, st, de, da))) return rc;
        ex.tensor = ex.tensor || ex2.tensor;
    }
    ex.refined_units += n_sel;
    if (energy && !e_dev)
        CK(cudaMemcpyAsync(energy, de, (size_t)n_out * sizeof(float), cudaMemcpyDeviceToHost, st), "energy D2H");
    if (assign && !a_dev)
        CK(cudaMemcpyAsync(assign, da, (size_t)n_assign * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "assign D2H");
    CK(cudaStreamSynchronize(st), "synchronise outputs");
    return HGM_OK;
}

// Units for offsets [first, first+n) of one pair in offset order (kernel-level entry points).
hgm_status single_pair_units(const hgm_model *m, const hgm_scene *s, const hgm_params *hp, int32_t first,
                             int32_t n, cudaStream_t st, Params &p, int &R)
{
    hgm_status rc = check_params(hp);
    if (rc) return rc;
    if (!valid_model(m) || !valid_scene(s)) return fail(HGM_EINVAL, "invalid handle");
    if (m->F_user != s->F_user) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    int32_t nall, f0;
    hgm_params all = *hp;
    all.offset_lo = INT32_MIN;
    all.offset_hi = INT32_MAX;
    pair_offsets(m, s, &all, &nall, &f0);
    if (n < 0 || first < f0 || (int64_t)first + n > (int64_t)f0 + nall)
        return fail(HGM_EINVAL, "offsets [%d, %d) outside the valid range [%d, %d)", first, first + n, f0, f0 + nall);
    p = to_params(hp);
    p.F = m->d.F;
    p.max_window = typical_window_points(s, p.window);
    R = m->d.M;
    const int K = p.K;
    const int64_t pitch = round_up4(std::max(s->d.S, 1));
    CK(g_ws.U.ensure((size_t)R * pitch * sizeof(float)), "workspace (unary table)");
    ModelRec mr{m->d.xy, m->d.t, m->d.perm, m->d.M, 0, m->d.f, m->d.geo};
    SceneRec sr{s->d.xy, s->d.t, s->d.frame_start, s->d.perm, g_ws.U.as<float>(), pitch, s->d.S, s->d.n_frames,
                s->d.f};
    CK(g_ws.mrec.ensure(sizeof(ModelRec)), "workspace");
    CK(g_ws.srec.ensure(sizeof(SceneRec)), "workspace");
    CK(cudaMemcpyAsync(g_ws.mrec.p, &mr, sizeof mr, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(g_ws.srec.p, &sr, sizeof sr, cudaMemcpyHostToDevice, st), "upload");
    if (hp->precision == 1) {
        CK(g_ws.mnorm.ensure((size_t)R * sizeof(float)), "workspace (norms)");
        CK(g_ws.snorm.ensure((size_t)std::max(s->d.S, 1) * sizeof(float)), "workspace (norms)");
        CK(g_ws.status.ensure(sizeof(int)), "workspace");
        CK(cudaMemsetAsync(g_ws.status.p, 0, sizeof(int), st), "memset");
        CK(launch_sqnorm_bf16(m->d.f, R, m->d.F, m->d.F, g_ws.mnorm.as<float>(), st), "norm kernel");
        CK(launch_sqnorm_bf16(s->d.f, s->d.S, m->d.F, m->d.F, g_ws.snorm.as<float>(), st), "norm kernel");
        CK(g_ws.ubf.ensure(unary_bf16_scratch_bytes(R, s->d.S, m->d.F)), "workspace (BF16 operands)");
        CK(launch_unary_bf16(m->d.f, R, s->d.f, s->d.S, m->d.F, m->d.F, g_ws.mnorm.as<float>(), g_ws.snorm.as<float>(),
                             p.lambda1, g_ws.U.as<float>(), pitch, g_ws.status.as<int>(), g_ws.ubf.p, g_ws.ubf.bytes,
                             st),
           "BF16 unary kernel");
    } else {
        CK(launch_unary(m->d.f, R, s->d.f, s->d.S, m->d.F, p.lambda1, g_ws.U.as<float>(), (int)pitch, st),
           "unary kernel");
    }
    std::vector<Unit> units((size_t)n);
    for (int32_t k = 0; k < n; ++k) {
        Unit u{};
        u.model = 0;
        u.scene = 0;
        u.offset = first + k;
        u.cand = (int64_t)k * m->d.M * K;
        u.beta = (int64_t)k * (m->d.M - 2) * K * K;
        u.out_e = k;
        u.out_a = (int64_t)k * m->d.M;
        units[(size_t)k] = u;
    }
    CK(g_ws.units.ensure(std::max<size_t>(1, units.size()) * sizeof(Unit)), "workspace (units)");
    if (n) CK(cudaMemcpyAsync(g_ws.units.p, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice, st),
              "upload units");
    CK(cudaStreamSynchronize(st), "synchronise");   // host vector goes out of scope
    return HGM_OK;
}

}  // namespace

namespace hgm {
// The parameter check of every matching entry point, for other translation units of the library.
hgm_status check_match_params(const hgm_params *p) { return check_params(p); }

int32_t typical_window_points(const hgm_scene *s, int window)
{
    const int nf = s->d.n_frames;
    if (nf <= 0) return 0;
    const int64_t span = std::min<int64_t>(2 * std::max(window, 0) + 1, nf);
    return (int32_t)(((int64_t)s->d.S * span + nf - 1) / nf);
}
}  // namespace hgm

extern "C" {

void hgm_default_params(hgm_params *p)
{
    if (!p) return;
    p->lambda1 = 0.6f;
    p->lambda2 = 0.2f;
    p->lambda3 = 5.0f;
    p->T = 10;
    p->window = 3;
    p->K = 64;
    p->precision = 0;
    p->offset_lo = INT32_MIN;
    p->offset_hi = INT32_MAX;
    p->prune = nullptr;
    p->keep = 8;
    p->refine = 0;
    p->dummy_cost = -1.0f;
}

const char *hgm_last_error(void) { return g_err.c_str(); }

// ---- plans: a batch laid out once and replayed as a CUDA graph ---------------------------------------------
struct hgm_plan {
    uint32_t magic;
    Workspace ws;
    std::vector<std::pair<void *, size_t>> pinned;   // host sources of the recorded uploads
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t pruned_units = 0;
    bool tensor = false;
};

namespace {
void free_plan(hgm_plan *pl)
{
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    for (auto &h : pl->pinned) cudaFreeHost(h.first);
    pl->pinned.clear();
}
}  // namespace

hgm_status hgm_create_model(const float *xy, const int32_t *t, const float *desc, int32_t M, int32_t F, void *stream,
                            hgm_model **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!out) return fail(HGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (M < 3) return fail(HGM_EINVAL, "a model needs M >= 3 points (got %d)", M);
    if (F < 1 || F > 4096) return fail(HGM_EINVAL, "F must be in 1..4096 (got %d)", F);
    if (!xy || !t || !desc) return fail(HGM_EINVAL, "NULL input array");
    cudaStream_t st = (cudaStream_t)stream;
    // positions and frames are sorted on the host (small); descriptors go to the device raw and are
    // permuted there
    std::vector<float> hxy;
    std::vector<int32_t> ht;
    hgm_status rc;
    if ((rc = fetch(xy, (size_t)M * 2, hxy, st)) || (rc = fetch(t, (size_t)M, ht, st))) return rc;
    for (float v : hxy)
        if (!std::isfinite(v)) return fail(HGM_EINVAL, "non-finite model coordinate");
    for (int32_t v : ht)
        if (v < 0) return fail(HGM_EINVAL, "negative model frame");
    std::vector<int32_t> perm;
    sort_points(ht, perm);
    const int Fp = round_up4(F);
    std::vector<float2> sxy((size_t)M);
    std::vector<int32_t> stt((size_t)M);
    for (int k = 0; k < M; ++k) {
        int q = perm[(size_t)k];
        sxy[(size_t)k] = make_float2(hxy[(size_t)q * 2], hxy[(size_t)q * 2 + 1]);
        stt[(size_t)k] = ht[(size_t)q];
    }
    hgm_model *m = new hgm_model();
    m->magic = kModelMagic;
    m->d = ModelDev{M, Fp, nullptr, nullptr, nullptr, nullptr, nullptr};
    m->F_user = F;
    m->t_sorted = stt;
    m->perm = perm;
    m->span_t1 = stt.front();
    m->span_tM = stt.back();
    if ((rc = upload(&m->d.xy, sxy, st)) || (rc = upload(&m->d.t, stt, st)) ||
        (rc = upload_sorted_rows(desc, M, F, Fp, perm, &m->d.f, "model", st)) ||
        (rc = upload(&m->d.perm, perm, st))) {
        free_model(m);
        delete m;
        return rc;
    }
    cudaError_t e = cudaMalloc((void **)&m->d.geo, (size_t)M * sizeof(float4));
    if (e == cudaSuccess) e = launch_model_geo(m->d.xy, m->d.t, M, m->d.geo, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_model(m);
        delete m;
        return cuda_fail(e, "create model");
    }
    // the fixed scratch of hgm_match_noalloc is created on this device now, not at its first call
    if ((rc = noalloc_prepare())) {
        free_model(m);
        delete m;
        return rc;
    }
    *out = m;
    return HGM_OK;
}

hgm_status hgm_create_scene(const float *xy, const int32_t *t, const float *desc, int32_t S, int32_t F,
                            int32_t n_frames, void *stream, hgm_scene **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!out) return fail(HGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (S < 0) return fail(HGM_EINVAL, "S must be >= 0");
    if (F < 1 || F > 4096) return fail(HGM_EINVAL, "F must be in 1..4096 (got %d)", F);
    if (S > 0 && (!xy || !t || !desc)) return fail(HGM_EINVAL, "NULL input array");
    cudaStream_t st = (cudaStream_t)stream;
    // positions and frames are sorted on the host (small); descriptors go to the device raw and are
    // permuted there
    std::vector<float> hxy;
    std::vector<int32_t> ht;
    hgm_status rc;
    if ((rc = fetch(xy, (size_t)S * 2, hxy, st)) || (rc = fetch(t, (size_t)S, ht, st))) return rc;
    int32_t tmax = -1;
    for (int32_t v : ht) {
        if (v < 0) return fail(HGM_EINVAL, "negative scene frame");
        tmax = std::max(tmax, v);
    }
    if (n_frames <= 0) n_frames = tmax + 1;
    if (tmax >= n_frames) return fail(HGM_EINVAL, "scene frame %d outside [0, %d)", tmax, n_frames);
    if (n_frames <= 0) n_frames = 0;
    for (float v : hxy)
        if (!std::isfinite(v)) return fail(HGM_EINVAL, "non-finite scene coordinate");
    // stable counting sort by frame; minnode(f) = first sorted index with frame >= f
    std::vector<int32_t> fs((size_t)n_frames + 1, 0);
    for (int32_t v : ht) fs[(size_t)v + 1]++;
    for (int32_t f = 0; f < n_frames; ++f) fs[(size_t)f + 1] += fs[(size_t)f];
    std::vector<int32_t> perm((size_t)S);
    {
        std::vector<int32_t> w(fs.begin(), fs.end() - 1);
        for (int32_t k = 0; k < S; ++k) perm[(size_t)w[(size_t)ht[(size_t)k]]++] = k;
    }
    const int Fp = round_up4(F);
    std::vector<float2> sxy((size_t)S);
    std::vector<int32_t> stt((size_t)S);
    for (int32_t k = 0; k < S; ++k) {
        int32_t q = perm[(size_t)k];
        sxy[(size_t)k] = make_float2(hxy[(size_t)q * 2], hxy[(size_t)q * 2 + 1]);
        stt[(size_t)k] = ht[(size_t)q];
    }
    hgm_scene *s = new hgm_scene();
    s->magic = kSceneMagic;
    s->d = SceneDev{S, Fp, n_frames, nullptr, nullptr, nullptr, nullptr, nullptr};
    s->F_user = F;
    s->perm = perm;
    s->fs_host = fs;
    if ((rc = upload(&s->d.xy, sxy, st)) || (rc = upload(&s->d.t, stt, st)) ||
        (rc = upload_sorted_rows(desc, S, F, Fp, perm, &s->d.f, "scene", st)) ||
        (rc = upload(&s->d.frame_start, fs, st)) || (rc = upload(&s->d.perm, perm, st))) {
        free_scene(s);
        delete s;
        return rc;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_scene(s);
        delete s;
        return cuda_fail(e, "create scene");
    }
    if ((rc = noalloc_prepare())) {   // as in hgm_create_model
        free_scene(s);
        delete s;
        return rc;
    }
    *out = s;
    return HGM_OK;
}

void hgm_destroy(void *handle)
{
    if (!handle) return;
    std::lock_guard<std::mutex> lk(g_mu);
    uint32_t magic = *static_cast<uint32_t *>(handle);
    if (magic == kModelMagic) {
        hgm_model *m = static_cast<hgm_model *>(handle);
        cudaDeviceSynchronize();
        free_model(m);
        m->magic = kDeadMagic;
        delete m;
    } else if (magic == kSceneMagic) {
        hgm_scene *s = static_cast<hgm_scene *>(handle);
        cudaDeviceSynchronize();
        free_scene(s);
        s->magic = kDeadMagic;
        delete s;
    } else if (magic == kPlanMagic) {
        hgm_plan *pl = static_cast<hgm_plan *>(handle);
        cudaDeviceSynchronize();
        free_plan(pl);
        pl->magic = kDeadMagic;
        delete pl;
    } else if (magic == kStreamMagic) {
        hgm_stream *sm = static_cast<hgm_stream *>(handle);
        cudaDeviceSynchronize();
        free_stream(sm);
        sm->magic = kDeadMagic;
        delete sm;
    } else if (magic == kPropMagic) {
        hgm_prop *p = static_cast<hgm_prop *>(handle);
        cudaDeviceSynchronize();
        prop_free(p);
        p->magic = kDeadMagic;
        delete p;
    }
}

hgm_status hgm_offsets(const hgm_model *model, const hgm_scene *scene, const hgm_params *params, int32_t *n_offsets,
                       int32_t *first_offset)
{
    g_err.clear();
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (!valid_model(model) || !valid_scene(scene)) return fail(HGM_EINVAL, "invalid handle");
    int32_t n, f;
    pair_offsets(model, scene, params, &n, &f);
    if (n_offsets) *n_offsets = n;
    if (first_offset) *first_offset = f;
    return HGM_OK;
}

hgm_status hgm_batch_layout(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                            int32_t n_scenes, const hgm_params *params, int32_t *first_offset,
                            int64_t *energy_start, int64_t *assign_start)
{
    g_err.clear();
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (n_models < 0 || n_scenes < 0 || (n_models && !models) || (n_scenes && !scenes))
        return fail(HGM_EINVAL, "bad model/scene arrays");
    Plan pl;
    rc = build_plan(models, n_models, scenes, n_scenes, params, pl);
    if (rc) return rc;
    size_t np = (size_t)n_models * n_scenes;
    if (first_offset) std::copy(pl.first.begin(), pl.first.end(), first_offset);
    if (energy_start) std::copy(pl.e_start.begin(), pl.e_start.begin() + np + 1, energy_start);
    if (assign_start) std::copy(pl.a_start.begin(), pl.a_start.begin() + np + 1, assign_start);
    return HGM_OK;
}

hgm_status hgm_match(const hgm_model *model, const hgm_scene *scene, const hgm_params *params, void *stream,
                     int32_t *n_offsets, int32_t *first_offset, float *energy, int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (!valid_model(model) || !valid_scene(scene)) return fail(HGM_EINVAL, "invalid handle");
    if (model->F_user != scene->F_user) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    int32_t n, f;
    pair_offsets(model, scene, params, &n, &f);
    if (n_offsets) *n_offsets = n;
    if (first_offset) *first_offset = f;
    if (!energy && !assign) return HGM_OK;
    Exec ex;
    hgm_status rc2 = run_matching(ex, &model, 1, &scene, 1, params, (cudaStream_t)stream, energy, assign);
    g_pruned_units += ex.pruned_units;
    g_refined_units += ex.refined_units;
    return rc2;
}

// ---- the "independent chains" variant (Sec. 4, multiple points per frame, method 2) -------------------
namespace hgm {
namespace {

__global__ void chain_gather_kernel(const float2 *__restrict__ xy, const int32_t *__restrict__ t,
                                    const float *__restrict__ f, int Fp, const int32_t *__restrict__ ks, int n,
                                    float2 *__restrict__ oxy, int32_t *__restrict__ ot, float *__restrict__ of)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * Fp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / Fp), j = (int)(e - (int64_t)q * Fp);
        const int k = ks[q];
        of[e] = f[(int64_t)k * Fp + j];
        if (j == 0) {
            oxy[q] = xy[k];
            ot[q] = t[k];
        }
    }
}

// One (model, scene) pair of a chains batch: its outputs, and its chains' results in the chain batch.
struct ChainPair {
    int64_t e0, a0;      // first energy / assignment element of the pair in the caller's outputs
    int32_t n, M;        // offsets of the pair, points of the model
    int32_t nc, c0;      // chains of the model, first ChainRef of the pair
    int32_t map0, pad;   // first chain_map entry of the model
};
struct ChainRef {
    int64_t ce0, ca0;    // the chain's first energy / assignment element in the chain batch
    int32_t mc, pad;     // points of the chain
};

// energy[k] = mean of the chains' energies at offset k, summed in chain order (+inf if any is infeasible);
// assignment rows scattered to the model's caller indices (map: concatenated chain point -> caller index).
__global__ void chain_combine_kernel(const ChainPair *__restrict__ pairs, int n_pairs,
                                     const ChainRef *__restrict__ refs, const int32_t *__restrict__ map,
                                     const float *__restrict__ ce, const int32_t *__restrict__ ca,
                                     float *__restrict__ energy, int32_t *__restrict__ assign)
{
    for (int q = blockIdx.y; q < n_pairs; q += gridDim.y) {
        const ChainPair pr = pairs[q];
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < pr.n; k += gridDim.x * blockDim.x) {
            if (energy) {
                float sum = 0.0f;
                bool fin = true;
                for (int c = 0; c < pr.nc; ++c) {
                    const float v = ce[refs[pr.c0 + c].ce0 + k];
                    fin = fin && v < __builtin_huge_valf();
                    sum = __fadd_rn(sum, v);
                }
                energy[pr.e0 + k] = fin ? __fdiv_rn(sum, (float)pr.nc) : __builtin_huge_valf();
            }
            if (assign) {
                int32_t *row = assign + pr.a0 + (int64_t)k * pr.M;
                for (int i = 0; i < pr.M; ++i) row[i] = -1;
                int m0 = pr.map0;
                for (int c = 0; c < pr.nc; ++c) {
                    const ChainRef r = refs[pr.c0 + c];
                    const int32_t *src = ca + r.ca0 + (int64_t)k * r.mc;
                    for (int i = 0; i < r.mc; ++i) row[map[m0 + i]] = src[i];
                    m0 += r.mc;
                }
            }
        }
    }
}

// Splits model m into its chains (chain k: the point of within-frame rank k, ranked by caller index, of every
// model frame that has one; chains with fewer than 3 points are dropped) and keeps them on the model.
hgm_status build_chains(const hgm_model *m, int n_chains, int index, cudaStream_t st)
{
    if (m->chain_n == n_chains) return HGM_OK;
    if (!m->chains.empty()) {
        CK(cudaDeviceSynchronize(), "synchronise before replacing a chain split");
        for (hgm_model *c : m->chains) {
            free_model(c);
            delete c;
        }
        m->chains.clear();
        m->chain_map.clear();
        m->chain_n = 0;
    }
    const int M = m->d.M;
    std::vector<int32_t> rank((size_t)M);
    for (int k = 0; k < M;) {
        int e = k;
        while (e < M && m->t_sorted[(size_t)e] == m->t_sorted[(size_t)k]) ++e;
        std::vector<int32_t> ord;
        for (int q = k; q < e; ++q) ord.push_back(q);
        std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return m->perm[(size_t)x] < m->perm[(size_t)y]; });
        for (size_t r = 0; r < ord.size(); ++r) rank[(size_t)ord[r]] = (int32_t)r;
        k = e;
    }
    std::vector<std::vector<int32_t>> members;
    for (int c = 0; c < n_chains; ++c) {
        std::vector<int32_t> ks;
        for (int k = 0; k < M; ++k)
            if (rank[(size_t)k] == c) ks.push_back(k);
        if (ks.size() >= 3) members.push_back(ks);
    }
    if (members.empty()) return fail(HGM_EINVAL, "models[%d]: no chain has 3 points", index);
    const int Fp = m->d.F;
    std::vector<hgm_model *> chains;
    std::vector<int32_t> map;
    cudaError_t e = cudaSuccess;
    int32_t *dks = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&dks, (size_t)M * sizeof(int32_t));
    for (const auto &ks : members) {
        if (e != cudaSuccess) break;
        hgm_model *cm = new hgm_model();
        chains.push_back(cm);
        const int mc = (int)ks.size();
        cm->magic = kModelMagic;
        cm->d = ModelDev{mc, Fp, nullptr, nullptr, nullptr, nullptr, nullptr};
        cm->F_user = m->F_user;
        std::vector<int32_t> ident((size_t)mc);
        for (int q = 0; q < mc; ++q) {
            ident[(size_t)q] = q;
            cm->t_sorted.push_back(m->t_sorted[(size_t)ks[(size_t)q]]);
            map.push_back(m->perm[(size_t)ks[(size_t)q]]);
        }
        cm->perm = ident;     // one point per frame, already in frame order
        cm->span_t1 = m->span_t1;
        cm->span_tM = m->span_tM;
        if (e == cudaSuccess) e = cudaMalloc((void **)&cm->d.xy, (size_t)mc * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&cm->d.t, (size_t)mc * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&cm->d.f, (size_t)mc * Fp * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&cm->d.perm, (size_t)mc * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&cm->d.geo, (size_t)mc * sizeof(float4));
        if (e == cudaSuccess) e = cudaMemcpyAsync(dks, ks.data(), (size_t)mc * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cm->d.perm, ident.data(), (size_t)mc * sizeof(int32_t), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            chain_gather_kernel<<<(unsigned)std::min<int64_t>(((int64_t)mc * Fp + 255) / 256, 4096), 256, 0, st>>>(
                m->d.xy, m->d.t, m->d.f, Fp, dks, mc, cm->d.xy, cm->d.t, cm->d.f);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = launch_model_geo(cm->d.xy, cm->d.t, mc, cm->d.geo, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // dks and ident are reused / released
    }
    cudaFree(dks);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        for (hgm_model *c : chains) {
            free_model(c);
            delete c;
        }
        return cuda_fail(e, "chain models");
    }
    m->chains = chains;
    m->chain_map = map;
    m->chain_n = n_chains;
    return HGM_OK;
}

hgm_status run_chains(const hgm_model *const *models, int nm, const hgm_scene *const *scenes, int ns,
                      const hgm_params *params, int n_chains, cudaStream_t st, float *energy, int32_t *assign)
{
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (n_chains < 1 || n_chains > 255) return fail(HGM_EINVAL, "n_chains must be in 1..255 (got %d)", n_chains);
    if (nm < 0 || ns < 0 || (nm && !models) || (ns && !scenes)) return fail(HGM_EINVAL, "bad model/scene arrays");
    Plan pl;
    if ((rc = build_plan(models, nm, scenes, ns, params, pl))) return rc;
    if (pl.e_start.back() == 0 || (!energy && !assign)) return HGM_OK;
    for (int m = 0; m < nm; ++m)
        if ((rc = build_chains(models[m], n_chains, m, st))) return rc;
    // the chain batch: every model's chains, in model order
    std::vector<const hgm_model *> cms;
    std::vector<int32_t> cbase((size_t)nm), map_start((size_t)nm);
    std::vector<int32_t> map;
    for (int m = 0; m < nm; ++m) {
        cbase[(size_t)m] = (int32_t)cms.size();
        map_start[(size_t)m] = (int32_t)map.size();
        for (hgm_model *c : models[m]->chains) cms.push_back(c);
        map.insert(map.end(), models[m]->chain_map.begin(), models[m]->chain_map.end());
    }
    const int NC = (int)cms.size();
    Plan cpl;
    if ((rc = build_plan(cms.data(), NC, scenes, ns, params, cpl))) return rc;
    std::vector<ChainPair> pairs;
    std::vector<ChainRef> refs;
    for (int m = 0; m < nm; ++m)
        for (int s = 0; s < ns; ++s) {
            const size_t q = (size_t)m * ns + s;
            const int32_t n = (int32_t)(pl.e_start[q + 1] - pl.e_start[q]);
            if (n == 0) continue;
            const int nc = (int)models[m]->chains.size();
            pairs.push_back(ChainPair{pl.e_start[q], pl.a_start[q], n, models[m]->d.M, nc, (int32_t)refs.size(),
                                      map_start[(size_t)m], 0});
            for (int c = 0; c < nc; ++c) {
                const size_t cq = (size_t)(cbase[(size_t)m] + c) * ns + s;
                if (cpl.e_start[cq + 1] - cpl.e_start[cq] != n)
                    return fail(HGM_ECUDA, "chain offset range differs from its model's");
                refs.push_back(ChainRef{cpl.e_start[cq], cpl.a_start[cq], cms[(size_t)(cbase[(size_t)m] + c)]->d.M, 0});
            }
        }
    Workspace &ws = g_ws;
    const int64_t n_e = cpl.e_start.back(), n_a = cpl.a_start.back();
    const size_t b_pairs = (pairs.size() * sizeof(ChainPair) + 255) & ~(size_t)255;
    const size_t b_refs = (refs.size() * sizeof(ChainRef) + 255) & ~(size_t)255;
    CK(ws.chain_e.ensure((size_t)n_e * sizeof(float)), "workspace (chains)");
    CK(ws.chain_a.ensure((size_t)n_a * sizeof(int32_t)), "workspace (chains)");
    CK(ws.chain_tab.ensure(b_pairs + b_refs + map.size() * sizeof(int32_t)), "workspace (chains)");
    // chain results on the device (the chain batch fills every chain energy and assignment)
    Exec ex;
    rc = run_batch(ex, cms.data(), NC, scenes, ns, params, st, ws.chain_e.as<float>(), ws.chain_a.as<int32_t>());
    g_pruned_units += ex.pruned_units;
    if (rc) return rc;
    char *tab = ws.chain_tab.as<char>();
    if ((rc = h2d(ex, tab, pairs.data(), pairs.size() * sizeof(ChainPair), st)) ||
        (rc = h2d(ex, tab + b_pairs, refs.data(), refs.size() * sizeof(ChainRef), st)) ||
        (rc = h2d(ex, tab + b_pairs + b_refs, map.data(), map.size() * sizeof(int32_t), st)))
        return rc;
    const bool e_dev = energy && is_device_ptr(energy), a_dev = assign && is_device_ptr(assign);
    const int64_t n_out = pl.e_start.back(), n_assign = pl.a_start.back();
    float *de = energy;
    int32_t *da = assign;
    if (energy && !e_dev) {
        CK(ws.chain_oe.ensure((size_t)n_out * sizeof(float)), "workspace (chains)");
        de = ws.chain_oe.as<float>();
    }
    if (assign && !a_dev) {
        CK(ws.chain_oa.ensure((size_t)n_assign * sizeof(int32_t)), "workspace (chains)");
        da = ws.chain_oa.as<int32_t>();
    }
    int32_t max_n = 0;
    for (const ChainPair &pr : pairs) max_n = std::max(max_n, pr.n);
    const dim3 grid((unsigned)std::min<int64_t>((max_n + 127) / 128, 1024),
                    (unsigned)std::min<size_t>(std::max<size_t>(pairs.size(), 1), 65535));
    chain_combine_kernel<<<grid, 128, 0, st>>>(reinterpret_cast<const ChainPair *>(tab), (int)pairs.size(),
                                               reinterpret_cast<const ChainRef *>(tab + b_pairs),
                                               reinterpret_cast<const int32_t *>(tab + b_pairs + b_refs),
                                               ws.chain_e.as<float>(), ws.chain_a.as<int32_t>(), de, da);
    CK(cudaGetLastError(), "chain combine");
    if (energy && !e_dev)
        CK(cudaMemcpyAsync(energy, de, (size_t)n_out * sizeof(float), cudaMemcpyDeviceToHost, st), "copy energy");
    if (assign && !a_dev)
        CK(cudaMemcpyAsync(assign, da, (size_t)n_assign * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy assign");
    if ((energy && !e_dev) || (assign && !a_dev)) CK(cudaStreamSynchronize(st), "synchronise outputs");
    return HGM_OK;
}

}  // namespace
}  // namespace hgm

hgm_status hgm_match_chains(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                            int32_t n_chains, void *stream, int32_t *n_offsets, int32_t *first_offset, float *energy,
                            int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (!valid_model(model) || !valid_scene(scene)) return fail(HGM_EINVAL, "invalid handle");
    if (model->F_user != scene->F_user) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    if (n_chains < 1 || n_chains > 255) return fail(HGM_EINVAL, "n_chains must be in 1..255 (got %d)", n_chains);
    int32_t n, f;
    pair_offsets(model, scene, params, &n, &f);
    if (n_offsets) *n_offsets = n;
    if (first_offset) *first_offset = f;
    return run_chains(&model, 1, &scene, 1, params, n_chains, (cudaStream_t)stream, energy, assign);
}

hgm_status hgm_match_chains_batch(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                                  int32_t n_scenes, const hgm_params *params, int32_t n_chains, void *stream,
                                  float *energy, int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    return run_chains(models, n_models, scenes, n_scenes, params, n_chains, (cudaStream_t)stream, energy, assign);
}

// ---- the whole-block problem (Sec. 2.2, Sec. 3: every scene point a candidate of every model point) --------
namespace {

hgm_status check_block_models(const hgm_model *const *models, int nm, int *F)
{
    *F = -1;
    for (int m = 0; m < nm; ++m) {
        if (!valid_model(models[m])) return fail(HGM_EINVAL, "models[%d] is not a model handle", m);
        if (*F < 0) *F = models[m]->F_user;
        if (models[m]->F_user != *F) return fail(HGM_EINVAL, "descriptor widths differ across models");
    }
    return HGM_OK;
}

// Gathers the models' sorted descriptors into one row block and uploads their records.
hgm_status prep_block_models(BlockBufs &bb, const hgm_model *const *models, int nm, cudaStream_t st)
{
    bb.R = 0;
    bb.urow.assign((size_t)nm, 0);
    for (int m = 0; m < nm; ++m) {
        bb.urow[(size_t)m] = bb.R;
        bb.R += models[m]->d.M;
    }
    const int Fp = nm ? models[0]->d.F : 0;
    CK(bb.model.ensure((size_t)std::max(bb.R, 1) * std::max(Fp, 1) * sizeof(float)), "workspace (block)");
    CK(bb.mrec.ensure((size_t)std::max(nm, 1) * sizeof(ModelRec)), "workspace (block)");
    std::vector<ModelRec> mrec((size_t)nm);
    for (int m = 0; m < nm; ++m) {
        const hgm_model *md = models[m];
        CK(cudaMemcpyAsync(bb.model.as<float>() + (size_t)bb.urow[(size_t)m] * Fp, md->d.f,
                           (size_t)md->d.M * Fp * sizeof(float), cudaMemcpyDeviceToDevice, st),
           "gather model descriptors");
        mrec[(size_t)m] = ModelRec{md->d.xy, md->d.t, md->d.perm, md->d.M, bb.urow[(size_t)m], md->d.f, md->d.geo};
    }
    Exec ex;
    return h2d(ex, bb.mrec.p, mrec.data(), mrec.size() * sizeof(ModelRec), st);
}

// The whole-block problem for every (model, scene) pair; the models were prepared by prep_block_models.
hgm_status run_block(BlockBufs &bb, const hgm_model *const *models, int nm, const hgm_scene *const *scenes, int ns,
                     const hgm_params *params, cudaStream_t st, float *energy, int32_t *assign)
{
    const int T = params->T;
    // band tables per scene (host, from the minnode table): lo(b), cs(b)
    std::vector<int64_t> lo_off((size_t)ns), cs_off((size_t)ns), cell_off((size_t)ns), cells((size_t)ns);
    std::vector<int32_t> lo_all;
    std::vector<int64_t> cs_all;
    int64_t total_cells = 0, max_cells = 0;
    for (int s = 0; s < ns; ++s) {
        const hgm_scene *sc = scenes[s];
        const std::vector<int32_t> &fs = sc->fs_host;
        const int S = sc->d.S, nf = sc->d.n_frames;
        lo_off[(size_t)s] = (int64_t)lo_all.size();
        cs_off[(size_t)s] = (int64_t)cs_all.size();
        int64_t c = 0;
        for (int f = 0; f < nf; ++f) {
            const int lo = T > 0 ? fs[(size_t)std::max(0, f - T + 1)] : 0;
            const int reach = (T > 0 ? fs[(size_t)std::min(nf, f + T)] : S) - fs[(size_t)f];
            if (reach > 0xffff)
                return fail(HGM_EUNSUPPORTED, "scenes[%d]: %d points within T frames of frame %d (at most 65535)", s,
                            reach, f);
            for (int b = fs[(size_t)f]; b < fs[(size_t)f + 1]; ++b) {
                lo_all.push_back(lo);
                cs_all.push_back(c);
                c += fs[(size_t)f + 1] - lo;
            }
        }
        cs_all.push_back(c);
        cells[(size_t)s] = c;
        cell_off[(size_t)s] = total_cells;
        total_cells += c;
        max_cells = std::max(max_cells, c);
    }
    // units and outputs: pair q = m * n_scenes + s, assignment rows of M_m in pair order
    std::vector<BlockUnit> units;
    int64_t beta_total = 0, a_total = 0;
    for (int m = 0; m < nm; ++m)
        for (int s = 0; s < ns; ++s) {
            units.push_back(BlockUnit{m, s, beta_total, (int64_t)m * ns + s, a_total});
            beta_total += (int64_t)(models[m]->d.M - 2) * cells[(size_t)s];
            a_total += models[m]->d.M;
        }
    const size_t beta_bytes = (size_t)std::max<int64_t>(beta_total, 1) * sizeof(uint16_t);
    if (beta_bytes > bb.beta.bytes) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
        if ((double)beta_bytes > 0.6 * (double)(free_b + bb.beta.bytes))
            return fail(HGM_ENOMEM, "whole-block argmin tables need %zu bytes", beta_bytes);
    }
    const int R = bb.R;
    const int Fp = models[0]->d.F;
    int64_t S_total = 0;
    std::vector<int64_t> u_off((size_t)ns);
    for (int s = 0; s < ns; ++s) {
        u_off[(size_t)s] = S_total * R;
        S_total += scenes[s]->d.S;
    }
    // one upload: [lo | cs | units | scene records | band records], each part 256-byte aligned
    auto al256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t o_cs = al256(lo_all.size() * sizeof(int32_t));
    const size_t o_units = o_cs + al256(cs_all.size() * sizeof(int64_t));
    const size_t o_srec = o_units + al256(units.size() * sizeof(BlockUnit));
    const size_t o_geo = o_srec + al256((size_t)ns * sizeof(SceneRec));
    const size_t tab_bytes = o_geo + al256((size_t)ns * sizeof(BlockGeo));
    CK(bb.tab.ensure(tab_bytes), "workspace (block)");
    CK(bb.cellb.ensure((size_t)std::max<int64_t>(total_cells, 1) * sizeof(int32_t)), "workspace (block)");
    CK(bb.dir.ensure((size_t)std::max<int64_t>(total_cells, 1) * 2 * sizeof(float)), "workspace (block)");
    CK(bb.U.ensure((size_t)std::max<int64_t>(S_total * R, 1) * sizeof(float)), "workspace (block)");
    CK(bb.beta.ensure(beta_bytes), "workspace (block)");
    char *dtab = bb.tab.as<char>();
    const int32_t *d_lo = reinterpret_cast<const int32_t *>(dtab);
    const int64_t *d_cs = reinterpret_cast<const int64_t *>(dtab + o_cs);
    std::vector<BlockGeo> geos((size_t)ns);
    std::vector<SceneRec> srec((size_t)ns);
    float *dirf_all = bb.dir.as<float>(), *dirb_all = dirf_all + total_cells;
    for (int s = 0; s < ns; ++s) {
        const hgm_scene *sc = scenes[s];
        geos[(size_t)s] = BlockGeo{d_lo + lo_off[(size_t)s], d_cs + cs_off[(size_t)s],
                                   bb.cellb.as<int32_t>() + cell_off[(size_t)s], dirf_all + cell_off[(size_t)s],
                                   dirb_all + cell_off[(size_t)s], cells[(size_t)s]};
        srec[(size_t)s] = SceneRec{sc->d.xy, sc->d.t, sc->d.frame_start, sc->d.perm, bb.U.as<float>() + u_off[(size_t)s],
                                   (int64_t)sc->d.S, sc->d.S, sc->d.n_frames, sc->d.f, nullptr, 0};
    }
    char *h = nullptr;
    std::vector<char> blob;
    if (bb.own_pinned) {
        if (!bb.upload_done) CK(cudaEventCreateWithFlags(&bb.upload_done, cudaEventDisableTiming), "event");
        CK(cudaEventSynchronize(bb.upload_done), "wait for the previous upload");
        if (bb.pinned_bytes < tab_bytes) {
            if (bb.pinned) cudaFreeHost(bb.pinned);
            bb.pinned = nullptr;
            bb.pinned_bytes = 0;
            CK(cudaMallocHost(&bb.pinned, 2 * tab_bytes), "pinned staging");
            bb.pinned_bytes = 2 * tab_bytes;
        }
        h = static_cast<char *>(bb.pinned);
    } else {
        blob.resize(tab_bytes);
        h = blob.data();
    }
    std::memcpy(h, lo_all.data(), lo_all.size() * sizeof(int32_t));
    std::memcpy(h + o_cs, cs_all.data(), cs_all.size() * sizeof(int64_t));
    std::memcpy(h + o_units, units.data(), units.size() * sizeof(BlockUnit));
    std::memcpy(h + o_srec, srec.data(), srec.size() * sizeof(SceneRec));
    std::memcpy(h + o_geo, geos.data(), geos.size() * sizeof(BlockGeo));
    CK(cudaMemcpyAsync(dtab, h, tab_bytes, cudaMemcpyHostToDevice, st), "upload block tables");
    if (bb.own_pinned) CK(cudaEventRecord(bb.upload_done, st), "event");
    for (int s = 0; s < ns; ++s) {
        const hgm_scene *sc = scenes[s];
        const BlockGeo &g = geos[(size_t)s];
        CK(launch_block_geo(sc->d.xy, sc->d.S, g.lo, g.cs, g.cells, const_cast<int32_t *>(g.cellb),
                            const_cast<float *>(g.dirf), const_cast<float *>(g.dirb), st),
           "block geometry");
        if (sc->d.S > 0)
            CK(launch_unary(bb.model.as<float>(), R, sc->d.f, sc->d.S, Fp, params->lambda1,
                            const_cast<float *>(srec[(size_t)s].U), sc->d.S, st),
               "unary kernel");
    }
    char *rec = dtab + o_units;
    const size_t b_units = o_srec - o_units, b_s = o_geo - o_srec;
    const bool e_dev = energy && is_device_ptr(energy), a_dev = assign && is_device_ptr(assign);
    float *de = energy;
    int32_t *da = assign;
    if (!energy || !e_dev) {
        CK(bb.oe.ensure(units.size() * sizeof(float)), "workspace (block)");
        de = bb.oe.as<float>();
    }
    if (!assign || !a_dev) {
        CK(bb.oa.ensure((size_t)a_total * sizeof(int32_t)), "workspace (block)");
        da = bb.oa.as<int32_t>();
    }
    Params p = to_params(params);
    p.F = Fp;
    float *scratch = nullptr;
    int grid_global = 0;
    static int64_t smem_cells = -1;
    if (smem_cells < 0) smem_cells = block_smem_cells();
    if (max_cells > smem_cells) {
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev), "device");
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
        grid_global = (int)std::min<int64_t>((int64_t)units.size(), (int64_t)sms * 2);
        CK(bb.scratch.ensure((size_t)grid_global * 2 * max_cells * sizeof(float)), "workspace (block)");
        scratch = bb.scratch.as<float>();
    }
    CK(launch_block_recurse(reinterpret_cast<const BlockUnit *>(rec), (int)units.size(), bb.mrec.as<ModelRec>(),
                            reinterpret_cast<const SceneRec *>(rec + b_units),
                            reinterpret_cast<const BlockGeo *>(rec + b_units + b_s), p, max_cells,
                            bb.beta.as<uint16_t>(), scratch, grid_global, de, da, st),
       "block recursion kernel");
    if (energy && !e_dev)
        CK(cudaMemcpyAsync(energy, de, units.size() * sizeof(float), cudaMemcpyDeviceToHost, st), "copy energy");
    if (assign && !a_dev)
        CK(cudaMemcpyAsync(assign, da, (size_t)a_total * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy assign");
    if ((energy && !e_dev) || (assign && !a_dev)) CK(cudaStreamSynchronize(st), "synchronise outputs");
    return HGM_OK;
}

}  // namespace

hgm_status hgm_match_block(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                           int32_t n_scenes, const hgm_params *params, void *stream, float *energy, int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (params->precision != 0 || params->prune || params->dummy_cost >= 0)
        return fail(HGM_EUNSUPPORTED,
                    "the whole-block problem runs in plain FP32 only (precision 0, no pruning, no dummy)");
    if (n_models < 0 || n_scenes < 0 || (n_models && !models) || (n_scenes && !scenes))
        return fail(HGM_EINVAL, "bad model/scene arrays");
    if (n_models == 0 || n_scenes == 0 || (!energy && !assign)) return HGM_OK;
    int F;
    if ((rc = check_block_models(models, n_models, &F))) return rc;
    for (int s = 0; s < n_scenes; ++s) {
        if (!valid_scene(scenes[s])) return fail(HGM_EINVAL, "scenes[%d] is not a scene handle", s);
        if (scenes[s]->F_user != F) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = prep_block_models(g_blk, models, n_models, st))) return rc;
    return run_block(g_blk, models, n_models, scenes, n_scenes, params, st, energy, assign);
}

// ---- streaming blocks (Sec. 4: the scene cut into blocks of ~60 frames, matched as they arrive) ----------
namespace hgm {
namespace {
size_t al16(size_t v) { return (v + 15) & ~(size_t)15; }

// Byte layout of a streamed block's upload: sorted xy | t | permutation | minnode table | raw descriptors.
struct StreamUpload {
    size_t o_t, o_perm, o_fs, o_raw;
    StreamUpload(int64_t n, int B)
    {
        o_t = al16((size_t)n * 8);
        o_perm = o_t + al16((size_t)n * 4);
        o_fs = o_perm + al16((size_t)n * 4);
        o_raw = o_fs + al16((size_t)(B + 1) * 4);
    }
};

// Every buffer a block of up to P points can need, allocated once: the upload staging (pinned) and its device
// copy, the sorted descriptors, the band tables (at most P cells per point: a band holds points of the block),
// the unary and argmin tables, the global alpha scratch when a band exceeds shared memory, the outputs.
hgm_status stream_reserve(hgm_stream *s, int64_t P, cudaStream_t st)
{
    (void)st;
    const int B = s->block_frames, F = s->F_user, Fp = s->Fp;
    const int64_t nm = (int64_t)s->models.size();
    int64_t R = 0, Rm2 = 0;
    for (const hgm_model *m : s->models) {
        R += m->d.M;
        Rm2 += m->d.M - 2;
    }
    const StreamUpload up(P, B);
    const size_t upload = up.o_raw + (size_t)P * F * sizeof(float);
    CK(cudaMallocHost(&s->pinned, upload), "pinned staging");
    s->pinned_bytes = upload;
    CK(s->sc_buf.ensure(upload), "stream buffers");
    CK(s->f.ensure((size_t)std::max<int64_t>(P, 1) * Fp * sizeof(float)), "stream buffers");
    CK(s->flag.ensure(sizeof(int)), "stream buffers");
    CK(s->dev_e.ensure((size_t)nm * sizeof(float)), "stream buffers");
    CK(s->dev_a.ensure((size_t)std::max<int64_t>(R, 1) * sizeof(int32_t)), "stream buffers");
    const size_t o_a = al16((size_t)nm * sizeof(float));
    s->pin_out_bytes = o_a + al16((size_t)R * sizeof(int32_t)) + 16;
    CK(cudaMallocHost(&s->pin_out, s->pin_out_bytes), "pinned staging");
    // run_block's buffers for one scene of P points
    BlockBufs &bb = s->bb;
    auto al256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t tab = al256((size_t)P * 4) + al256((size_t)(P + 1) * 8) + al256((size_t)nm * sizeof(BlockUnit)) +
                       al256(sizeof(SceneRec)) + al256(sizeof(BlockGeo));
    const int64_t cells = std::max<int64_t>(P * P, 1);
    CK(bb.tab.ensure(tab), "stream buffers");
    CK(cudaMallocHost(&bb.pinned, tab), "pinned staging");
    bb.pinned_bytes = tab;
    CK(bb.cellb.ensure((size_t)cells * sizeof(int32_t)), "stream buffers");
    CK(bb.dir.ensure((size_t)cells * 2 * sizeof(float)), "stream buffers");
    CK(bb.U.ensure((size_t)std::max<int64_t>(P * R, 1) * sizeof(float)), "stream buffers");
    CK(bb.beta.ensure((size_t)std::max<int64_t>(Rm2 * cells, 1) * sizeof(uint16_t)), "stream buffers");
    CK(bb.oe.ensure((size_t)nm * sizeof(float)), "stream buffers");
    CK(bb.oa.ensure((size_t)std::max<int64_t>(R, 1) * sizeof(int32_t)), "stream buffers");
    if (cells > block_smem_cells()) {
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev), "device");
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
        const int64_t grid = std::min<int64_t>(nm, (int64_t)sms * 2);
        CK(bb.scratch.ensure((size_t)grid * 2 * cells * sizeof(float)), "stream buffers");
    }
    return HGM_OK;
}
}  // namespace
}  // namespace hgm

hgm_status hgm_stream_create(const hgm_model *const *models, int32_t n_models, const hgm_params *params,
                             int32_t block_frames, int32_t max_points, void *stream, hgm_stream **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!out) return fail(HGM_EINVAL, "out is NULL");
    *out = nullptr;
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (params->precision != 0 || params->prune || params->dummy_cost >= 0)
        return fail(HGM_EUNSUPPORTED,
                    "the whole-block problem runs in plain FP32 only (precision 0, no pruning, no dummy)");
    if (n_models < 1 || !models) return fail(HGM_EINVAL, "need at least one model");
    if (block_frames < 1) return fail(HGM_EINVAL, "block_frames must be >= 1 (got %d)", block_frames);
    if (max_points < 1) return fail(HGM_EINVAL, "max_points must be >= 1 (got %d)", max_points);
    int F;
    if ((rc = check_block_models(models, n_models, &F))) return rc;
    hgm_stream *s = new hgm_stream();
    s->magic = kStreamMagic;
    s->models.assign(models, models + n_models);
    s->params = *params;
    s->block_frames = block_frames;
    s->max_points = max_points;
    s->F_user = F;
    s->Fp = models[0]->d.F;
    s->view.magic = kSceneMagic;
    s->view.F_user = F;
    s->bb.own_pinned = true;
    cudaStream_t st = (cudaStream_t)stream;
    rc = prep_block_models(s->bb, s->models.data(), n_models, st);
    if (!rc) rc = stream_reserve(s, max_points, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "stream create");
    if (rc) {
        free_stream(s);
        s->magic = kDeadMagic;
        delete s;
        return rc;
    }
    *out = s;
    return HGM_OK;
}

hgm_status hgm_stream_match(hgm_stream *s, const float *xy, const int32_t *t, const float *desc, int32_t n,
                            void *stream, float *energy, int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!valid_stream(s)) return fail(HGM_EINVAL, "not a stream handle");
    if (n < 0) return fail(HGM_EINVAL, "n must be >= 0");
    if (n > s->max_points)
        return fail(HGM_EUNSUPPORTED, "block of %d points; this stream was created for at most %d", n, s->max_points);
    if (n > 0 && (!xy || !t || !desc)) return fail(HGM_EINVAL, "NULL input array");
    cudaStream_t st = (cudaStream_t)stream;
    const int B = s->block_frames, F = s->F_user, Fp = s->Fp;
    std::vector<float> hxy;
    std::vector<int32_t> ht;
    hgm_status rc;
    if ((rc = fetch(xy, (size_t)n * 2, hxy, st)) || (rc = fetch(t, (size_t)n, ht, st))) return rc;
    for (int32_t v : ht)
        if (v < 0 || v >= B) return fail(HGM_EINVAL, "block frame %d outside [0, %d)", v, B);
    for (float v : hxy)
        if (!std::isfinite(v)) return fail(HGM_EINVAL, "non-finite scene coordinate");
    // stable counting sort by frame; the block's points, permutation and minnode table in one upload
    std::vector<int32_t> fs((size_t)B + 1, 0);
    for (int32_t v : ht) fs[(size_t)v + 1]++;
    for (int f = 0; f < B; ++f) fs[(size_t)f + 1] += fs[(size_t)f];
    std::vector<int32_t> perm((size_t)n);
    {
        std::vector<int32_t> w(fs.begin(), fs.end() - 1);
        for (int32_t k = 0; k < n; ++k) perm[(size_t)w[(size_t)ht[(size_t)k]]++] = k;
    }
    const StreamUpload up(n, B);
    const size_t o_xy = 0, o_t = up.o_t, o_perm = up.o_perm, o_fs = up.o_fs, o_raw = up.o_raw;
    const bool desc_dev = n > 0 && is_device_ptr(desc);
    const size_t total = o_raw + (desc_dev ? 0 : (size_t)n * F * sizeof(float));
    if (total > s->pinned_bytes) return fail(HGM_ECUDA, "stream staging smaller than its capacity (internal)");
    CK(cudaStreamSynchronize(st), "synchronise the staging buffer");   // the previous block's upload
    char *h = static_cast<char *>(s->pinned);
    float2 *sxy = reinterpret_cast<float2 *>(h + o_xy);
    int32_t *stt = reinterpret_cast<int32_t *>(h + o_t);
    for (int32_t k = 0; k < n; ++k) {
        const int32_t q = perm[(size_t)k];
        sxy[k] = make_float2(hxy[(size_t)q * 2], hxy[(size_t)q * 2 + 1]);
        stt[k] = ht[(size_t)q];
    }
    std::memcpy(h + o_perm, perm.data(), (size_t)n * 4);
    std::memcpy(h + o_fs, fs.data(), (size_t)(B + 1) * 4);
    if (!desc_dev && n > 0) std::memcpy(h + o_raw, desc, (size_t)n * F * sizeof(float));
    CK(s->sc_buf.ensure(total), "stream buffers");
    CK(s->f.ensure((size_t)std::max(n, 1) * Fp * sizeof(float)), "stream buffers");
    CK(s->flag.ensure(sizeof(int)), "stream buffers");
    CK(cudaMemcpyAsync(s->sc_buf.p, h, total, cudaMemcpyHostToDevice, st), "upload block");
    char *d = s->sc_buf.as<char>();
    CK(cudaMemsetAsync(s->flag.p, 0, sizeof(int), st), "memset");
    if (n > 0) {
        const float *dsrc = desc_dev ? desc : reinterpret_cast<const float *>(d + o_raw);
        const int64_t blocks = std::min<int64_t>(((int64_t)n * Fp + 255) / 256, 65536);
        gather_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(dsrc, F, reinterpret_cast<const int32_t *>(d + o_perm), n,
                                                             Fp, s->f.as<float>(), s->flag.as<int>());
        CK(cudaGetLastError(), "gather kernel");
    }
    hgm_scene &v = s->view;
    v.d = SceneDev{n, Fp, B, reinterpret_cast<float2 *>(d + o_xy), reinterpret_cast<int32_t *>(d + o_t),
                   s->f.as<float>(), reinterpret_cast<int32_t *>(d + o_fs), reinterpret_cast<int32_t *>(d + o_perm)};
    v.perm = perm;
    v.fs_host = fs;
    const hgm_scene *sv = &v;
    std::vector<const hgm_model *> &ms = s->models;
    const bool e_host = energy && !is_device_ptr(energy), a_host = assign && !is_device_ptr(assign);
    if (!e_host && !a_host) return run_block(s->bb, ms.data(), (int)ms.size(), &sv, 1, &s->params, st, energy, assign);
    // host outputs: results into device buffers, then one read-back of energies, assignments and the
    // descriptor flag through pinned memory and a single wait
    const size_t nm = ms.size();
    size_t a_total = 0;
    for (const hgm_model *m : ms) a_total += (size_t)m->d.M;
    CK(s->dev_e.ensure(nm * sizeof(float)), "stream buffers");
    CK(s->dev_a.ensure(std::max<size_t>(a_total, 1) * sizeof(int32_t)), "stream buffers");
    rc = run_block(s->bb, ms.data(), (int)nm, &sv, 1, &s->params, st, s->dev_e.as<float>(), s->dev_a.as<int32_t>());
    if (rc) return rc;
    const size_t o_a = al16(nm * sizeof(float));
    const size_t o_f = o_a + al16(a_total * sizeof(int32_t));
    if (o_f + 16 > s->pin_out_bytes) return fail(HGM_ECUDA, "stream read-back smaller than its capacity (internal)");
    char *ho = static_cast<char *>(s->pin_out);
    CK(cudaMemcpyAsync(ho, s->dev_e.p, nm * sizeof(float), cudaMemcpyDeviceToHost, st), "copy energy");
    CK(cudaMemcpyAsync(ho + o_a, s->dev_a.p, a_total * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "copy assign");
    CK(cudaMemcpyAsync(ho + o_f, s->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
    CK(cudaStreamSynchronize(st), "synchronise");
    int bad = 0;
    std::memcpy(&bad, ho + o_f, sizeof(int));
    if (bad) return fail(HGM_EINVAL, "non-finite block descriptor (outputs are not valid)");
    if (energy) {
        if (e_host) std::memcpy(energy, ho, nm * sizeof(float));
        else CK(cudaMemcpyAsync(energy, s->dev_e.p, nm * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy energy");
    }
    if (assign) {
        if (a_host) std::memcpy(assign, ho + o_a, a_total * sizeof(int32_t));
        else CK(cudaMemcpyAsync(assign, s->dev_a.p, a_total * sizeof(int32_t), cudaMemcpyDeviceToDevice, st),
                "copy assign");
    }
    return HGM_OK;
}

hgm_status hgm_match_batch(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                           int32_t n_scenes, const hgm_params *params, void *stream, float *energy, int32_t *assign)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (n_models < 0 || n_scenes < 0 || (n_models && !models) || (n_scenes && !scenes))
        return fail(HGM_EINVAL, "bad model/scene arrays");
    Exec ex;
    hgm_status rc = run_matching(ex, models, n_models, scenes, n_scenes, params, (cudaStream_t)stream, energy,
                                 assign);
    g_pruned_units += ex.pruned_units;
    g_refined_units += ex.refined_units;
    return rc;
}

hgm_status hgm_model_order(const hgm_model *model, int32_t *perm)
{
    g_err.clear();
    if (!valid_model(model) || !perm) return fail(HGM_EINVAL, "invalid argument");
    std::copy(model->perm.begin(), model->perm.end(), perm);
    return HGM_OK;
}

hgm_status hgm_scene_order(const hgm_scene *scene, int32_t *perm)
{
    g_err.clear();
    if (!valid_scene(scene) || !perm) return fail(HGM_EINVAL, "invalid argument");
    std::copy(scene->perm.begin(), scene->perm.end(), perm);
    return HGM_OK;
}

hgm_status hgm_unary(const hgm_model *model, const hgm_scene *scene, float lambda1, void *stream, float *U)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (!valid_model(model) || !valid_scene(scene)) return fail(HGM_EINVAL, "invalid handle");
    if (model->F_user != scene->F_user) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    if (!U || !is_device_ptr(U)) return fail(HGM_EINVAL, "U must be a device pointer");
    if (!std::isfinite(lambda1) || lambda1 < 0) return fail(HGM_EINVAL, "lambda1 must be finite and >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    CK(launch_unary(model->d.f, model->d.M, scene->d.f, scene->d.S, model->d.F, lambda1, U, scene->d.S, st),
       "unary kernel");
    return HGM_OK;
}

hgm_status hgm_unary_bf16(const hgm_model *model, const hgm_scene *scene, float lambda1, void *stream, float *U)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (!valid_model(model) || !valid_scene(scene)) return fail(HGM_EINVAL, "invalid handle");
    if (model->F_user != scene->F_user) return fail(HGM_EINVAL, "descriptor width differs between model and scene");
    if (!U || !is_device_ptr(U)) return fail(HGM_EINVAL, "U must be a device pointer");
    if (!std::isfinite(lambda1) || lambda1 < 0) return fail(HGM_EINVAL, "lambda1 must be finite and >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const int F = model->d.F, M = model->d.M, S = scene->d.S;
    CK(g_ws.mnorm.ensure((size_t)M * sizeof(float)), "workspace (norms)");
    CK(g_ws.snorm.ensure((size_t)std::max(S, 1) * sizeof(float)), "workspace (norms)");
    CK(g_ws.status.ensure(sizeof(int)), "workspace");
    CK(cudaMemsetAsync(g_ws.status.p, 0, sizeof(int), st), "memset");
    CK(launch_sqnorm_bf16(model->d.f, M, F, F, g_ws.mnorm.as<float>(), st), "norm kernel");
    CK(launch_sqnorm_bf16(scene->d.f, S, F, F, g_ws.snorm.as<float>(), st), "norm kernel");
    CK(g_ws.ubf.ensure(unary_bf16_scratch_bytes(M, S, F)), "workspace (BF16 operands)");
    CK(launch_unary_bf16(model->d.f, M, scene->d.f, S, F, F, g_ws.mnorm.as<float>(), g_ws.snorm.as<float>(), lambda1,
                         U, S, g_ws.status.as<int>(), g_ws.ubf.p, g_ws.ubf.bytes, st),
       "BF16 unary kernel");
    int status = 0;
    CK(cudaMemcpyAsync(&status, g_ws.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    CK(cudaStreamSynchronize(st), "synchronise");
    if (status) return fail(HGM_ETIMEOUT, "a bounded wait for the tensor core gave up");
    return HGM_OK;
}

hgm_status hgm_candidates(const hgm_model *model, const hgm_scene *scene, const hgm_params *params, int32_t first,
                          int32_t n, void *stream, int32_t *idx, int32_t *cnt, float *cost)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (!idx || !cnt || !is_device_ptr(idx) || !is_device_ptr(cnt) || (cost && !is_device_ptr(cost)))
        return fail(HGM_EINVAL, "outputs must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    Params p;
    int R;
    hgm_status rc = single_pair_units(model, scene, params, first, n, st, p, R);
    if (rc) return rc;
    if (n == 0) return HGM_OK;
    if (!cost) {
        CK(g_ws.cand_u.ensure((size_t)n * model->d.M * p.K * sizeof(float)), "workspace (candidates)");
        cost = g_ws.cand_u.as<float>();
    }
    CK(launch_select(g_ws.units.as<Unit>(), n, g_ws.mrec.as<ModelRec>(), g_ws.srec.as<SceneRec>(), p, model->d.M, idx,
                     cost, cnt, st),
       "select kernel");
    return HGM_OK;
}

hgm_status hgm_prop_scores(const hgm_prop *prop, const hgm_model *model, const hgm_scene *scene,
                           const hgm_params *params, int32_t first, int32_t n, void *stream, float *scores)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (!prop || prop->magic != kPropMagic) return fail(HGM_EINVAL, "prop is not a proposal-network handle");
    if (!scores || !is_device_ptr(scores)) return fail(HGM_EINVAL, "scores must be a device pointer");
    if (params && params->K > 64) return fail(HGM_EUNSUPPORTED, "proposal scoring needs K <= 64");
    cudaStream_t st = (cudaStream_t)stream;
    Params p;
    int R;
    hgm_status rc = single_pair_units(model, scene, params, first, n, st, p, R);
    if (rc) return rc;
    const int Fu = model->F_user, F = model->d.F, M = model->d.M, S = scene->d.S;
    if (prop->L.F != Fu) return fail(HGM_EINVAL, "proposal network built for F = %d, descriptors have F = %d",
                                     prop->L.F, Fu);
    if (n == 0) return HGM_OK;
    const size_t ce = (size_t)n * M * p.K;
    CK(g_ws.cand_idx.ensure(ce * sizeof(int32_t)), "workspace (candidates)");
    CK(g_ws.cand_u.ensure(ce * sizeof(float)), "workspace (candidates)");
    CK(g_ws.cand_cnt.ensure((size_t)n * M * sizeof(int32_t)), "workspace (candidates)");
    CK(launch_select(g_ws.units.as<Unit>(), n, g_ws.mrec.as<ModelRec>(), g_ws.srec.as<SceneRec>(), p, M,
                     g_ws.cand_idx.as<int32_t>(), g_ws.cand_u.as<float>(), g_ws.cand_cnt.as<int32_t>(), st),
       "select kernel");
    const float *th = prop->theta;
    CK(g_ws.P.ensure((size_t)M * kPropHidden * sizeof(float)), "workspace (projections)");
    CK(g_ws.Q.ensure((size_t)std::max(S, 1) * kPropHidden * sizeof(float)), "workspace (projections)");
    CK(g_ws.status.ensure(sizeof(int)), "workspace");
    CK(cudaMemsetAsync(g_ws.status.p, 0, sizeof(int), st), "memset");
    CK(launch_rowdot_plain(model->d.f, M, F, th + prop->L.o_W1, kPropHidden, prop->L.dp, Fu, th + prop->L.o_b1,
                           g_ws.P.as<float>(), kPropHidden, g_ws.status.as<int>(), st),
       "projection kernel");
    CK(g_ws.Pb.ensure((size_t)M * kPropHidden * sizeof(__nv_bfloat16)), "workspace (projections)");
    CK(launch_prop_fold_xy(g_ws.P.as<float>(), M, reinterpret_cast<const float *>(model->d.xy),
                           th + prop->L.o_W1 + 2 * Fu, prop->L.dp, -1.0f, g_ws.Pb.as<__nv_bfloat16>(), st),
       "projection kernel");
    CK(launch_rowdot_plain(scene->d.f, S, F, th + prop->L.o_W1 + Fu, kPropHidden, prop->L.dp, Fu, nullptr,
                           g_ws.Q.as<float>(), kPropHidden, g_ws.status.as<int>(), st),
       "projection kernel");
    CK(g_ws.Qb.ensure((size_t)std::max(S, 1) * kPropHidden * sizeof(__nv_bfloat16)), "workspace (projections)");
    CK(launch_prop_fold_xy(g_ws.Q.as<float>(), S, reinterpret_cast<const float *>(scene->d.xy),
                           th + prop->L.o_W1 + 2 * Fu, prop->L.dp, 1.0f, g_ws.Qb.p, st),
       "projection kernel");
    const int64_t pitch = round_up4(std::max(S, 1));
    SceneRec sr{scene->d.xy, scene->d.t, scene->d.frame_start, scene->d.perm, g_ws.U.as<float>(), pitch, S,
                scene->d.n_frames, scene->d.f};
    sr.pq = g_ws.Qb.as<__nv_bfloat16>();
    CK(cudaMemcpyAsync(g_ws.srec.p, &sr, sizeof sr, cudaMemcpyHostToDevice, st), "upload");
    PropInfer pi{};
    pi.Pb = g_ws.Pb.as<__nv_bfloat16>();
    pi.W2 = th + prop->L.o_W2;
    pi.b2 = th + prop->L.o_b2;
    pi.w3 = th + prop->L.o_w3;
    pi.b3 = th + prop->L.o_b3;
    pi.w1c = th + prop->L.o_W1 + 2 * Fu;
    pi.dp = prop->L.dp;
    pi.inv_window = 1.0f / (float)std::max(params->window, 1);
    pi.keep = p.K;
    CK(launch_prop_score(g_ws.units.as<Unit>(), n, g_ws.mrec.as<ModelRec>(), g_ws.srec.as<SceneRec>(), p, pi,
                         g_ws.cand_idx.as<int32_t>(), g_ws.cand_cnt.as<int32_t>(), scores, g_ws.status.as<int>(), st),
       "scoring kernel");
    int status = 0;
    CK(cudaMemcpyAsync(&status, g_ws.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    CK(cudaStreamSynchronize(st), "synchronise");
    if (status) return fail(HGM_ETIMEOUT, "a bounded tensor-core wait gave up");
    return HGM_OK;
}

hgm_status hgm_count_triples(const hgm_model *model, const hgm_scene *scene, const hgm_params *params, int32_t first,
                             int32_t n, void *stream, int64_t *triples)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (!triples || !is_device_ptr(triples)) return fail(HGM_EINVAL, "triples must be a device pointer");
    cudaStream_t st = (cudaStream_t)stream;
    Params p;
    int R;
    hgm_status rc = single_pair_units(model, scene, params, first, n, st, p, R);
    if (rc) return rc;
    if (n == 0) return HGM_OK;
    const size_t ce = (size_t)n * model->d.M * p.K;
    CK(g_ws.cand_idx.ensure(ce * sizeof(int32_t)), "workspace (candidates)");
    CK(g_ws.cand_u.ensure(ce * sizeof(float)), "workspace (candidates)");
    CK(g_ws.cand_cnt.ensure((size_t)n * model->d.M * sizeof(int32_t)), "workspace (candidates)");
    CK(launch_select(g_ws.units.as<Unit>(), n, g_ws.mrec.as<ModelRec>(), g_ws.srec.as<SceneRec>(), p, model->d.M,
                     g_ws.cand_idx.as<int32_t>(), g_ws.cand_u.as<float>(), g_ws.cand_cnt.as<int32_t>(), st),
       "select kernel");
    CK(launch_count(g_ws.units.as<Unit>(), n, g_ws.mrec.as<ModelRec>(), g_ws.srec.as<SceneRec>(), p,
                    g_ws.cand_idx.as<int32_t>(), g_ws.cand_cnt.as<int32_t>(), triples, st),
       "count kernel");
    return HGM_OK;
}

hgm_status hgm_set_recurse_variant(int32_t variant)
{
    g_err.clear();
    if (variant < 0 || variant >= recurse_variant_count()) return fail(HGM_EINVAL, "variant out of range");
    set_recurse_variant(variant);
    return HGM_OK;
}

int32_t hgm_get_recurse_variant(void) { return get_recurse_variant(); }

hgm_status hgm_autotune(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                        int32_t n_scenes, const hgm_params *params, void *stream, int32_t sample_offsets,
                        int32_t *best_variant, float *ms_per_variant)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    WsGuard wsg((cudaStream_t)stream);
    if (n_models < 1 || n_scenes < 1 || !models || !scenes || sample_offsets < 1)
        return fail(HGM_EINVAL, "bad autotune arguments");
    hgm_status rc = check_params(params);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    hgm_params ps = *params;
    ps.offset_lo = std::max(params->offset_lo, 0);
    ps.offset_hi = (int32_t)std::min<int64_t>(params->offset_hi, (int64_t)ps.offset_lo + sample_offsets - 1);
    const int nv = recurse_variant_count();
    const int keep = get_recurse_variant();
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a), "event");
    CK(cudaEventCreate(&b), "event");
    float best_ms = 3.0e38f;
    int best = keep;
    for (int v = 0; v < nv; ++v) {
        set_recurse_variant(v);
        float vbest = 3.0e38f;
        for (int rep = 0; rep < 3; ++rep) {          // first repetition is a warm-up
            CK(cudaEventRecord(a, st), "event");
            Exec ex;
            rc = run_batch(ex, models, n_models, scenes, n_scenes, &ps, st, nullptr, nullptr);
            if (rc) { set_recurse_variant(keep); cudaEventDestroy(a); cudaEventDestroy(b); return rc; }
            CK(cudaEventRecord(b, st), "event");
            CK(cudaEventSynchronize(b), "event");
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, a, b), "event");
            if (rep > 0) vbest = std::min(vbest, ms);
        }
        if (ms_per_variant) ms_per_variant[v] = vbest;
        if (vbest < best_ms) { best_ms = vbest; best = v; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_recurse_variant(best);
    if (best_variant) *best_variant = best;
    return HGM_OK;
}

hgm_status hgm_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on == 1;
    g_count_mode = on == 2;
    return HGM_OK;
}

hgm_status hgm_plan_create(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                           int32_t n_scenes, const hgm_params *params, float *energy, int32_t *assign, void *stream,
                           hgm_plan **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!out) return fail(HGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_models < 1 || n_scenes < 1 || !models || !scenes) return fail(HGM_EINVAL, "bad model/scene arrays");
    if ((energy && !is_device_ptr(energy)) || (assign && !is_device_ptr(assign)))
        return fail(HGM_EINVAL, "plan outputs must be device pointers");
    hgm_status rc = check_params(params);
    if (rc) return rc;
    if (params->prune && params->refine > 0)
        return fail(HGM_EUNSUPPORTED, "plans do not run the refinement (it reads the pruned energies on the host)");
    cudaStream_t st = (cudaStream_t)stream;
    hgm_plan *pl = new hgm_plan();
    pl->magic = kPlanMagic;
    auto bail = [&](hgm_status r) {
        g_capturing = false;
        free_plan(pl);
        delete pl;
        return r;
    };
    // sizing pass: runs the batch once on the plan's workspace (growing it) and keeps the host uploads
    Exec ex;
    ex.mode = Exec::kSizing;
    ex.ws = &pl->ws;
    ex.pinned = &pl->pinned;
    if ((rc = run_batch(ex, models, n_models, scenes, n_scenes, params, st, energy, assign))) return bail(rc);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "plan sizing pass"));
    pl->pruned_units = ex.pruned_units;
    pl->tensor = ex.tensor;
    g_pruned_units += ex.pruned_units;   // the sizing pass ran the batch
    // recorded pass, on a private stream (the legacy stream cannot be captured)
    if ((e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "plan stream"));
    Exec rec;
    rec.mode = Exec::kCapture;
    rec.ws = &pl->ws;
    rec.pinned = &pl->pinned;
    rec.budget = ex.budget;
    if ((e = cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail(cuda_fail(e, "begin capture"));
    g_capturing = true;
    rc = run_batch(rec, models, n_models, scenes, n_scenes, params, pl->cap, energy, assign);
    g_capturing = false;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(pl->cap, &g);
    pl->graph = g;
    if (rc) return bail(rc);
    if (e != cudaSuccess) return bail(cuda_fail(e, "end capture"));
    if (rec.pin_next != pl->pinned.size()) return bail(fail(HGM_ECUDA, "plan: recorded pass skipped uploads"));
    if ((e = cudaGraphInstantiate(&pl->exec, pl->graph, 0)) != cudaSuccess)
        return bail(cuda_fail(e, "graph instantiate"));
    *out = pl;
    return HGM_OK;
}

hgm_status hgm_plan_run(hgm_plan *plan, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!plan || plan->magic != kPlanMagic) return fail(HGM_EINVAL, "invalid plan");
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->tensor) CK(cudaMemsetAsync(plan->ws.status.p, 0, sizeof(int), st), "memset");
    CK(cudaGraphLaunch(plan->exec, st), "graph launch");
    g_pruned_units += plan->pruned_units;
    return HGM_OK;
}

hgm_status hgm_plan_check(hgm_plan *plan, void *stream)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!plan || plan->magic != kPlanMagic) return fail(HGM_EINVAL, "invalid plan");
    cudaStream_t st = (cudaStream_t)stream;
    int status = 0;
    if (plan->tensor) CK(cudaMemcpyAsync(&status, plan->ws.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    CK(cudaStreamSynchronize(st), "synchronise");
    if (status) return fail(HGM_ETIMEOUT, "a bounded tensor-core wait gave up");
    return HGM_OK;
}

hgm_status hgm_set_workspace_budget(int64_t bytes)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (bytes < 0) return fail(HGM_EINVAL, "budget must be >= 0");
    g_budget_override = (size_t)bytes;
    return HGM_OK;
}

hgm_status hgm_refine_counter(int64_t *refined_units, int32_t reset)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (refined_units) *refined_units = g_refined_units;
    if (reset) g_refined_units = 0;
    return HGM_OK;
}

hgm_status hgm_prune_counters(int64_t *pruned_units, int64_t *fallback_units, int32_t reset)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    unsigned long long fb = 0;
    if (g_ws.fb_total.p) {
        CK(cudaDeviceSynchronize(), "synchronise");
        CK(cudaMemcpy(&fb, g_ws.fb_total.p, sizeof fb, cudaMemcpyDeviceToHost), "read counter");
        if (reset) CK(cudaMemset(g_ws.fb_total.p, 0, sizeof fb), "reset counter");
    }
    if (pruned_units) *pruned_units = g_pruned_units;
    if (fallback_units) *fallback_units = (int64_t)fb;
    if (reset) g_pruned_units = 0;
    return HGM_OK;
}

hgm_status hgm_profile_evaluated(int64_t *evaluated, int32_t reset)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_err.clear();
    if (!evaluated) return fail(HGM_EINVAL, "evaluated is NULL");
    *evaluated = 0;
    if (!g_ws.evaluated.p) {
        if (reset) CK(g_ws.evaluated.ensure(sizeof(unsigned long long)), "workspace");
        else return HGM_OK;
    }
    CK(cudaDeviceSynchronize(), "synchronise");
    unsigned long long v = 0;
    CK(cudaMemcpy(&v, g_ws.evaluated.p, sizeof v, cudaMemcpyDeviceToHost), "read counter");
    *evaluated = (int64_t)v;
    if (reset) CK(cudaMemset(g_ws.evaluated.p, 0, sizeof v), "reset counter");
    return HGM_OK;
}

hgm_status hgm_profile_read(double *ms, int64_t *launches, int32_t n_kernels)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_err.clear();
    for (ProfRec &r : g_prof_pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
        float t = 0.0f;
        cudaEventElapsedTime(&t, r.a, r.b);
        g_prof_ms[r.kernel] += t;
        g_prof_n[r.kernel] += 1;
        g_prof_free.push_back(r.a);
        g_prof_free.push_back(r.b);
    }
    g_prof_pending.clear();
    for (int k = 0; k < n_kernels && k < kProfCount; ++k) {
        if (ms) ms[k] = g_prof_ms[k];
        if (launches) launches[k] = g_prof_n[k];
    }
    return HGM_OK;
}

hgm_status hgm_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (ProfRec &r : g_prof_pending) {
        cudaEventSynchronize(r.b);
        g_prof_free.push_back(r.a);
        g_prof_free.push_back(r.b);
    }
    g_prof_pending.clear();
    for (int k = 0; k < kProfCount; ++k) {
        g_prof_ms[k] = 0;
        g_prof_n[k] = 0;
    }
    return HGM_OK;
}

}  // extern "C"
