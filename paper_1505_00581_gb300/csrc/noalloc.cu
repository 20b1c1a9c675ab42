// noalloc.cu -- hgm_match_noalloc: the single-pair match without any device allocation.
//
// Who needs this: programs that must not allocate device memory once they are
// running -- a real-time video loop that may not stall (cudaMalloc and
// cudaFree can synchronise the whole device and take allocator locks), or a
// host application or plugin framework that reserves all device memory at
// start-up and forbids allocations afterwards. hgm_match sizes its workspace
// per call and may grow it with cudaMalloc; this entry point instead works in
// one fixed scratch array that is part of the library image.
//
// The scratch is a file-scope __device__ array of kScratchBytes (64 MiB). The
// CUDA runtime creates it on a GPU when it loads this file's device code there,
// and it stays there until the process exits. The runtime loads code lazily
// (on first use) by default, so the array would otherwise appear only at the
// first hgm_match_noalloc call, possibly after the caller has reserved all
// device memory. Host code cannot use the array's name as a device address (on
// the host it names a stand-in object), so noalloc_prepare() asks the runtime
// for the real address with cudaGetSymbolAddress, with the device current, and
// caches it per device; that lookup loads the code and creates the array. It
// also has the runtime load the code of every kernel this entry point launches.
// hgm_create_model and hgm_create_scene call noalloc_prepare(), so the scratch
// exists on a device from the first handle created there, and the address is
// known before the caller reserves memory or captures a stream.
//
// All calls share the one array and it keeps the previous call's contents:
// the persistent-kernel work counter is cleared on every call, everything else
// is fully rewritten before it is read. Two calls whose GPU work overlaps in
// time (different streams, or different host threads) race on the scratch.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "hgm_internal.cuh"

namespace hgm {
namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once per device).
hgm_status scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(HGM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(HGM_EUNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            return set_error(HGM_ECUDA, msg);
        }
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return HGM_OK;
}

// Writes the unit list of one chunk of offsets and the model/scene records into scratch.
__global__ void fill_units_kernel(Unit *units, int n, int first_offset, int chunk_begin, int M, int K,
                                  ModelRec *mr, SceneRec *sr, ModelRec m, SceneRec s)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        *mr = m;
        *sr = s;
    }
    if (k < n) {
        Unit u{};
        u.model = 0;
        u.scene = 0;
        u.offset = first_offset + chunk_begin + k;
        u.cand = (int64_t)k * M * K;
        u.beta = (int64_t)k * (M - 2) * K * K;
        u.out_e = chunk_begin + k;
        u.out_a = (int64_t)(chunk_begin + k) * M;
        units[k] = u;
    }
}

bool is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

hgm_status noalloc_prepare()
{
    unsigned char *p = nullptr;
    hgm_status rc = scratch_address(&p);
    if (rc) return rc;
    // the kernels this entry point launches: their code is loaded now as well
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, fill_units_kernel);
    if (e == cudaSuccess) e = preload_unary();
    if (e == cudaSuccess) e = preload_select();
    if (e == cudaSuccess) e = preload_recurse();
    if (e == cudaSuccess) e = preload_recurse_small();
    if (e == cudaSuccess) e = preload_backtrack();
    if (e != cudaSuccess) return set_error(HGM_ECUDA, cudaGetErrorString(e));
    return HGM_OK;
}
}  // namespace hgm

using namespace hgm;

extern "C" hgm_status hgm_match_noalloc(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                                        void *stream, float *energy, int32_t *assign)
{
    // the checks of hgm_match first (invalid values: HGM_EINVAL), then the options this entry point leaves out
    hgm_status rc = check_match_params(params);
    if (rc) return rc;
    if (!valid_model(model) || !valid_scene(scene)) return set_error(HGM_EINVAL, "invalid handle");
    if (model->F_user != scene->F_user)
        return set_error(HGM_EINVAL, "descriptor width differs between model and scene");
    if (params->precision != 0)
        return set_error(HGM_EUNSUPPORTED, "hgm_match_noalloc: only precision 0 (FP32 exact); use hgm_match");
    if (params->dummy_cost >= 0)
        return set_error(HGM_EUNSUPPORTED, "hgm_match_noalloc: no dummy assignment (dummy_cost >= 0); use hgm_match");
    if (params->prune)
        return set_error(HGM_EUNSUPPORTED, "hgm_match_noalloc: no pruning (prune != NULL); use hgm_match");
    if (params->refine > 0)
        return set_error(HGM_EUNSUPPORTED, "hgm_match_noalloc: no refinement (refine > 0); use hgm_match");
    if (!energy || !assign || !is_device(energy) || !is_device(assign))
        return set_error(HGM_EINVAL, "energy and assign must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;

    // offset range (same rule as hgm_offsets)
    const int64_t t1 = model->span_t1, tM = model->span_tM;
    int64_t lo = std::max<int64_t>(-t1, params->offset_lo);
    int64_t hi = std::min<int64_t>((int64_t)scene->d.n_frames - 1 - tM, params->offset_hi);
    const int n_off = hi >= lo ? (int)(hi - lo + 1) : 0;
    if (n_off == 0) return HGM_OK;

    const int M = model->d.M, K = params->K, S = scene->d.S;
    const int64_t pitch = ((int64_t)std::max(S, 1) + 3) & ~(int64_t)3;
    // fixed part: counter | model record | scene record | unary table
    const size_t off_mr = 256, off_sr = off_mr + align256(sizeof(ModelRec)), off_u = off_sr + align256(sizeof(SceneRec));
    const size_t u_bytes = align256((size_t)M * pitch * sizeof(float));
    const size_t fixed = off_u + u_bytes;
    // per unit: unit record, result, counts, candidate indices and costs, argmin tables
    const size_t per_unit = sizeof(Unit) + sizeof(UnitResult) + (size_t)M * 4 + (size_t)M * K * 8 +
                            (size_t)(M - 2) * K * K;
    const size_t slack = 6 * 256;
    if (fixed + slack + per_unit > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "hgm_match_noalloc: this pair needs %zu bytes of scratch for one offset, the fixed scratch holds "
                 "%zu (the unary table alone is M x S x 4 = %zu bytes); use hgm_match",
                 fixed + slack + per_unit, kScratchBytes, u_bytes);
        return set_error(HGM_EUNSUPPORTED, msg);
    }
    const int cap = (int)std::min<size_t>((kScratchBytes - fixed - slack) / per_unit, (size_t)n_off);

    unsigned char *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    int *counter = reinterpret_cast<int *>(base);
    ModelRec *d_mr = reinterpret_cast<ModelRec *>(base + off_mr);
    SceneRec *d_sr = reinterpret_cast<SceneRec *>(base + off_sr);
    float *d_U = reinterpret_cast<float *>(base + off_u);
    size_t off = fixed;
    Unit *d_units = reinterpret_cast<Unit *>(base + off);
    off += align256((size_t)cap * sizeof(Unit));
    UnitResult *d_res = reinterpret_cast<UnitResult *>(base + off);
    off += align256((size_t)cap * sizeof(UnitResult));
    int32_t *d_cnt = reinterpret_cast<int32_t *>(base + off);
    off += align256((size_t)cap * M * 4);
    int32_t *d_idx = reinterpret_cast<int32_t *>(base + off);
    off += align256((size_t)cap * M * K * 4);
    float *d_cu = reinterpret_cast<float *>(base + off);
    off += align256((size_t)cap * M * K * 4);
    uint8_t *d_beta = reinterpret_cast<uint8_t *>(base + off);
    off += align256((size_t)cap * (M - 2) * K * K);
    if (off > kScratchBytes) return set_error(HGM_EUNSUPPORTED, "hgm_match_noalloc: scratch layout overflow");

    Params p;
    p.lambda1 = params->lambda1;
    p.lambda2 = params->lambda2;
    p.lambda3 = params->lambda3;
    p.T = params->T;
    p.window = params->window;
    p.K = K;
    p.max_window = typical_window_points(scene, p.window);
    const ModelRec mr{model->d.xy, model->d.t, model->d.perm, M, 0, model->d.f, model->d.geo};
    const SceneRec sr{scene->d.xy, scene->d.t, scene->d.frame_start, scene->d.perm, d_U, pitch, S, scene->d.n_frames};

    cudaError_t e = launch_unary(model->d.f, M, scene->d.f, S, model->d.F, p.lambda1, d_U, (int)pitch, st);
    if (e != cudaSuccess) return set_error(HGM_ECUDA, cudaGetErrorString(e));
    for (int c0 = 0; c0 < n_off; c0 += cap) {
        const int n = std::min(cap, n_off - c0);
        fill_units_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_units, n, (int)lo, c0, M, K, d_mr, d_sr, mr, sr);
        if ((e = cudaGetLastError()) != cudaSuccess) return set_error(HGM_ECUDA, cudaGetErrorString(e));
        if ((e = launch_select(d_units, n, d_mr, d_sr, p, M, d_idx, d_cu, d_cnt, st)) != cudaSuccess ||
            (e = launch_recurse(d_units, n, d_mr, d_sr, p, d_idx, d_cu, d_cnt, d_beta, d_res, counter, st)) !=
                cudaSuccess ||
            (e = launch_backtrack(d_units, n, d_mr, d_sr, p, d_idx, d_beta, d_res, energy, assign, st)) !=
                cudaSuccess)
            return set_error(HGM_ECUDA, cudaGetErrorString(e));
    }
    return HGM_OK;
}
