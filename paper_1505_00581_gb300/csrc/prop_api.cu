// prop_api.cu -- C ABI of the candidate-proposal network (see include/hgm.h).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "prop.cuh"

using namespace hgm;

namespace {

std::mutex g_prop_mu;

bool valid_prop(const hgm_prop *p) { return p && p->magic == kPropMagic; }

bool is_dev(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

hgm_status cuerr(cudaError_t e, const char *what)
{
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return set_error(e == cudaErrorMemoryAllocation ? HGM_ENOMEM : HGM_ECUDA, msg);
}

hgm_status check_status(hgm_prop *p, cudaStream_t st)
{
    int s = 0;
    cudaError_t e = cudaMemcpyAsync(&s, p->train.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuerr(e, "status");
    if (s) return set_error(HGM_ETIMEOUT, "a bounded wait for the tensor core gave up");
    return HGM_OK;
}

}  // namespace

void prop_free(hgm_prop *p)
{
    cudaFree(p->theta);
    cudaFree(p->grad);
    cudaFree(p->m);
    cudaFree(p->v);
    if (p->train.buf) cudaFree(p->train.buf);
}

extern "C" {

hgm_status hgm_prop_create(int32_t F, const float *weights, uint64_t seed, hgm_prop **out)
{
    std::lock_guard<std::mutex> lk(g_prop_mu);
    if (!out) return set_error(HGM_EINVAL, "out is NULL");
    *out = nullptr;
    if (F < 1 || F > 4096) return set_error(HGM_EINVAL, "F must be in 1..4096");
    hgm_prop *p = new hgm_prop();
    p->magic = kPropMagic;
    p->L = prop_layout(F);
    std::vector<float> logical;
    if (weights) logical.assign(weights, weights + p->L.n_logical);
    else prop_init(p->L, seed, logical);
    for (float v : logical)
        if (!std::isfinite(v)) { delete p; return set_error(HGM_EINVAL, "non-finite weight"); }
    std::vector<float> flat;
    prop_pack(p->L, logical.data(), flat);
    const size_t bytes = sizeof(float) * (size_t)p->L.n;
    cudaError_t e;
    if ((e = cudaMalloc(&p->theta, bytes)) || (e = cudaMalloc(&p->grad, bytes)) || (e = cudaMalloc(&p->m, bytes)) ||
        (e = cudaMalloc(&p->v, bytes)) || (e = cudaMemcpy(p->theta, flat.data(), bytes, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(p->grad, 0, bytes)) || (e = cudaMemset(p->m, 0, bytes)) || (e = cudaMemset(p->v, 0, bytes))) {
        prop_free(p);
        delete p;
        return cuerr(e, "create proposal network");
    }
    *out = p;
    return HGM_OK;
}

int64_t hgm_prop_size(int32_t F) { return F >= 1 ? prop_layout(F).n_logical : -1; }

hgm_status hgm_prop_get(const hgm_prop *prop, float *weights, int64_t *step)
{
    if (!valid_prop(prop) || !weights) return set_error(HGM_EINVAL, "invalid argument");
    std::vector<float> flat((size_t)prop->L.n);
    cudaError_t e = cudaMemcpy(flat.data(), prop->theta, sizeof(float) * flat.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuerr(e, "read weights");
    prop_unpack(prop->L, flat.data(), weights);
    if (step) *step = prop->step;
    return HGM_OK;
}

hgm_status hgm_prop_set(hgm_prop *prop, const float *weights, int64_t step)
{
    if (!valid_prop(prop) || !weights) return set_error(HGM_EINVAL, "invalid argument");
    std::vector<float> flat;
    prop_pack(prop->L, weights, flat);
    cudaError_t e = cudaMemcpy(prop->theta, flat.data(), sizeof(float) * flat.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuerr(e, "write weights");
    const size_t bytes = sizeof(float) * (size_t)prop->L.n;
    if ((e = cudaMemset(prop->m, 0, bytes)) || (e = cudaMemset(prop->v, 0, bytes))) return cuerr(e, "reset moments");
    prop->step = step;
    return HGM_OK;
}

hgm_status hgm_prop_forward(hgm_prop *prop, const float *X, int32_t B, void *stream, float *logits)
{
    std::lock_guard<std::mutex> lk(g_prop_mu);
    if (!valid_prop(prop) || B < 1 || !is_dev(X) || !is_dev(logits)) return set_error(HGM_EINVAL, "invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = prop->train.ensure(prop->L, B))) return cuerr(e, "workspace");
    if ((e = prop_forward(prop->L, prop->theta, prop->train, X, prop->L.d_in, B, st))) return cuerr(e, "forward");
    if ((e = cudaMemcpyAsync(logits, prop->train.z3, sizeof(float) * B, cudaMemcpyDeviceToDevice, st)))
        return cuerr(e, "copy");
    return check_status(prop, st);
}

hgm_status hgm_prop_gradients(hgm_prop *prop, const float *X, const float *y, int32_t B, void *stream, float *loss,
                              float *grad)
{
    std::lock_guard<std::mutex> lk(g_prop_mu);
    if (!valid_prop(prop) || B < 1 || !is_dev(X) || !is_dev(y) || !grad)
        return set_error(HGM_EINVAL, "invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = prop->train.ensure(prop->L, B))) return cuerr(e, "workspace");
    if ((e = prop_forward(prop->L, prop->theta, prop->train, X, prop->L.d_in, B, st))) return cuerr(e, "forward");
    if ((e = prop_backward(prop->L, prop->theta, prop->train, X, prop->L.d_in, y, B, prop->grad, st)))
        return cuerr(e, "backward");
    hgm_status rc = check_status(prop, st);
    if (rc) return rc;
    std::vector<float> flat((size_t)prop->L.n);
    if ((e = cudaMemcpy(flat.data(), prop->grad, sizeof(float) * flat.size(), cudaMemcpyDeviceToHost)))
        return cuerr(e, "read gradients");
    prop_unpack(prop->L, flat.data(), grad);
    if (loss && (e = cudaMemcpy(loss, prop->train.loss, sizeof(float), cudaMemcpyDeviceToHost)))
        return cuerr(e, "read loss");
    return HGM_OK;
}

hgm_status hgm_prop_train_step(hgm_prop *prop, const float *X, const float *y, int32_t B, float lr, void *stream,
                               float *loss)
{
    std::lock_guard<std::mutex> lk(g_prop_mu);
    if (!valid_prop(prop) || B < 1 || !is_dev(X) || !is_dev(y) || !(lr > 0) || !std::isfinite(lr))
        return set_error(HGM_EINVAL, "invalid argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = prop->train.ensure(prop->L, B))) return cuerr(e, "workspace");
    if ((e = prop_forward(prop->L, prop->theta, prop->train, X, prop->L.d_in, B, st))) return cuerr(e, "forward");
    if ((e = prop_backward(prop->L, prop->theta, prop->train, X, prop->L.d_in, y, B, prop->grad, st)))
        return cuerr(e, "backward");
    prop->step += 1;
    if ((e = prop_adam(prop->L, prop->theta, prop->grad, prop->m, prop->v, prop->step, lr, st))) return cuerr(e, "adam");
    if (loss) {
        if ((e = cudaMemcpyAsync(loss, prop->train.loss, sizeof(float), is_dev(loss) ? cudaMemcpyDeviceToDevice
                                                                                          : cudaMemcpyDeviceToHost, st)))
            return cuerr(e, "loss");
    }
    return HGM_OK;
}

}  // extern "C"
