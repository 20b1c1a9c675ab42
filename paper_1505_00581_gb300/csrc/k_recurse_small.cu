// k_recurse_small.cu -- kernel (b) for short candidate lists (the pruned form: K' <= 16).
//
// Same recursion as k_recurse.cu (Eqs. 10-13, readings R1-R6) for lists of at
// most KS candidates. With K' = 8 a step has 64 cells of 8 candidates each, so
// a whole CTA per unit would idle: here one warp owns a unit, lanes own cells
// (b, c), each lane minimises over a in slot order, and the warp steps i with
// __syncwarp only. Per step the per-(a, b) terms (base, p1, p2) and the
// theta(a->c) table are computed once by the warp; then a lane owns CT
// consecutive cells of one b and minimises over a in slot order. Every value
// is computed with the same FP32 operations in the same order as the
// large-list kernel (fast_atan2 directions, wrap, the two circular folds,
// sqrt.approx, fma; the model constants from the same per-model table), so
// both kernels give the same bits.
#include "recurse_common.cuh"

namespace hgm {
namespace {

constexpr float kInf = __builtin_huge_valf();
constexpr int kWarps = 4;

template <int KS>
struct WarpSmem {
    float2 xy[3][KS];
    int32_t t[3][KS];
    float u[3][KS];
    int32_t idx[3][KS];
    int32_t n[3];
    float alpha[KS * (KS + 1)];     // alpha_{i+1}(a,b) at b*(KS+1)+a; alpha_i(b,c) written at c*(KS+1)+b
    float4 fb[KS * KS];             // per (b, a) at b*KS+a: (base(a,b) or +inf, p1, p2, -)
    float thac[KS * (KS + 4)];      // theta(a->c) or +inf at a*(KS+4)+c (rows of whole 16-byte groups)
};

// Lanes own CT consecutive cells (b, c0 .. c0+CT-1) of one b: the per-(a, b) terms are read once per a for
// CT cells, and the cells go through the packed FP32x2 arithmetic in pairs.
template <int KS>
__global__ void __launch_bounds__(kWarps * 32) recurse_small_kernel(
    const Unit *__restrict__ units, int64_t n_units, const ModelRec *__restrict__ models,
    const SceneRec *__restrict__ scenes, Params p, const int32_t *__restrict__ cand_idx,
    const float *__restrict__ cand_u, const int32_t *__restrict__ cand_cnt, uint8_t *__restrict__ beta,
    UnitResult *__restrict__ res)
{
    __shared__ WarpSmem<KS> all[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem<KS> &sm = all[warp];
    constexpr int AS = KS + 1;
    constexpr int RS = KS + 4;
    constexpr int CT = KS * KS / 32;        // cells per lane: 8 (KS = 16) or 2 (KS = 8)
    static_assert(CT % 2 == 0 && KS % CT == 0, "cells per lane");
    const int K = p.K, T = p.T;
    const float lam2 = p.lambda2, lam23 = p.lambda2 * p.lambda3;
    const int my_b = lane / (KS / CT), my_c0 = (lane % (KS / CT)) * CT;

    for (int64_t u = (int64_t)blockIdx.x * kWarps + warp; u < n_units; u += (int64_t)gridDim.x * kWarps) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int32_t *cidx = cand_idx + un.cand;
        const float *cu = cand_u + un.cand;
        const int32_t *ccnt = cand_cnt + un.cand / K;
        uint8_t *ubeta = beta + un.beta;
        auto load = [&](int slot, int i) {
            const int n = ccnt[i];
            for (int k = lane; k < KS; k += 32) {
                if (k < n) {
                    const int j = cidx[(int64_t)i * K + k];
                    sm.idx[slot][k] = j;
                    sm.xy[slot][k] = sc.xy[j];
                    sm.t[slot][k] = sc.t[j];
                    sm.u[slot][k] = cu[(int64_t)i * K + k];
                } else {
                    sm.idx[slot][k] = -1;
                    sm.xy[slot][k] = make_float2(0.f, 0.f);
                    sm.t[slot][k] = 0x3fffffff;
                    sm.u[slot][k] = kInf;
                }
            }
            if (lane == 0) sm.n[slot] = n;
        };
        for (int e = lane; e < KS * AS; e += 32) sm.alpha[e] = 0.0f;   // alpha_{M+1} = 0
        load((M - 1) % 3, M - 1);
        load((M - 2) % 3, M - 2);
        for (int i = M - 1; i >= 2; --i) {
            const int sa = i % 3, sb = (i - 1) % 3, scc = (i - 2) % 3;
            load(scc, i - 2);
            __syncwarp();
            const int na = sm.n[sa], nb = sm.n[sb], nc = sm.n[scc];
            // the model's per-step constants (A1, k2, frame differences), as the large-list kernel reads them
            const float4 g = md.geo[i];
            const float A1 = g.x, k2 = g.y;
            const float k2c = wrap_pi(__fsub_rn(k2, kPi));   // a and b at the same position (reading R1)
            const int dt_ab = __float_as_int(g.z), dt_bc = __float_as_int(g.w);
            // per (a, b): base = U(a) + lambda2 Delta + alpha_{i+1}(a,b), p1 = A1 + theta(b->a), p2 = p1 + k2;
            // per (a, c): theta(a->c), +inf where (a, c) breaks closeness or distinctness
            for (int e = lane; e < KS * KS; e += 32) {
                const int a = e % KS, x = e / KS;
                const int ta = sm.t[sa][a], ia = sm.idx[sa][a];
                const float2 pa = sm.xy[sa][a];
                float4 f = make_float4(kInf, 0.f, 0.f, 0.f);
                if (a < na && x < nb && ta >= sm.t[sb][x] && ia != sm.idx[sb][x]) {
                    const float2 pb = sm.xy[sb][x];
                    f.x = base_cost(sm.u[sa][a], lam2, dt_ab, ta, sm.t[sb][x], sm.alpha[x * AS + a]);
                    f.y = wrap_pi(__fadd_rn(A1, direction(pb, pa)));
                    f.z = __fadd_rn(f.y, pa.x == pb.x && pa.y == pb.y ? k2c : k2);
                }
                sm.fb[x * KS + a] = f;
                float tr = kInf;
                if (a < na && x < nc && !(T > 0 && ta - sm.t[scc][x] >= T) && ia != sm.idx[scc][x])
                    tr = direction(pa, sm.xy[scc][x]);
                sm.thac[a * RS + x] = tr;
            }
            __syncwarp();   // every lane has read alpha_{i+1}
            uint8_t *bstep = ubeta + (int64_t)(i - 2) * K * K;
            const int b = my_b;
            if (b < nb) {
                const int tb = sm.t[sb][b], ib = sm.idx[sb][b];
                const float2 pb = sm.xy[sb][b];
                float best[CT];
                int arg[CT];
                unsigned long long q1p[CT / 2];
#pragma unroll
                for (int q = 0; q < CT; q += 2) {
                    float q1[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int c = my_c0 + q + h;
                        q1[h] = c < nc && sm.t[scc][c] <= tb && sm.idx[scc][c] != ib ? direction(pb, sm.xy[scc][c])
                                                                                      : kInf;   // theta(b->c)
                        best[q + h] = kInf;
                        arg[q + h] = kNoSlot;
                    }
                    q1p[q / 2] = pk2(q1[0], q1[1]);
                }
                const unsigned long long lamp = pk2(lam23, lam23);
                for (int a = 0; a < na; ++a) {
                    const float4 f = sm.fb[b * KS + a];
                    if (!(f.x < kInf)) continue;      // a breaks causality or distinctness with b
                    const unsigned long long bp = pk2(f.x, f.x), p1p = pk2(f.y, f.y), p2p = pk2(f.z, f.z);
#pragma unroll
                    for (int q = 0; q < CT; q += 2) {
                        const float2 r2 = *reinterpret_cast<const float2 *>(&sm.thac[a * RS + my_c0 + q]);
                        float v0, v1;
                        triple_cost2(bp, p1p, p2p, q1p[q / 2], pk2(r2.x, r2.y), lamp, v0, v1);
                        if (v0 < best[q]) { best[q] = v0; arg[q] = a; }
                        if (v1 < best[q + 1]) { best[q + 1] = v1; arg[q + 1] = a; }
                    }
                }
#pragma unroll
                for (int q = 0; q < CT; ++q) {
                    const int c = my_c0 + q;
                    if (c < nc) {
                        const bool ok = best[q] < kInf;
                        sm.alpha[c * AS + b] = ok ? cell_alpha(best[q], lam2, dt_bc, tb, sm.t[scc][c]) : kInf;
                        bstep[b * K + c] = (uint8_t)(ok ? arg[q] : kNoSlot);
                    }
                }
            }
            __syncwarp();
        }
        // Eq. 13 over alpha_3(z_2, z_1); ties -> lowest (z_1, z_2)
        const int n0 = sm.n[0], n1 = sm.n[1];
        float bv = kInf;
        int bk = 0x7fffffff;
        for (int e = lane; e < KS * KS; e += 32) {
            const int c = e / KS, b = e % KS;
            if (c < n0 && b < n1) {
                const float v = sm.u[0][c] + sm.u[1][b] + sm.alpha[c * AS + b];
                if (v < bv || (v == bv && e < bk)) { bv = v; bk = e; }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
            const int ok = __shfl_xor_sync(0xffffffffu, bk, off);
            if (ov < bv || (ov == bv && ok < bk)) { bv = ov; bk = ok; }
        }
        if (lane == 0) {
            UnitResult r;
            r.pad = 0;
            if (bv < kInf) {
                r.energy = bv;
                r.z1 = bk / KS;
                r.z2 = bk % KS;
            } else {
                r.energy = kInf;
                r.z1 = -1;
                r.z2 = -1;
            }
            res[u] = r;
        }
        __syncwarp();
    }
}

template <int KS>
cudaError_t launch_small(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes, Params p,
                         const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt, uint8_t *beta,
                         UnitResult *res, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, recurse_small_kernel<KS>, kWarps * 32, 0)) !=
        cudaSuccess)
        return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int64_t want = (n_units + kWarps - 1) / kWarps;
    const int64_t grid = std::min<int64_t>(want, (int64_t)sms * per_sm);
    prof_begin(kProfRecurse, st);
    recurse_small_kernel<KS><<<(unsigned)grid, kWarps * 32, 0, st>>>(units, n_units, models, scenes, p, cand_idx,
                                                                     cand_u, cand_cnt, beta, res);
    prof_end(kProfRecurse, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_recurse_small(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                                 uint8_t *beta, UnitResult *res, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    if (p.K <= 8)
        return launch_small<8>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res, st);
    return launch_small<16>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res, st);
}

cudaError_t preload_recurse_small()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, recurse_small_kernel<8>);
    return e == cudaSuccess ? cudaFuncGetAttributes(&a, recurse_small_kernel<16>) : e;
}

}  // namespace hgm
