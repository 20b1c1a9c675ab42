// k_recurse_small.cu -- kernel (b) for short candidate lists (the pruned form: K' <= 16).
//
// Same recursion as k_recurse.cu (Eqs. 10-13, readings R1-R6) for lists of at
// most KS candidates. With K' = 8 a step has 64 cells of 8 candidates each, so
// a whole CTA per unit would idle: here one warp owns a unit, lanes own cells
// (b, c), each lane minimises over a in slot order, and the warp steps i with
// __syncwarp only. Every value is computed with the same FP32 operations in
// the same order as the large-list kernel (fast_atan2 directions, wrap, the
// two circular folds, sqrt.approx, fma), so both kernels give the same bits.
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
    float thab[KS * KS];            // theta(b->a) at a*KS+b
    float thac[KS * KS];            // theta(a->c) at a*KS+c
};

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
    constexpr int CELLS = KS * KS;
    constexpr int PER = (CELLS + 31) / 32;
    const int K = p.K, T = p.T;
    const float lam2 = p.lambda2, lam23 = p.lambda2 * p.lambda3;

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
            const float2 mi = md.xy[i], mj = md.xy[i - 1], mk = md.xy[i - 2];
            const float A1 = signed_angle(mj, mi, mk);
            const float A2 = signed_angle(mi, mj, mk);
            const float k2 = wrap_pi(__fadd_rn(__fsub_rn(A2, A1), kPi));
            const float k2c = wrap_pi(__fsub_rn(k2, kPi));   // a and b at the same position (reading R1)
            const int dt_ab = md.t[i] - md.t[i - 1], dt_bc = md.t[i - 1] - md.t[i - 2];
            for (int e = lane; e < CELLS; e += 32) {
                const int a = e / KS, x = e % KS;
                float th = 0.0f, tr = kInf;
                if (a < na && x < nb) th = direction(sm.xy[sb][x], sm.xy[sa][a]);                  // theta(b->a)
                if (a < na && x < nc && !(T > 0 && sm.t[sa][a] - sm.t[scc][x] >= T) && sm.idx[sa][a] != sm.idx[scc][x])
                    tr = direction(sm.xy[sa][a], sm.xy[scc][x]);                                    // theta(a->c)
                sm.thab[a * KS + x] = th;
                sm.thac[a * KS + x] = tr;
            }
            __syncwarp();
            float out_al[PER];
            int out_cell[PER];
            uint8_t *bstep = ubeta + (int64_t)(i - 2) * K * K;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int e = lane + 32 * q;
                out_cell[q] = -1;
                if (e >= CELLS) continue;
                const int b = e / KS, c = e % KS;
                if (b >= nb || c >= nc) continue;
                out_cell[q] = e;
                const int tb = sm.t[sb][b], ib = sm.idx[sb][b];
                const float2 pb = sm.xy[sb][b];
                float best = kInf;
                int arg = kNoSlot;
                if (sm.t[scc][c] <= tb && sm.idx[scc][c] != ib) {
                    const float q1 = direction(pb, sm.xy[scc][c]);
                    for (int a = 0; a < na; ++a) {
                        const int ta = sm.t[sa][a];
                        if (ta < tb || sm.idx[sa][a] == ib) continue;
                        const float base = base_cost(sm.u[sa][a], lam2, dt_ab, ta, tb, sm.alpha[b * AS + a]);
                        const float p1 = wrap_pi(__fadd_rn(A1, sm.thab[a * KS + b]));
                        const float2 pa = sm.xy[sa][a];
                        const float p2 = __fadd_rn(p1, pa.x == pb.x && pa.y == pb.y ? k2c : k2);
                        const float v = triple_cost(base, p1, p2, q1, sm.thac[a * KS + c], lam23);
                        if (v < best) { best = v; arg = a; }
                    }
                }
                out_al[q] = kInf;
                if (best < kInf) out_al[q] = cell_alpha(best, lam2, dt_bc, tb, sm.t[scc][c]);
                bstep[b * K + c] = (uint8_t)(best < kInf ? arg : kNoSlot);
            }
            __syncwarp();   // every lane has read alpha_{i+1}
#pragma unroll
            for (int q = 0; q < PER; ++q)
                if (out_cell[q] >= 0) {
                    const int b = out_cell[q] / KS, c = out_cell[q] % KS;
                    sm.alpha[c * AS + b] = out_al[q];
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
