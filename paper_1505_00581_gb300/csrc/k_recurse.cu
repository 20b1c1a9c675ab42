// k_recurse.cu -- kernel (b): the exact second-order min-sum recursion.
//
// For one unit (model, scene, offset), with lists A = C_i, B = C_{i-1},
// C = C_{i-2} (0-based chain index i = M-1 .. 2, the paper's i+1), Eq. 10:
//   alpha_i(b,c) = min_{a in A feasible} [ U(a) + D(a,b,c) + alpha_{i+1}(a,b) ]
// with alpha_{M+1} = 0 (Eq. 11), the argmin kept in beta_i(b,c) (Eq. 12),
// and finally the initial pair search of Eq. 13 over alpha_3.
//
// GB300 design (differs from the paper's one-launch-per-i OpenCL kernel with
// the CPU as global barrier, Sec. 3.1): one CTA owns a whole unit for its
// lifetime and steps i with CTA barriers; CTAs are persistent and take units
// from a global counter in decreasing-size order. Everything a step touches
// lives in shared memory (Sec. 3.5's local-memory rows, extended to the
// whole alpha_{i+1} table and the geometry):
//   sAB[a][b] = (U(a) + lambda2*Delta(i,i-1) + alpha_{i+1}(a,b),  wrap(A1 + theta(b->a)))
//   sR [a][c] = theta(a->c)
//   per cell (b,c) in registers: theta(b->c)
// where theta(p->q) = atan2(q-p) and A1, A2 are the model's angles at i-1 and
// at i. The angle differences of Eq. 6 become
//   d1 = wrap(A1 + theta(b->a) - theta(b->c)),  d2 = wrap(A2 + theta(a->b) - theta(a->c))
// so a triple costs two subtractions, two circular folds, one FMA for the
// squared norm, one square root and one FMA -- every pair-only term is hoisted
// into the tables (Sec. 3.3's look-up idea applied to the geometry too).
// Infeasible pairs carry +inf in the tables (causality t'(c)<=t'(b)<=t'(a),
// closeness t'(a)-t'(c) < T, distinct points; Eqs. 7-8, Sec. 3.2's validity
// mask) and the a-loop starts at the first a with t'(a) >= t'(b) (Sec. 3.4's
// minnode bound on a list sorted by frame).
//
// Work split per step: tiles of one b and CT consecutive c (a register tile),
// only for c with t'(c) <= t'(b), flattened across the CTA's threads. Each
// thread loops a in increasing slot order with a strict '<', so the lowest
// slot wins exact ties, as in the oracle.
#include "hgm_internal.cuh"

namespace hgm {
namespace {

constexpr float kInf = __builtin_huge_valf();

__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float wrap_pi(float v)
{
    // argument in [-3pi, 3pi]: one fold to [-pi, pi]
    if (v > kPi) v -= kTwoPi;
    else if (v < -kPi) v += kTwoPi;
    return v;
}

template <int KM>
struct List {
    float2 xy[KM];
    int32_t t[KM];
    float u[KM];
    int32_t idx[KM];
    int32_t n;
};

template <int KM, int NT, int CT>
struct Smem {
    static constexpr int RS = KM + 4;     // row stride of sR (bank skew, 16-byte rows)
    float2 ab[KM * KM];                   // (base, p1) indexed a*KM + b
    float r[KM * RS];                     // theta(a->c), indexed a*RS + c
    float alpha[KM * KM];                 // alpha_{i+1}(a,b) at a*KM+b; alpha_i(b,c) written at b*KM+c
    List<KM> list[3];
    int32_t lo[KM];                       // first a with t'(a) >= t'(b)
    int32_t pre[KM + 1];                  // tile prefix over b
    float red_v[NT / 32];
    int32_t red_k[NT / 32];
    int32_t unit;
};

template <int KM>
__device__ void load_list(List<KM> &L, const SceneRec &sc, const int32_t *cidx, const float *cu, int n,
                          int tid, int nt)
{
    for (int k = tid; k < KM; k += nt) {
        if (k < n) {
            int j = cidx[k];
            L.idx[k] = j;
            L.xy[k] = sc.xy[j];
            L.t[k] = sc.t[j];
            L.u[k] = cu[k];
        } else {
            L.idx[k] = -1;
            L.xy[k] = make_float2(0.f, 0.f);
            L.t[k] = 0x3fffffff;
            L.u[k] = kInf;
        }
    }
    if (tid == 0) L.n = n;
}

__device__ __forceinline__ float model_angle(float2 v, float2 p, float2 q)
{
    // signed angle at v from v->p to v->q (reading R1), wrapped to [-pi, pi]
    float a = atan2f(q.y - v.y, q.x - v.x) - atan2f(p.y - v.y, p.x - v.x);
    return wrap_pi(a);
}

template <int KM, int NT, int CT>
__global__ void __launch_bounds__(NT) recurse_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                     const ModelRec *__restrict__ models,
                                                     const SceneRec *__restrict__ scenes, Params p,
                                                     const int32_t *__restrict__ cand_idx,
                                                     const float *__restrict__ cand_u,
                                                     const int32_t *__restrict__ cand_cnt,
                                                     uint8_t *__restrict__ beta, UnitResult *__restrict__ res,
                                                     int *__restrict__ work_counter)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<KM, NT, CT> &sm = *reinterpret_cast<Smem<KM, NT, CT> *>(smem_raw);
    constexpr int RS = Smem<KM, NT, CT>::RS;
    const int tid = threadIdx.x;
    const int K = p.K;
    const float lam2 = p.lambda2;
    const float lam23 = p.lambda2 * p.lambda3;

    for (;;) {
        if (tid == 0) sm.unit = atomicAdd(work_counter, 1);
        __syncthreads();
        const int64_t u = sm.unit;
        if (u >= n_units) break;
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int32_t *cidx = cand_idx + un.cand;
        const float *cu = cand_u + un.cand;
        const int32_t *ccnt = cand_cnt + un.cand / K;
        uint8_t *ubeta = beta + un.beta;

        // alpha_{M+1} == 0 (Eq. 11)
        for (int e = tid; e < KM * KM; e += NT) sm.alpha[e] = 0.0f;
        load_list<KM>(sm.list[(M - 1) % 3], sc, cidx + (int64_t)(M - 1) * K, cu + (int64_t)(M - 1) * K,
                      ccnt[M - 1], tid, NT);
        load_list<KM>(sm.list[(M - 2) % 3], sc, cidx + (int64_t)(M - 2) * K, cu + (int64_t)(M - 2) * K,
                      ccnt[M - 2], tid, NT);

        for (int i = M - 1; i >= 2; --i) {
            List<KM> &LA = sm.list[i % 3];
            List<KM> &LB = sm.list[(i - 1) % 3];
            List<KM> &LC = sm.list[(i - 2) % 3];
            load_list<KM>(LC, sc, cidx + (int64_t)(i - 2) * K, cu + (int64_t)(i - 2) * K, ccnt[i - 2], tid, NT);
            __syncthreads();
            const int na = LA.n, nb = LB.n, nc = LC.n;

            // per-b loop bound and number of c-tiles (c with t'(c) <= t'(b) form a prefix)
            if (tid < KM) {
                int b = tid, lo = 0, nq = 0;
                if (b < nb) {
                    int tb = LB.t[b];
                    while (lo < na && LA.t[lo] < tb) ++lo;
                    int cc = 0;
                    while (cc < nc && LC.t[cc] <= tb) ++cc;
                    nq = (cc + CT - 1) / CT;
                }
                sm.lo[b] = lo;
                sm.pre[b + 1] = nq;
            }
            // model geometry of hyperedge (i, i-1, i-2)
            const float2 mi = md.xy[i], mj = md.xy[i - 1], mk = md.xy[i - 2];
            const float A1 = model_angle(mj, mi, mk);   // at i-1, from ->i to ->i-2
            const float A2 = model_angle(mi, mj, mk);   // at i, from ->i-1 to ->i-2
            const float k2 = wrap_pi(A2 - A1 + kPi);    // p2 = p1 + k2 (mod 2pi)
            const int dt_ab = md.t[i] - md.t[i - 1];
            const int dt_bc = md.t[i - 1] - md.t[i - 2];
            __syncthreads();
            if (tid < 32) {
                // exclusive scan of tile counts over b (KM <= 64: two per lane)
                int v0 = (2 * tid + 1 <= KM) ? sm.pre[2 * tid + 1] : 0;
                int v1 = (2 * tid + 2 <= KM) ? sm.pre[2 * tid + 2] : 0;
                int s = v0 + v1, incl = s;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    int w = __shfl_up_sync(0xffffffffu, incl, off);
                    if (tid >= off) incl += w;
                }
                int excl = incl - s;
                if (2 * tid + 1 <= KM) sm.pre[2 * tid + 1] = excl + v0;
                if (2 * tid + 2 <= KM) sm.pre[2 * tid + 2] = excl + v0 + v1;
                if (tid == 0) sm.pre[0] = 0;
            }
            // tables
            for (int e = tid; e < KM * KM; e += NT) {
                int a = e / KM, b = e % KM;
                if (a < na && b < nb) {
                    float2 pa = LA.xy[a], pb = LB.xy[b];
                    float th = atan2f(pa.y - pb.y, pa.x - pb.x);            // theta(b->a)
                    float p1 = wrap_pi(A1 + th);
                    int ta = LA.t[a], tb = LB.t[b];
                    float base = kInf;
                    if (ta >= tb && LA.idx[a] != LB.idx[b]) {
                        float dt = fabsf((float)(dt_ab - (ta - tb)));
                        base = LA.u[a] + lam2 * dt + sm.alpha[a * KM + b];
                    }
                    sm.ab[a * KM + b] = make_float2(base, p1);
                }
                int c = b;
                if (a < na && c < nc) {
                    int ta = LA.t[a], tc = LC.t[c];
                    float r = kInf;
                    if (!(p.T > 0 && ta - tc >= p.T) && LA.idx[a] != LC.idx[c]) {
                        float2 pa = LA.xy[a], pc = LC.xy[c];
                        r = atan2f(pc.y - pa.y, pc.x - pa.x);               // theta(a->c)
                    }
                    sm.r[a * RS + c] = r;
                } else if (a < KM && c < KM) {
                    sm.r[a * RS + c] = kInf;
                }
            }
            __syncthreads();

            const int ntile = nb > 0 ? sm.pre[nb] : 0;
            uint8_t *bstep = ubeta + (int64_t)(i - 2) * K * K;
            for (int tile = tid; tile < ntile; tile += NT) {
                // b = last index with pre[b] <= tile
                int lo_b = 0, hi_b = nb;
                while (hi_b - lo_b > 1) {
                    int mid = (lo_b + hi_b) >> 1;
                    if (sm.pre[mid] <= tile) lo_b = mid; else hi_b = mid;
                }
                const int b = lo_b;
                const int c0 = (tile - sm.pre[b]) * CT;
                const float2 pb = LB.xy[b];
                const int tb = LB.t[b];
                const int ib = LB.idx[b];
                float q1[CT], best[CT];
                int arg[CT];
#pragma unroll
                for (int k = 0; k < CT; ++k) {
                    int c = c0 + k;
                    bool ok = c < nc && LC.t[c] <= tb && LC.idx[c] != ib;
                    q1[k] = ok ? atan2f(LC.xy[c].y - pb.y, LC.xy[c].x - pb.x) : kInf;   // theta(b->c)
                    best[k] = kInf;
                    arg[k] = kNoSlot;
                }
                for (int a = sm.lo[b]; a < na; ++a) {
                    const float2 abv = sm.ab[a * KM + b];
                    const float p2 = abv.y + k2;
                    float rv[CT];
                    if constexpr (CT == 4) {
                        float4 r4 = *reinterpret_cast<const float4 *>(&sm.r[a * RS + c0]);
                        rv[0] = r4.x; rv[1] = r4.y; rv[2] = r4.z; rv[3] = r4.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < CT; ++k) rv[k] = sm.r[a * RS + c0 + k];
                    }
#pragma unroll
                    for (int k = 0; k < CT; ++k) {
                        float d1 = abv.y - q1[k];
                        float d2 = p2 - rv[k];
                        float w1 = fminf(fabsf(d1), kTwoPi - fabsf(d1));
                        float w2 = fminf(fabsf(d2), kTwoPi - fabsf(d2));
                        float s = fmaf(w2, w2, w1 * w1);
                        float v = fmaf(lam23, sqrt_fast(s), abv.x);
                        if (v < best[k]) { best[k] = v; arg[k] = a; }
                    }
                }
#pragma unroll
                for (int k = 0; k < CT; ++k) {
                    int c = c0 + k;
                    if (c < nc) {
                        float al = kInf;
                        int bt = kNoSlot;
                        if (best[k] < kInf) {
                            float dt = fabsf((float)(dt_bc - (tb - LC.t[c])));
                            al = best[k] + lam2 * dt;
                            bt = arg[k];
                        }
                        sm.alpha[b * KM + c] = al;
                        bstep[b * K + c] = (uint8_t)bt;
                    }
                }
            }
            // cells (b, c) beyond the tiled prefix are infeasible
            for (int e = tid; e < KM * KM; e += NT) {
                int b = e / KM, c = e % KM;
                if (b < nb && c < nc) {
                    int covered = (sm.pre[b + 1] - sm.pre[b]) * CT;
                    if (c >= covered) {
                        sm.alpha[b * KM + c] = kInf;
                        bstep[b * K + c] = (uint8_t)kNoSlot;
                    }
                }
            }
            __syncthreads();
        }

        // Eq. 13: (z_1, z_2) = argmin U(z_1) + U(z_2) + alpha_3(z_2, z_1); ties -> lowest (z_1, z_2)
        {
            const List<KM> &L0 = sm.list[0];
            const List<KM> &L1 = sm.list[1];
            const int n0 = L0.n, n1 = L1.n;
            float bv = kInf;
            int bk = 0x7fffffff;
            for (int e = tid; e < KM * KM; e += NT) {
                int c = e / KM, b = e % KM;    // e = z1 * KM + z2: lexicographic order
                if (c < n0 && b < n1) {
                    float v = L0.u[c] + L1.u[b] + sm.alpha[b * KM + c];
                    if (v < bv || (v == bv && e < bk)) { bv = v; bk = e; }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, bv, off);
                int ok = __shfl_xor_sync(0xffffffffu, bk, off);
                if (ov < bv || (ov == bv && ok < bk)) { bv = ov; bk = ok; }
            }
            if ((tid & 31) == 0) { sm.red_v[tid >> 5] = bv; sm.red_k[tid >> 5] = bk; }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < NT / 32; ++w) {
                    float ov = sm.red_v[w];
                    int ok = sm.red_k[w];
                    if (ov < bv || (ov == bv && ok < bk)) { bv = ov; bk = ok; }
                }
                sm.red_v[0] = bv; sm.red_k[0] = bk;
                UnitResult r;
                r.pad = 0;
                if (bv < kInf) {
                    r.energy = bv;
                    r.z1 = bk / KM;
                    r.z2 = bk % KM;
                } else {
                    r.energy = kInf;
                    r.z1 = -1;
                    r.z2 = -1;
                }
                res[u] = r;
            }
            __syncthreads();
        }
    }
}

template <int KM, int NT, int CT>
cudaError_t launch_recurse_t(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                             Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                             uint8_t *beta, UnitResult *res, int *work_counter, cudaStream_t st)
{
    auto kern = recurse_kernel<KM, NT, CT>;
    const size_t smem = sizeof(Smem<KM, NT, CT>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_units) grid = n_units;
    e = cudaMemsetAsync(work_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    prof_begin(kProfRecurse, st);
    kern<<<(unsigned)grid, NT, smem, st>>>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                                           work_counter);
    prof_end(kProfRecurse, st);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_recurse(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                           Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                           uint8_t *beta, UnitResult *res, int *work_counter, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    if (p.K <= 32)
        return launch_recurse_t<32, 128, 4>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta,
                                            res, work_counter, st);
    return launch_recurse_t<64, 256, 4>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                                        work_counter, st);
}

}  // namespace hgm
