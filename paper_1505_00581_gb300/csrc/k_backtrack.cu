// k_backtrack.cu -- kernel (c): backtracking (Eq. 12), plus the triple counter.
//
// Backtracking starts from the initial pair (z_1, z_2) of Eq. 13 that kernel
// (b) stored per unit and follows z_i = beta_i(z_{i-1}, z_{i-2}) through the
// byte tables kernel (b) left in global memory. The paper does this step on
// the CPU after copying the trellis back (Sec. 3.7); here it stays on the GPU
// and only energies and assignments leave the device. Slots are mapped to
// sorted scene indices through the unit's candidate lists, then to the
// caller's scene indices, and written in the caller's model order.
#include "backtrack.cuh"
#include "hgm_internal.cuh"

namespace hgm {
namespace {

__global__ void backtrack_kernel(const Unit *__restrict__ units, int64_t n_units,
                                 const ModelRec *__restrict__ models, const SceneRec *__restrict__ scenes,
                                 Params p, const int32_t *__restrict__ cand_idx, const uint8_t *__restrict__ beta,
                                 const UnitResult *__restrict__ res, float *__restrict__ energy,
                                 int32_t *__restrict__ assign)
{
    const int K = p.K;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_units;
         u += (int64_t)gridDim.x * blockDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        backtrack_unit(un, md, sc, K, cand_idx + un.cand, beta + un.beta, res[u], energy, assign);
    }
}

// Feasible triples per unit, by direct enumeration over the candidate lists
// (reading of Eqs. 7-8 with distinct points). Work accounting only.
__global__ void count_kernel(const Unit *__restrict__ units, int64_t n_units, const ModelRec *__restrict__ models,
                             const SceneRec *__restrict__ scenes, Params p, const int32_t *__restrict__ cand_idx,
                             const int32_t *__restrict__ cand_cnt, int64_t *__restrict__ triples)
{
    __shared__ unsigned long long acc;
    const int K = p.K;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        if (threadIdx.x == 0) acc = 0;
        __syncthreads();
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int32_t *cidx = cand_idx + un.cand;
        const int32_t *ccnt = cand_cnt + un.cand / K;
        unsigned long long mine = 0;
        for (int i = 2; i < md.M; ++i) {
            const int na = ccnt[i], nb = ccnt[i - 1], nc = ccnt[i - 2];
            for (int e = threadIdx.x; e < nb * nc; e += blockDim.x) {
                int jb = cidx[(int64_t)(i - 1) * K + e / nc];
                int jc = cidx[(int64_t)(i - 2) * K + e % nc];
                int tb = sc.t[jb], tc = sc.t[jc];
                if (jb == jc || tc > tb) continue;
                for (int a = 0; a < na; ++a) {
                    int ja = cidx[(int64_t)i * K + a];
                    int ta = sc.t[ja];
                    if (ja == jb || ja == jc || ta < tb) continue;
                    if (p.T > 0 && ta - tc >= p.T) continue;
                    ++mine;
                }
            }
        }
        atomicAdd(&acc, mine);
        __syncthreads();
        if (threadIdx.x == 0) triples[un.out_e] = (int64_t)acc;
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_backtrack(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                             Params p, const int32_t *cand_idx, const uint8_t *beta, const UnitResult *res,
                             float *energy, int32_t *assign, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    int64_t blocks = (n_units + 127) / 128;
    if (blocks > 65535 * 16) blocks = 65535 * 16;
    prof_begin(kProfBacktrack, st);
    backtrack_kernel<<<(unsigned)blocks, 128, 0, st>>>(units, n_units, models, scenes, p, cand_idx, beta, res,
                                                       energy, assign);
    prof_end(kProfBacktrack, st);
    return cudaGetLastError();
}

cudaError_t launch_count(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                         Params p, const int32_t *cand_idx, const int32_t *cand_cnt, int64_t *triples,
                         cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    int64_t blocks = n_units < (1 << 20) ? n_units : (1 << 20);
    count_kernel<<<(unsigned)blocks, 256, 0, st>>>(units, n_units, models, scenes, p, cand_idx, cand_cnt, triples);
    return cudaGetLastError();
}

cudaError_t preload_backtrack()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, backtrack_kernel);
}

}  // namespace hgm
