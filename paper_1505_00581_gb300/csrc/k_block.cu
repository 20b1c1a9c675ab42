// k_block.cu -- the whole-block problem: every scene point is a candidate of every model point (the
// paper's own formulation, Sec. 2.2 and Sec. 3), no time offsets. The trellis of Eq. 10 is S x S per
// step; causality and temporal closeness (Eqs. 7-8) restrict z_{i-2} to the points of the T frames up
// to z_{i-1}'s (the band of Sec. 3.3), and z_i to the frames [t'(z_{i-1}), t'(z_{i-2}) + T) through the
// minnode table (Sec. 3.5).
//
// Band layout (per scene, shared by every model matched against it): point b owns the cells (b, c) for
// c in [lo(b), hi(b)), lo(b) = minnode(t'(b) - T + 1), hi(b) = minnode(t'(b) + 1); the cell (b, b) is
// kept (always +inf) so that a cell's index is cs(b) + c - lo(b). Per cell the table holds theta(b->c)
// and theta(c->b), computed once per scene.
//
// One CTA per (model, scene) unit, persistent over units. alpha_{i+1} and alpha_i live in shared memory
// when two band tables fit, else in a per-CTA global scratch (L2-resident for the sizes this form
// serves). The argmin of every cell is stored as a 16-bit offset from minnode(t'(b)). The CTA finds the
// initial pair (Eq. 13) by a block-wide reduction and backtracks (Eq. 12) itself.
#include "hgm_internal.cuh"
#include "recurse_common.cuh"

namespace hgm {
namespace {

constexpr int kBlockThreads = 256;       // many units: several CTAs per SM
constexpr int kBlockThreadsWide = 1024;  // fewer units than SMs: one wide CTA per unit (latency-bound steps)

__global__ void block_cells_kernel(const int64_t *__restrict__ cs, int S, int32_t *__restrict__ cellb)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < S; b += gridDim.x * blockDim.x)
        for (int64_t k = cs[b]; k < cs[b + 1]; ++k) cellb[k] = b;
}

__global__ void block_dirs_kernel(const float2 *__restrict__ xy, const int32_t *__restrict__ lo,
                                  const int64_t *__restrict__ cs, const int32_t *__restrict__ cellb, int64_t cells,
                                  float *__restrict__ dirf, float *__restrict__ dirb)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cells; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = cellb[k];
        const int c = lo[b] + (int)(k - cs[b]);
        dirf[k] = direction(xy[b], xy[c]);
        dirb[k] = direction(xy[c], xy[b]);
    }
}

struct InitBest {
    float v;
    int c, b;
};

// (v, c, b) ordered by v, then by the slot of z_1 (= c), then of z_2 (= b): Eq. 13 with reading R6.
__device__ __forceinline__ bool init_better(float v, int c, int b, const InitBest &o)
{
    if (v != o.v) return v < o.v;
    if (c != o.c) return c < o.c;
    return b < o.b;
}

template <bool kSmem, int NT>
__global__ void __launch_bounds__(NT, 1) block_recurse_kernel(
    const BlockUnit *__restrict__ units, int n_units, const ModelRec *__restrict__ models,
    const SceneRec *__restrict__ scenes, const BlockGeo *__restrict__ geos, Params p, uint16_t *__restrict__ beta,
    float *__restrict__ scratch, int64_t scratch_cells, float *__restrict__ energy, int32_t *__restrict__ assign)
{
    extern __shared__ float sm[];
    __shared__ InitBest red[NT / 32];
    const float lam2 = p.lambda2, lam23 = __fmul_rn(p.lambda2, p.lambda3);
    const float inf = __int_as_float(0x7f800000);
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const BlockUnit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const BlockGeo g = geos[un.scene];
        const int64_t C = g.cells;
        float *an = kSmem ? sm : scratch + (int64_t)blockIdx.x * 2 * scratch_cells;
        float *ac = kSmem ? sm + C : an + scratch_cells;
        const int M = md.M;
        for (int i = M - 1; i >= 2; --i) {
            const float2 mi = md.xy[i], mj = md.xy[i - 1], mk = md.xy[i - 2];
            const float A1 = signed_angle(mj, mi, mk);   // at i-1, from ->i to ->i-2
            const float A2 = signed_angle(mi, mj, mk);   // at i, from ->i-1 to ->i-2
            const int dt1 = md.t[i] - md.t[i - 1], dt2 = md.t[i - 1] - md.t[i - 2];
            const float *Ui = sc.U + (int64_t)(md.urow + i) * sc.upitch;
            uint16_t *bt = beta + un.beta + (int64_t)(i - 2) * C;
            const bool last = i == M - 1;
            for (int64_t cell = threadIdx.x; cell < C; cell += blockDim.x) {
                const int b = g.cellb[cell];
                const int c = g.lo[b] + (int)(cell - g.cs[b]);
                float best = inf;
                int arg = 0xffff;
                if (c != b) {
                    const int tb = sc.t[b], tc = sc.t[c];
                    const int a0 = sc.frame_start[tb];
                    const int a1 = p.T > 0 ? sc.frame_start[min(tc + p.T, sc.n_frames)] : sc.S;
                    const float q1 = g.dirf[cell];                      // theta(b->c)
                    for (int a = a0; a < a1; ++a) {
                        if (a == b || a == c) continue;
                        const int64_t ca = g.cs[a] - g.lo[a];
                        const int64_t cab = ca + b, cac = ca + c;
                        const float alpha = last ? 0.0f : an[cab];
                        const float base = base_cost(__ldg(Ui + a), lam2, dt1, sc.t[a], tb, alpha);
                        const float p1 = __fadd_rn(A1, g.dirb[cab]);     // A1 + theta(b->a)
                        const float p2 = __fadd_rn(A2, g.dirf[cab]);     // A2 + theta(a->b)
                        const float v = triple_cost(base, p1, p2, q1, g.dirf[cac], lam23);
                        if (v < best) {
                            best = v;
                            arg = a - a0;
                        }
                    }
                    if (best < inf) best = cell_alpha(best, lam2, dt2, tb, tc);
                }
                ac[cell] = best;
                bt[cell] = (uint16_t)arg;
            }
            __syncthreads();
            float *tmp = an;
            an = ac;
            ac = tmp;
        }
        // Eq. 13: (z_1, z_2) = argmin U_1(z_1) + U_2(z_2) + alpha_3(z_2, z_1) over the cells (b = z_2, c = z_1)
        const float *U0 = sc.U + (int64_t)md.urow * sc.upitch;
        const float *U1 = U0 + sc.upitch;
        InitBest mine{inf, 0x7fffffff, 0x7fffffff};
        for (int64_t cell = threadIdx.x; cell < C; cell += blockDim.x) {
            const float al = an[cell];
            if (!(al < inf)) continue;
            const int b = g.cellb[cell];
            const int c = g.lo[b] + (int)(cell - g.cs[b]);
            const float v = __fadd_rn(__fadd_rn(__ldg(U0 + c), __ldg(U1 + b)), al);
            if (init_better(v, c, b, mine)) mine = InitBest{v, c, b};
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            InitBest o{__shfl_xor_sync(0xffffffffu, mine.v, off), __shfl_xor_sync(0xffffffffu, mine.c, off),
                       __shfl_xor_sync(0xffffffffu, mine.b, off)};
            if (init_better(o.v, o.c, o.b, mine)) mine = o;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            InitBest best = red[0];
            for (int w = 1; w < NT / 32; ++w)
                if (init_better(red[w].v, red[w].c, red[w].b, best)) best = red[w];
            int32_t *row = assign + un.out_a;
            if (best.v < inf) {
                // Eq. 12: z_i = beta_i(z_{i-1}, z_{i-2})
                int z2 = best.c, z1 = best.b;   // z_{i-2}, z_{i-1}
                row[md.perm[0]] = sc.perm[z2];
                row[md.perm[1]] = sc.perm[z1];
                for (int i = 2; i < M; ++i) {
                    const int64_t cell = g.cs[z1] + (z2 - g.lo[z1]);
                    const int za = sc.frame_start[sc.t[z1]] + beta[un.beta + (int64_t)(i - 2) * C + cell];
                    row[md.perm[i]] = sc.perm[za];
                    z2 = z1;
                    z1 = za;
                }
                energy[un.out_e] = best.v;
            } else {
                for (int i = 0; i < M; ++i) row[i] = -1;
                energy[un.out_e] = inf;
            }
        }
        __syncthreads();   // the reduction slots and the alpha tables are reused by the next unit
    }
}

}  // namespace

cudaError_t launch_block_geo(const float2 *xy, int S, const int32_t *lo, const int64_t *cs, int64_t cells,
                             int32_t *cellb, float *dirf, float *dirb, cudaStream_t st)
{
    if (S <= 0 || cells <= 0) return cudaSuccess;
    block_cells_kernel<<<(S + 255) / 256, 256, 0, st>>>(cs, S, cellb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    block_dirs_kernel<<<(unsigned)std::min<int64_t>((cells + 255) / 256, 8192), 256, 0, st>>>(xy, lo, cs, cellb,
                                                                                           cells, dirf, dirb);
    return cudaGetLastError();
}

int64_t block_smem_cells()
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    const int64_t avail = (int64_t)optin - (int64_t)sizeof(InitBest) * (kBlockThreadsWide / 32) - 1024;
    return avail > 0 ? avail / (2 * (int64_t)sizeof(float)) : 0;
}

cudaError_t launch_block_recurse(const BlockUnit *units, int n_units, const ModelRec *models, const SceneRec *scenes,
                                 const BlockGeo *geos, Params p, int64_t max_cells, uint16_t *beta, float *scratch,
                                 int grid_global, float *energy, int32_t *assign, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    prof_begin(kProfRecurse, st);
    const bool wide = n_units < sms;
    if (scratch == nullptr) {
        const size_t smem = (size_t)max_cells * 2 * sizeof(float);
        auto kern = wide ? block_recurse_kernel<true, kBlockThreadsWide> : block_recurse_kernel<true, kBlockThreads>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            const int grid = std::min(n_units, sms * 8);
            kern<<<grid, wide ? kBlockThreadsWide : kBlockThreads, smem, st>>>(units, n_units, models, scenes, geos, p,
                                                                                beta, nullptr, 0, energy, assign);
            e = cudaGetLastError();
        }
    } else {
        auto kern = wide ? block_recurse_kernel<false, kBlockThreadsWide> : block_recurse_kernel<false, kBlockThreads>;
        kern<<<grid_global, wide ? kBlockThreadsWide : kBlockThreads, 0, st>>>(units, n_units, models, scenes, geos, p,
                                                                                beta, scratch, max_cells, energy,
                                                                                assign);
        e = cudaGetLastError();
    }
    prof_end(kProfRecurse, st);
    return e;
}

}  // namespace hgm
