// k_prop_infer.cu -- learned pruning of the candidate lists before the recursion.
//
// For each (unit, model point i) list of up to K candidates, the proposal
// network scores every candidate j and keeps the `keep` best (ties: lower
// slot), listed in slot order (ascending scene index, as the recursion
// expects). The first layer is decomposed as
//   W1 x + b1 = (W1a f_i + b1) + W1b f'_j + W1c (dx, dy, dt)
// where the two point projections P (per model point) and Q (per scene point)
// are computed once per batch by the tensor-core row-product kernel; here each
// thread builds one candidate's 128 hidden units, the CTA stages 128 candidates
// (two lists) as BF16, and layer 2 (128 x 128) runs as tcgen05.mma with W2
// resident in shared memory and the accumulator in tensor memory. The epilogue
// applies relu(+b2), the dot with w3 (+b3) and the per-list top-keep.
#include "hgm_internal.cuh"
#include "prop.cuh"
#include "tc05.cuh"

namespace hgm {
namespace {

constexpr int H = kPropHidden;
constexpr int TM = 128;
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = (H / 8) * 128;   // K = 128 components per row
constexpr uint32_t kPolls = 1u << 26;
constexpr float kNegInf = -__builtin_huge_valf();

struct Smem {
    unsigned char a[TM * H * 2];     // hidden layer 1 of 128 candidates, BF16, canonical K-major
    unsigned char w2[H * H * 2];     // W2 (rows = output units), BF16
    float part[2][TM];               // half-sums of the last layer
    float b2[H], w3[H];
    float w1c[3][H];
    float b3;
    uint64_t mbar;
    uint32_t tslot;
    int bad;
};

__device__ __forceinline__ float exact_u(const float *a, const float *b, int F, float lambda1)
{
    float s = 0.0f;
    for (int k = 0; k < F; ++k) {
        const float d = __fsub_rn(a[k], b[k]);
        s = __fmaf_rn(d, d, s);
    }
    return __fmul_rn(lambda1, __fsqrt_rn(s));
}

// Logits of every candidate of every list: scores [n_lists x K] (-inf for empty slots).
// 256 threads: row r = tid % 128 of the tile, half = tid / 128 owns hidden units [64 half, 64 half + 64).
__global__ void __launch_bounds__(256) prop_score_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                         const ModelRec *__restrict__ models,
                                                         const SceneRec *__restrict__ scenes, Params p, PropInfer pi,
                                                         const int32_t *__restrict__ cand_idx,
                                                         const int32_t *__restrict__ cand_cnt,
                                                         float *__restrict__ scores, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (TM - 1), half = tid >> 7;
    const int K = p.K;

    if (warp == 0) tc05::tmem_alloc<H>(&sm.tslot);
    for (int e = tid; e < H * (H / 8); e += 256) {          // W2 -> BF16, canonical layout
        const int r = e / (H / 8), k = (e % (H / 8)) * 8;
        __align__(16) __nv_bfloat162 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            h[q] = __floats2bfloat162_rn(pi.W2[r * H + k + 2 * q], pi.W2[r * H + k + 2 * q + 1]);
        *reinterpret_cast<uint4 *>(sm.w2 + tc05::kmajor_offset(r, k, kLBO, kSBO)) = *reinterpret_cast<uint4 *>(h);
    }
    for (int h = tid; h < H; h += 256) {
        sm.b2[h] = pi.b2[h];
        sm.w3[h] = pi.w3[h];
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.w1c[c][h] = pi.w1c[(int64_t)h * pi.dp + c];
    }
    if (tid == 0) {
        sm.b3 = pi.b3[0];
        sm.bad = 0;
        tc05::mbar_init(&sm.mbar, 1);
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t taddr = sm.tslot;
    // warp w reads TMEM lanes 32 (w % 4) .. + 31, columns [64 half, 64 half + 64)
    const uint32_t tlane = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(64 * half);
    constexpr uint32_t idesc = tc05::idesc_bf16_f32(TM, H);
    uint32_t phase = 0;

    for (int64_t u = blockIdx.x; u < n_units && !sm.bad; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int64_t lbase = un.cand / K;
        for (int i0 = 0; i0 < M && !sm.bad; i0 += 2) {
            const int list = i0 + (row >= 64 ? 1 : 0), slot = row & 63;
            const int n = list < M ? cand_cnt[lbase + list] : 0;
            const bool valid = slot < n;
            const int h0 = 64 * half;
            if (valid) {
                const int j = cand_idx[un.cand + (int64_t)list * K + slot];
                const float2 mxy = md.xy[list], sxy = sc.xy[j];
                const float dx = (sxy.x - mxy.x) * 0.01f, dy = (sxy.y - mxy.y) * 0.01f;
                const float dt = (float)(sc.t[j] - md.t[list] - un.offset) * pi.inv_window;
                const float4 *P4 = reinterpret_cast<const float4 *>(pi.P + (int64_t)(md.urow + list) * H + h0);
                const float4 *Q4 = reinterpret_cast<const float4 *>(sc.pq + (int64_t)(j - sc.ucol0) * H + h0);
#pragma unroll 2
                for (int h = 0; h < 64; h += 8) {
                    const float4 pa = P4[h / 4], pb = P4[h / 4 + 1], qa = Q4[h / 4], qb = Q4[h / 4 + 1];
                    float v[8] = {pa.x + qa.x, pa.y + qa.y, pa.z + qa.z, pa.w + qa.w,
                                  pb.x + qb.x, pb.y + qb.y, pb.z + qb.z, pb.w + qb.w};
                    __align__(16) __nv_bfloat162 hh[4];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        v[q] = fmaf(sm.w1c[0][h0 + h + q], dx, v[q]);
                        v[q] = fmaf(sm.w1c[1][h0 + h + q], dy, v[q]);
                        v[q] = fmaxf(fmaf(sm.w1c[2][h0 + h + q], dt, v[q]), 0.0f);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) hh[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    *reinterpret_cast<uint4 *>(sm.a + tc05::kmajor_offset(row, h0 + h, kLBO, kSBO)) =
                        *reinterpret_cast<uint4 *>(hh);
                }
            } else {
                for (int h = 0; h < 64; h += 8)
                    *reinterpret_cast<uint4 *>(sm.a + tc05::kmajor_offset(row, h0 + h, kLBO, kSBO)) =
                        make_uint4(0, 0, 0, 0);
            }
            tc05::fence_proxy_async_smem();
            tc05::fence_before_sync();
            __syncthreads();
            tc05::fence_after_sync();
            if (tid == 0) {
                const uint32_t a0 = tc05::smem_u32(sm.a), b0 = tc05::smem_u32(sm.w2);
                for (int ks = 0; ks < H / 16; ++ks)
                    tc05::mma_bf16(taddr, tc05::smem_desc(a0 + ks * 2 * kLBO, kLBO, kSBO),
                                   tc05::smem_desc(b0 + ks * 2 * kLBO, kLBO, kSBO), idesc, ks > 0);
                tc05::mma_commit(&sm.mbar);
            }
            const bool ok = tc05::mbar_wait(&sm.mbar, phase, kPolls);
            phase ^= 1u;
            if (!ok && lane == 0) { atomicExch(status, 1); sm.bad = 1; }
            tc05::fence_after_sync();
            float acc = 0.0f;
            if (ok) {
#pragma unroll
                for (int c0 = 0; c0 < 64; c0 += 32) {
                    float v[32];
                    tc05::tmem_ld32(tlane + (uint32_t)c0, v);
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        acc = fmaf(fmaxf(v[q] + sm.b2[h0 + c0 + q], 0.0f), sm.w3[h0 + c0 + q], acc);
                }
            }
            sm.part[half][row] = acc;
            tc05::fence_before_sync();
            __syncthreads();
            tc05::fence_after_sync();
            if (half == 0 && list < M && slot < K)
                scores[(lbase + list) * K + slot] = valid ? sm.b3 + sm.part[0][row] + sm.part[1][row] : kNegInf;
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc<H>(taddr);
}

// Per (unit, i) list: keep the `keep` best scores (ties: lower slot), in slot order; precision mode
// re-scores the kept candidates' unary costs in FP32. One warp per list.
__global__ void __launch_bounds__(256) prop_keep_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                        const ModelRec *__restrict__ models,
                                                        const SceneRec *__restrict__ scenes, Params p, int keep,
                                                        int rescore, const float *__restrict__ scores,
                                                        const int32_t *__restrict__ cand_idx,
                                                        const float *__restrict__ cand_u,
                                                        const int32_t *__restrict__ cand_cnt,
                                                        int32_t *__restrict__ out_idx, float *__restrict__ out_u,
                                                        int32_t *__restrict__ out_cnt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = p.K;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int64_t lbase = un.cand / K;
        for (int li = warp; li < md.M; li += 8) {
            const int nl = cand_cnt[lbase + li];
            const int kk = nl < keep ? nl : keep;
            const float *sl = scores + (lbase + li) * K;
            float v0 = lane < nl ? sl[lane] : kNegInf;
            float v1 = lane + 32 < nl ? sl[lane + 32] : kNegInf;
            bool c0 = false, c1 = false;
            for (int q = 0; q < kk; ++q) {
                float bv = v0 >= v1 ? v0 : v1;
                int bs = v0 >= v1 ? lane : lane + 32;
                if (lane >= nl) bs = 1 << 20;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
                    const int os = __shfl_xor_sync(0xffffffffu, bs, off);
                    if (ov > bv || (ov == bv && os < bs)) { bv = ov; bs = os; }
                }
                if (bs == lane) { c0 = true; v0 = kNegInf; }
                if (bs == lane + 32) { c1 = true; v1 = kNegInf; }
            }
            const uint32_t m0 = __ballot_sync(0xffffffffu, c0), m1 = __ballot_sync(0xffffffffu, c1);
            const int64_t obase = (lbase + li) * keep;
            const int64_t ibase = un.cand + (int64_t)li * K;
            if (c0) {
                const int pos = __popc(m0 & lt);
                const int j = cand_idx[ibase + lane];
                out_idx[obase + pos] = j;
                out_u[obase + pos] = rescore ? exact_u(md.f + (int64_t)li * p.F, sc.f + (int64_t)j * p.F, p.F,
                                                       p.lambda1)
                                             : cand_u[ibase + lane];
            }
            if (c1) {
                const int pos = __popc(m0) + __popc(m1 & lt);
                const int j = cand_idx[ibase + lane + 32];
                out_idx[obase + pos] = j;
                out_u[obase + pos] = rescore ? exact_u(md.f + (int64_t)li * p.F, sc.f + (int64_t)j * p.F, p.F,
                                                       p.lambda1)
                                             : cand_u[ibase + lane + 32];
            }
            for (int q = kk + lane; q < keep; q += 32) out_idx[obase + q] = -1;
            if (lane == 0) out_cnt[lbase + li] = kk;
        }
    }
}

// Units of the pruned pass: same problems, lists of `keep` candidates.
__global__ void derive_units_kernel(const Unit *__restrict__ in, int64_t n, int K, int keep, Unit *__restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        Unit u = in[k];
        u.cand = u.cand / K * keep;
        u.beta = u.beta / ((int64_t)K * K) * keep * keep;
        out[k] = u;
    }
}

// Units whose pruned optimum is infeasible, appended to `list` (fallback to the full lists).
__global__ void collect_infeasible_kernel(const UnitResult *__restrict__ res, const Unit *__restrict__ units,
                                          int64_t n, int beta_stride, Unit *__restrict__ list, int *__restrict__ count)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (res[k].z1 < 0) {
            const int at = atomicAdd(count, 1);
            Unit u = units[k];
            u.beta = (int64_t)at * beta_stride;
            list[at] = u;
        }
    }
}

}  // namespace

cudaError_t launch_prop_prune(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                              Params p, const PropInfer &pi, const int32_t *cand_idx, const float *cand_u,
                              const int32_t *cand_cnt, float *scores, int32_t *out_idx, float *out_u,
                              int32_t *out_cnt, int *status, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    const size_t smem = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(prop_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prop_score_kernel, 256, smem)) != cudaSuccess)
        return e;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);   // 4 x 128 TMEM columns
    const int64_t grid = std::min<int64_t>(n_units, (int64_t)sms * per_sm);
    prof_begin(kProfPrune, st);
    prop_score_kernel<<<(unsigned)grid, 256, smem, st>>>(units, n_units, models, scenes, p, pi, cand_idx, cand_cnt,
                                                         scores, status);
    if ((e = cudaGetLastError()) == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>(n_units, (int64_t)1 << 20);
        prop_keep_kernel<<<(unsigned)blocks, 256, 0, st>>>(units, n_units, models, scenes, p, pi.keep, pi.rescore,
                                                           scores, cand_idx, cand_u, cand_cnt, out_idx, out_u,
                                                           out_cnt);
        e = cudaGetLastError();
    }
    prof_end(kProfPrune, st);
    return e;
}

cudaError_t launch_derive_units(const Unit *in, int64_t n, int K, int keep, Unit *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    derive_units_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(in, n, K, keep, out);
    return cudaGetLastError();
}

cudaError_t launch_collect_infeasible(const UnitResult *res, const Unit *units, int64_t n, int beta_stride, Unit *list,
                                      int *count, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    collect_infeasible_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(res, units, n,
                                                                                                  beta_stride, list,
                                                                                                  count);
    return cudaGetLastError();
}

}  // namespace hgm
