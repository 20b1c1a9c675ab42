// k_select.cu -- candidate lists C_i(o): window + top-K cap.
//
// For unit (model m, scene s, offset o) and model point i, the window is the
// frame range [t_i+o-w, t_i+o+w] clipped to the scene; through the minnode
// table of Sec. 3.4 it is the contiguous sorted-scene range
// [minnode(f0), minnode(f1+1)). If it holds more than K points, the K with
// the smallest unary cost are kept (ties to the lower scene index), and the
// kept points are listed in ascending scene index (hence ascending frame).
//
// One warp per (unit, i). The K-th smallest key is found exactly by a radix
// select on the IEEE bit patterns (unary costs are >= 0, so the bit pattern
// orders like the value), one 8-bit digit per pass from the top; a final
// ballot pass keeps every key below the threshold plus the first equal ones in
// index order. Integer decisions therefore depend only on the FP32 keys of
// kernel (a), bit for bit. The costs of one window share their top bits (same
// exponent range), so the digits on which all keys agree are read off an AND
// and an OR of the keys instead of being histogrammed: the first pass that
// would otherwise put every key into one shared-memory bin -- 32 lanes adding
// to the same counter, serialised -- is skipped.
#include "hgm_internal.cuh"
#include "unary_common.cuh"

namespace hgm {
namespace {

constexpr int kWarps = 8;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// kKeyRegs keys per lane are held in registers: windows of up to 32 kKeyRegs keys are selected from them,
// longer ones from memory in every pass. The launch picks 8 (three CTAs per SM) when the call's typical
// window (the scenes' mean density over 2w+1 frames) fits 256 keys, else 20 (two CTAs per SM, the registers
// the larger arrays need).
template <int kKeyRegs, int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) select_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                             const ModelRec *__restrict__ models,
                                                             const SceneRec *__restrict__ scenes, Params p,
                                                             int32_t *__restrict__ cand_idx,
                                                             float *__restrict__ cand_u,
                                                             int32_t *__restrict__ cand_cnt)
{
    __shared__ uint32_t hist[kWarps][256];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int K = p.K;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        for (int i = warp; i < md.M; i += kWarps) {
            int32_t *oidx = cand_idx + un.cand + (int64_t)i * K;
            float *ou = cand_u + un.cand + (int64_t)i * K;
            const int ti = md.t[i];
            int f0 = ti + un.offset - p.window, f1 = ti + un.offset + p.window;
            f0 = max(f0, 0);
            f1 = min(f1, sc.n_frames - 1);
            int j0 = 0, n = 0;
            if (f0 <= f1) {
                j0 = sc.frame_start[f0];
                n = sc.frame_start[f1 + 1] - j0;
            }
            const float *key = sc.U + (int64_t)(md.urow + i) * sc.upitch + (j0 - sc.ucol0);
            int kept = n < K ? n : K;
            if (n <= K) {
                for (int e = lane; e < K; e += 32) {
                    oidx[e] = e < n ? j0 + e : -1;
                    ou[e] = e < n ? key[e] : __int_as_float(0x7f800000);
                }
            } else {
                // radix select of the K-th smallest key (1-based rank kk); windows of up to 32 kKeyRegs keys are
                // read once into registers (lane + 32 q), longer ones from memory in every pass
                const bool inreg = n <= 32 * kKeyRegs;
                uint32_t kb[kKeyRegs];
#pragma unroll
                for (int q = 0; q < kKeyRegs; ++q) {
                    const int e = lane + 32 * q;
                    kb[q] = inreg && e < n ? __float_as_uint(key[e]) : 0xffffffffu;
                }
                // bits on which every key of the window agrees
                uint32_t kand = 0xffffffffu, kor = 0u;
                if (inreg) {
#pragma unroll
                    for (int q = 0; q < kKeyRegs; ++q)
                        if (lane + 32 * q < n) { kand &= kb[q]; kor |= kb[q]; }
                } else {
                    for (int e = lane; e < n; e += 32) {
                        const uint32_t b = __float_as_uint(key[e]);
                        kand &= b;
                        kor |= b;
                    }
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    kand &= __shfl_xor_sync(0xffffffffu, kand, off);
                    kor |= __shfl_xor_sync(0xffffffffu, kor, off);
                }
                const uint32_t differ = kand ^ kor;
                uint32_t prefix = 0, mask = 0;
                int kk = K;
                for (int shift = 24; shift >= 0; shift -= 8) {
                    if (((differ >> shift) & 255u) == 0) {   // one digit value for every key: no histogram
                        prefix |= kand & (255u << shift);
                        mask |= 255u << shift;
                        continue;
                    }
                    for (int d = lane; d < 256; d += 32) hist[warp][d] = 0;
                    __syncwarp();
                    if (inreg) {
                        // slots past the window hold 0xffffffff: costs are >= 0 (bit 31 clear), so such a slot
                        // either fails the prefix test or lands in bin 255, above every real key's bin
#pragma unroll
                        for (int q = 0; q < kKeyRegs; ++q) {
                            const uint32_t b = kb[q];
                            if ((b & mask) == prefix) atomicAdd(&hist[warp][(b >> shift) & 255u], 1u);
                        }
                    } else {
                        for (int e = lane; e < n; e += 32) {
                            uint32_t b = __float_as_uint(key[e]);
                            if ((b & mask) == prefix) atomicAdd(&hist[warp][(b >> shift) & 255u], 1u);
                        }
                    }
                    __syncwarp();
                    uint32_t c[8];
                    uint32_t sum = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) { c[q] = hist[warp][lane * 8 + q]; sum += c[q]; }
                    uint32_t incl = sum;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += v;
                    }
                    uint32_t excl = incl - sum;
                    bool mine = excl < (uint32_t)kk && (uint32_t)kk <= incl;
                    int digit = 0;
                    uint32_t below = excl;
                    if (mine) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            if (below + c[q] >= (uint32_t)kk) { digit = lane * 8 + q; break; }
                            below += c[q];
                        }
                    }
                    uint32_t ball = __ballot_sync(0xffffffffu, mine);
                    int src = __ffs(ball) - 1;
                    digit = __shfl_sync(0xffffffffu, digit, src);
                    below = __shfl_sync(0xffffffffu, below, src);
                    prefix |= (uint32_t)digit << shift;
                    mask |= 255u << shift;
                    kk -= (int)below;
                    __syncwarp();
                }
                // keep keys < tau, plus the first kk keys == tau in index order (tau is a real key's bits, so
                // the 0xffffffff of slots past the window is never kept)
                const uint32_t tau = prefix;
                const uint32_t lt_mask = lanemask_lt();
                int base = 0, eqseen = 0;
                auto keep_step = [&](uint32_t b, int e) {
                    const bool lt = b < tau;
                    const bool eq = b == tau;
                    const uint32_t eqm = __ballot_sync(0xffffffffu, eq);
                    const int eqrank = eqseen + __popc(eqm & lt_mask);
                    const bool keep = lt || (eq && eqrank < kk);
                    const uint32_t km = __ballot_sync(0xffffffffu, keep);
                    const int pos = base + __popc(km & lt_mask);
                    if (keep && pos < K) { oidx[pos] = j0 + e; ou[pos] = __uint_as_float(b); }
                    base += __popc(km);
                    eqseen += __popc(eqm);
                };
                if (inreg) {
#pragma unroll
                    for (int q = 0; q < kKeyRegs; ++q)
                        if (32 * q < n) keep_step(kb[q], lane + 32 * q);
                } else {
                    for (int c0 = 0; c0 < n; c0 += 32) {
                        const int e = c0 + lane;
                        keep_step(e < n ? __float_as_uint(key[e]) : 0xffffffffu, e);
                    }
                }
            }
            if (lane == 0) cand_cnt[un.cand / K + i] = kept;
            if (p.rescore > 0 && kept > 0) {
                // precision mode: the p.rescore smallest approximate costs (ties: lower slot) are
                // recomputed from the FP32 descriptors in the exact kernel's fixed FMA order
                __syncwarp();
                float kv[2];
                kv[0] = lane < kept ? ou[lane] : __int_as_float(0x7f800000);
                kv[1] = lane + 32 < kept ? ou[lane + 32] : __int_as_float(0x7f800000);
                int mine = -1;
                const int rounds = p.rescore < kept ? p.rescore : kept;
                for (int q = 0; q < rounds; ++q) {
                    float bv = kv[0] <= kv[1] ? kv[0] : kv[1];
                    int bs = kv[0] <= kv[1] ? lane : lane + 32;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
                        const int os = __shfl_xor_sync(0xffffffffu, bs, off);
                        if (ov < bv || (ov == bv && os < bs)) { bv = ov; bs = os; }
                    }
                    if (lane == q) mine = bs;
                    if (bs == lane) kv[0] = __int_as_float(0x7f800000);
                    if (bs == lane + 32) kv[1] = __int_as_float(0x7f800000);
                }
                if (mine >= 0 && mine < kept) {
                    ou[mine] = unary_fp32(md.f + (int64_t)i * p.F, sc.f + (int64_t)oidx[mine] * p.F, p.F, p.lambda1);
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_select(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                          Params p, int max_M, int32_t *cand_idx, float *cand_u, int32_t *cand_cnt,
                          cudaStream_t st)
{
    (void)max_M;
    if (n_units <= 0) return cudaSuccess;
    int64_t blocks = n_units < (int64_t)1 << 20 ? n_units : (int64_t)1 << 20;
    prof_begin(kProfSelect, st);
    if (p.max_window <= 32 * 8)
        select_kernel<8, 3><<<(unsigned)blocks, kWarps * 32, 0, st>>>(units, n_units, models, scenes, p, cand_idx,
                                                                      cand_u, cand_cnt);
    else
        select_kernel<20, 2><<<(unsigned)blocks, kWarps * 32, 0, st>>>(units, n_units, models, scenes, p, cand_idx,
                                                                       cand_u, cand_cnt);
    prof_end(kProfSelect, st);
    return cudaGetLastError();
}

cudaError_t preload_select()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, select_kernel<8, 3>);
    return e == cudaSuccess ? cudaFuncGetAttributes(&a, select_kernel<20, 2>) : e;
}

}  // namespace hgm
