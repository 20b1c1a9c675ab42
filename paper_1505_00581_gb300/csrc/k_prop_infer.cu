// k_prop_infer.cu -- learned pruning of the candidate lists before the recursion.
//
// For each (unit, model point i) list of up to K candidates, the proposal
// network scores every candidate j and keeps the `keep` best (ties: lower
// slot), listed in slot order (ascending scene index, as the recursion
// expects). The first layer is decomposed as
//   W1 x + b1 = (W1a f_i + b1 - W1c.(x_i, y_i, 0) / 100) + (W1b f'_j + W1c.(x'_j, y'_j, 0) / 100)
//             + W1c_t (t'_j - t_i - o) / w
// (x = [f_i, f'_j, dx / 100, dy / 100, dt / w]): the two point projections P
// (per model point) and Q (per scene point) are computed once per batch by the
// tensor-core row-product kernel with the linear position terms folded in, so
// a candidate's 128 hidden units cost one add and one fma each.
//
// P and Q are held as BF16 rows, so that a candidate's first layer is BF16x2
// arithmetic: per pair of hidden units one add (P + Q, rounded to BF16) and
// one fused multiply-add with ReLU (+ dt (W1c_t / w), rounded once), whose
// result is the layer-2 operand as it stands.
//
// The scoring kernel stages 128 candidates per tile (128 / 2^ceil(log2 K)
// lists) as BF16 and runs layer 2 (128 x 128) as tcgen05.mma with W2 resident
// in shared memory, the bias b2 (BF16) entering as one more K step against a
// constant column of ones. Tiles are double-buffered in shared memory and in
// tensor memory: tile k is gathered while the MMA of tile k - 1 runs, its
// epilogue (relu, dot with w3) follows the issue of tile k, and the two column
// halves of a row are summed one tile later, so one barrier per tile suffices.
#include "hgm_internal.cuh"
#include "prop.cuh"
#include "tc05.cuh"
#include "unary_common.cuh"
#include "f32x2.cuh"

namespace hgm {
namespace {

constexpr int H = kPropHidden;
constexpr int TM = 128;
constexpr uint32_t kLBO = 128;
constexpr uint32_t kSBO = (H / 8) * 128;   // K = 128 components per row
constexpr uint32_t kPolls = 1u << 26;
constexpr float kNegInf = -__builtin_huge_valf();

constexpr uint32_t kSBO16 = 2 * 128;       // K = 16 components per row (the bias block)

struct Smem {
    unsigned char a[2][TM * H * 2];  // hidden layer 1 of two tiles, BF16, canonical K-major
    unsigned char w2[H * H * 2];     // W2 (rows = output units), BF16
    // the layer-2 bias as a 17th K step of the MMA: A gets a constant block (component 0 = 1, the rest 0)
    // shared by both tiles, W2 a block whose component 0 is b2 (BF16)
    unsigned char a1[TM * 16 * 2];
    unsigned char b2k[H * 16 * 2];
    float part[2][2][TM];            // [buffer][column half][row]: half-sums of the last layer
    float w3[H];                     // output weights
    float b3;
    uint64_t mbar[2];
    uint32_t tslot;
};


// rows[r][h] += sign * (W1c[h][0] x_r + W1c[h][1] y_r) / 100: the position terms of the first layer.
// With out_bf16, the sum is written there rounded to BF16 (rows left unchanged).
__global__ void fold_xy_kernel(float *__restrict__ rows, int64_t n, const float2 *__restrict__ xy,
                               const float *__restrict__ w1c, int dp, float sign, __nv_bfloat16 *__restrict__ out_bf16)
{
    const int64_t total = n * H;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / H;
        const int h = (int)(e % H);
        const float2 p = xy[r];
        const float t = fmaf(w1c[(int64_t)h * dp], p.x, w1c[(int64_t)h * dp + 1] * p.y);
        const float v = fmaf(sign * 0.01f, t, rows[e]);
        if (out_bf16) out_bf16[e] = __float2bfloat16_rn(v);
        else rows[e] = v;
    }
}

// Final logit of every candidate of every list: scores [n_lists x K] (-inf for empty slots).
// 256 threads. Building a tile: warp w owns hidden units [32 (w%4), +32) of rows [64 (w/4), +64); lane l
// takes row 8g + l/4 of each group g of 8 and the 8 units 32 (w%4) + 8 (l%4) .. +8, so a warp reads 8 BF16
// Q rows as whole 32-byte sectors and writes 4 contiguous core matrices of the A tile. Epilogue: row
// r = tid % 128, half = tid / 128 owns accumulator columns [64 half, 64 half + 64).
__global__ void __launch_bounds__(256, 2) prop_score_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                            const ModelRec *__restrict__ models,
                                                            const SceneRec *__restrict__ scenes, Params p,
                                                            PropInfer pi, int kp_log2,
                                                            const int32_t *__restrict__ cand_idx,
                                                            const int32_t *__restrict__ cand_cnt,
                                                            float *__restrict__ scores, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (TM - 1), half = tid >> 7, h0 = 64 * half;
    const int K = p.K;
    const int lpt = TM >> kp_log2;                                  // lists per tile
    const int lsub = row >> kp_log2, slot = row & ((1 << kp_log2) - 1);
    // build-phase roles
    // a row's four 16-byte chunks sit on adjacent lanes (measured faster for the gathers than the
    // bank-conflict-free order of the A-tile stores)
    const int bh0 = 32 * (warp & 3) + 8 * (lane & 3);              // first of this lane's 8 hidden units
    const int brow0 = 64 * (warp >> 2) + (lane >> 2);                // its row in group 0 (+8 per group)
    __nv_bfloat162 w1t[4];                                           // W1c_t / w for those units, BF16 pairs
#pragma unroll
    for (int e = 0; e < 4; ++e)
        w1t[e] = __floats2bfloat162_rn(pi.w1c[(int64_t)(bh0 + 2 * e) * pi.dp + 2] * pi.inv_window,
                                       pi.w1c[(int64_t)(bh0 + 2 * e + 1) * pi.dp + 2] * pi.inv_window);

    if (warp == 0) tc05::tmem_alloc<2 * H>(&sm.tslot);
    for (int e = tid; e < H * (H / 8); e += 256) {          // W2 -> BF16, canonical layout
        const int r = e / (H / 8), k = (e % (H / 8)) * 8;
        __align__(16) __nv_bfloat162 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            h[q] = __floats2bfloat162_rn(pi.W2[r * H + k + 2 * q], pi.W2[r * H + k + 2 * q + 1]);
        *reinterpret_cast<uint4 *>(sm.w2 + tc05::kmajor_offset(r, k, kLBO, kSBO)) = *reinterpret_cast<uint4 *>(h);
    }
    for (int h = tid; h < H; h += 256) sm.w3[h] = pi.w3[h];
    for (int e = tid; e < TM * 2; e += 256) {          // the bias blocks: 16-byte chunks of 8 components
        const int r = e >> 1, k = (e & 1) * 8;
        __align__(16) __nv_bfloat16 ha[8], hb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            ha[q] = __float2bfloat16_rn(k + q == 0 ? 1.0f : 0.0f);
            hb[q] = __float2bfloat16_rn(k + q == 0 ? pi.b2[r] : 0.0f);
        }
        *reinterpret_cast<uint4 *>(sm.a1 + tc05::kmajor_offset(r, k, kLBO, kSBO16)) = *reinterpret_cast<uint4 *>(ha);
        *reinterpret_cast<uint4 *>(sm.b2k + tc05::kmajor_offset(r, k, kLBO, kSBO16)) = *reinterpret_cast<uint4 *>(hb);
    }
    if (tid == 0) {
        sm.b3 = pi.b3[0];
        tc05::mbar_init(&sm.mbar[0], 1);
        tc05::mbar_init(&sm.mbar[1], 1);
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t taddr = sm.tslot;
    // warp w reads TMEM lanes 32 (w % 4) .. + 31, columns [64 half, 64 half + 64) of either accumulator
    const uint32_t tlane = taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)h0;
    constexpr uint32_t idesc = tc05::idesc_bf16_f32(TM, H);

    uint32_t parity = 0;      // bit b: phase parity of the next completion of mbar[b]
    uint32_t pending = 0;     // bit b: an MMA committed to mbar[b] whose completion was not yet observed
    int64_t o1 = -1, o2 = -1; // score index of this row in tiles k-1 and k-2 (half 0 only; -1 none)
    bool v1 = false, v2 = false;
    bool bad = false, stop = false;
    int64_t k = 0;

    // epilogue of the tile in accumulator b: relu(z) . w3 over this thread's 64 columns (z holds b2)
    auto epilogue = [&](int b) {
        bool ok = tc05::mbar_wait(&sm.mbar[b], (parity >> b) & 1u, kPolls);
        ok = __all_sync(0xffffffffu, ok);
        float acc = 0.0f;
        if (ok) {
            parity ^= 1u << b;
            pending &= ~(1u << b);
            tc05::fence_after_sync();
            // columns in pairs (packed FP32x2 add and FMA): even and odd columns accumulate separately
            unsigned long long acc2 = pk2(0.0f, 0.0f);
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 32) {
                float v[32];
                tc05::tmem_ld32(tlane + (uint32_t)(H * b + c0), v);
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    const float4 w3 = *reinterpret_cast<const float4 *>(&sm.w3[h0 + c0 + q]);
                    acc2 = fma2(pk2(fmaxf(v[q], 0.0f), fmaxf(v[q + 1], 0.0f)), pk2(w3.x, w3.y), acc2);
                    acc2 = fma2(pk2(fmaxf(v[q + 2], 0.0f), fmaxf(v[q + 3], 0.0f)), pk2(w3.z, w3.w), acc2);
                }
            }
            float a0, a1;
            upk2(acc2, a0, a1);
            acc = a0 + a1;
        } else {
            bad = true;
            if (lane == 0) atomicExch(status, 1);
        }
        sm.part[b][half][row] = acc;
        tc05::fence_before_sync();
    };
    auto final_score = [&](int64_t o, bool v, int b) {
        if (o >= 0) scores[o] = v ? sm.b3 + sm.part[b][0][row] + sm.part[b][1][row] : kNegInf;
    };

    for (int64_t u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int64_t lbase = un.cand / K;
        // the 8 row groups' list counts and raw candidate indices of the tile at i0 (the slot clamped into the
        // unit's lists, so the index load does not wait for the count); the next tile's are loaded right after
        // this tile's build, so that they arrive while the barrier, the MMA issue and the epilogue run
        int cn[8], jr[8];
        auto load_idx = [&](int i0n) {
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int r = brow0 + 8 * g, lst = i0n + (r >> kp_log2), sl = r & ((1 << kp_log2) - 1);
                const int lc = lst < M ? lst : M - 1, sc_ = sl < K ? sl : K - 1;
                cn[g] = cand_cnt[lbase + lc];
                jr[g] = cand_idx[un.cand + (int64_t)lc * K + sc_];
            }
        };
        load_idx(0);
        for (int i0 = 0; i0 < M; i0 += lpt) {
            const int buf = (int)(k & 1);
            unsigned char *arow = sm.a[buf];
            // gather: the candidate indices (loaded before), then their frames and Q chunks
            int jg[8];
            bool vg[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int r = brow0 + 8 * g, lst = i0 + (r >> kp_log2), sl = r & ((1 << kp_log2) - 1);
                vg[g] = lst < M && sl < cn[g];
                jg[g] = vg[g] ? jr[g] : 0;
            }
            int tg[8];
            uint4 qg[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                if (vg[g]) {
                    tg[g] = sc.t[jg[g]];
                    qg[g] = __ldg(reinterpret_cast<const uint4 *>(sc.pq + (int64_t)(jg[g] - sc.ucol0) * H + bh0));
                } else {
                    tg[g] = 0;
                    qg[g] = make_uint4(0, 0, 0, 0);
                }
            }
            int plist = -1;
            uint4 pv = make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const int r = brow0 + 8 * g, lst = i0 + (r >> kp_log2);
                __align__(16) __nv_bfloat162 hh[4];
                if (vg[g]) {
                    if (lst != plist) {   // the row's list: this lane's 8 units of P (rows of a group share it)
                        pv = __ldg(reinterpret_cast<const uint4 *>(pi.Pb + (int64_t)(md.urow + lst) * H + bh0));
                        plist = lst;
                    }
                    const __nv_bfloat162 dt = __float2bfloat162_rn((float)(tg[g] - md.t[lst] - un.offset));
                    const __nv_bfloat162 *p2 = reinterpret_cast<const __nv_bfloat162 *>(&pv);
                    const __nv_bfloat162 *q2 = reinterpret_cast<const __nv_bfloat162 *>(&qg[g]);
#pragma unroll
                    for (int e = 0; e < 4; ++e)   // two hidden units per BF16x2 add and fused multiply-add-relu
                        hh[e] = __hfma2_relu(dt, w1t[e], __hadd2(p2[e], q2[e]));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) hh[e] = __floats2bfloat162_rn(0.0f, 0.0f);
                }
                *reinterpret_cast<uint4 *>(arow + tc05::kmajor_offset(r, bh0, kLBO, kSBO)) =
                    *reinterpret_cast<uint4 *>(hh);
            }
            if (i0 + lpt < M) load_idx(i0 + lpt);
            // this thread's epilogue row
            const int list = i0 + lsub;
            const bool valid = list < M && slot < cand_cnt[lbase + (list < M ? list : 0)];
            const int64_t o0 = (half == 0 && list < M && slot < K) ? (lbase + list) * K + slot : -1;
            tc05::fence_proxy_async_smem();
            tc05::fence_before_sync();
            stop = __syncthreads_or(bad) != 0;
            tc05::fence_after_sync();
            if (stop) break;
            final_score(o2, v2, buf);   // tile k-2: both halves were written in the previous iteration
            if (tid == 0) {
                const uint32_t a0 = tc05::smem_u32(arow), b0 = tc05::smem_u32(sm.w2);
                for (int ks = 0; ks < H / 16; ++ks)
                    tc05::mma_bf16(taddr + (uint32_t)(H * buf), tc05::smem_desc(a0 + ks * 2 * kLBO, kLBO, kSBO),
                                   tc05::smem_desc(b0 + ks * 2 * kLBO, kLBO, kSBO), idesc, ks > 0);
                tc05::mma_bf16(taddr + (uint32_t)(H * buf), tc05::smem_desc(tc05::smem_u32(sm.a1), kLBO, kSBO16),
                               tc05::smem_desc(tc05::smem_u32(sm.b2k), kLBO, kSBO16), idesc, true);
                tc05::mma_commit(&sm.mbar[buf]);
            }
            pending |= 1u << buf;
            if (k >= 1) epilogue(buf ^ 1);
            o2 = o1; v2 = v1;
            o1 = o0; v1 = valid;
            ++k;
        }
    }
    // drain: the last iteration's reads of part[] (tile k-3) come before the last tile's epilogue writes
    tc05::fence_before_sync();
    stop = __syncthreads_or(bad) != 0;
    tc05::fence_after_sync();
    if (!stop && k >= 1) epilogue((int)((k - 1) & 1));
    tc05::fence_before_sync();
    stop = __syncthreads_or(bad) != 0;
    tc05::fence_after_sync();
    if (!stop) {
        if (k >= 2) final_score(o2, v2, (int)(k & 1));
        if (k >= 1) final_score(o1, v1, (int)((k - 1) & 1));
    } else {
        // a wait gave up: give the MMAs still in flight a bounded time before the accumulators are freed
        for (int b = 0; b < 2; ++b)
            if ((pending >> b) & 1u) tc05::mbar_wait(&sm.mbar[b], (parity >> b) & 1u, kPolls);
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc<2 * H>(taddr);
}

// Per (unit, i) list: keep the `keep` best scores (ties: lower slot), in slot order, with their FP32 unary
// costs from the candidate list (re-scored afterwards in the precision mode). One warp per list.
__global__ void __launch_bounds__(256) prop_keep_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                        const ModelRec *__restrict__ models, Params p, int keep,
                                                        const float *__restrict__ scores,
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
        const int M = models[un.model].M;
        const int64_t lbase = un.cand / K;
        for (int li = warp; li < M; li += 8) {
            const int nl = cand_cnt[lbase + li];
            const int kk = nl < keep ? nl : keep;
            const float *sl = scores + (lbase + li) * K;
            bool c0 = false, c1 = false;
            if (kk <= 10) {
                // a few rounds of a warp-wide argmax (ties: lower slot); longer keeps bisect for the threshold
                float v0 = lane < nl ? sl[lane] : kNegInf;
                float v1 = lane + 32 < nl ? sl[lane + 32] : kNegInf;
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
            } else {
                // the kept set: the kk largest scores, ties to the lower slot (slots in [0, nl)). Scores become
                // order-preserving keys (larger score, larger key); empty slots get key 0, below every score's key
                // (a score is finite or -inf, whose key is 0x007fffff)
                auto okey = [](float v) {
                    const uint32_t b = __float_as_uint(v == 0.0f ? 0.0f : v);   // -0 ties with +0, as a float compare
                    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
                };
                const uint32_t k0 = lane < nl ? okey(sl[lane]) : 0u;
                const uint32_t k1 = lane + 32 < nl ? okey(sl[lane + 32]) : 0u;
                // the kk-th largest key T, bit by bit from the top: the largest T with at least kk keys >= T.
                // Bits on which every key of the list agrees are read off an AND and an OR of the keys.
                uint32_t kand = k0 & k1, kor = k0 | k1;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    kand &= __shfl_xor_sync(0xffffffffu, kand, off);
                    kor |= __shfl_xor_sync(0xffffffffu, kor, off);
                }
                const uint32_t differ = kand ^ kor;
                uint32_t T = kand & ~differ;   // the common bits
                // only the differing bits need a test, from the highest down
                for (int bit = differ ? 31 - __clz(differ) : -1; bit >= 0; --bit) {
                    if (!((differ >> bit) & 1u)) continue;
                    const uint32_t cand = T | (1u << bit);
                    const int cnt = __popc(__ballot_sync(0xffffffffu, k0 >= cand)) +
                                    __popc(__ballot_sync(0xffffffffu, k1 >= cand));
                    if (cnt >= kk) T = cand;
                }
                // keep every key above T, then the keys equal to T in slot order up to kk
                const int above =
                    __popc(__ballot_sync(0xffffffffu, k0 > T)) + __popc(__ballot_sync(0xffffffffu, k1 > T));
                const uint32_t e0 = __ballot_sync(0xffffffffu, k0 == T && lane < nl);
                const uint32_t e1 = __ballot_sync(0xffffffffu, k1 == T && lane + 32 < nl);
                const int need = kk - above;
                const int r0 = __popc(e0 & lt), r1 = __popc(e0) + __popc(e1 & lt);
                c0 = lane < nl && (k0 > T || (((e0 >> lane) & 1u) && r0 < need));
                c1 = lane + 32 < nl && (k1 > T || (((e1 >> lane) & 1u) && r1 < need));
            }
            const uint32_t m0 = __ballot_sync(0xffffffffu, c0), m1 = __ballot_sync(0xffffffffu, c1);
            const int64_t obase = (lbase + li) * keep;
            const int64_t ibase = un.cand + (int64_t)li * K;
            if (c0) {
                const int pos = __popc(m0 & lt);
                out_idx[obase + pos] = cand_idx[ibase + lane];
                out_u[obase + pos] = cand_u[ibase + lane];
            }
            if (c1) {
                const int pos = __popc(m0) + __popc(m1 & lt);
                out_idx[obase + pos] = cand_idx[ibase + lane + 32];
                out_u[obase + pos] = cand_u[ibase + lane + 32];
            }
            for (int q = kk + lane; q < keep; q += 32) out_idx[obase + q] = -1;
            if (lane == 0) out_cnt[lbase + li] = kk;
        }
    }
}

// Precision mode: the kept candidates' unary costs in FP32 (components in order, IEEE sqrt, times lambda1 --
// the same value as the FP32 table). One thread per kept slot; lists in unit order.
__global__ void __launch_bounds__(256) prop_rescore_kernel(const Unit *__restrict__ units, int64_t n_units,
                                                           const ModelRec *__restrict__ models,
                                                           const SceneRec *__restrict__ scenes, Params p, int keep,
                                                           const int32_t *__restrict__ out_idx,
                                                           const int32_t *__restrict__ out_cnt,
                                                           float *__restrict__ out_u)
{
    const int K = p.K;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int64_t lbase = un.cand / K;
        for (int e = threadIdx.x; e < md.M * keep; e += blockDim.x) {
            const int li = e / keep, c = e - li * keep;
            if (c >= out_cnt[lbase + li]) continue;
            const int64_t o = (lbase + li) * keep + c;
            const int j = out_idx[o];
            out_u[o] = unary_fp32(md.f + (int64_t)li * p.F, sc.f + (int64_t)j * p.F, p.F, p.lambda1);
        }
    }
}

// Precision mode, fallback units: every candidate of their full lists gets its FP32 unary cost (the same
// value as the FP32 table). Unit count read on the device; one CTA per unit at a time.
__global__ void __launch_bounds__(256) rescore_units_kernel(const Unit *__restrict__ units, int64_t n_max,
                                                            const int *__restrict__ n_dev,
                                                            const ModelRec *__restrict__ models,
                                                            const SceneRec *__restrict__ scenes, Params p,
                                                            const int32_t *__restrict__ cand_idx,
                                                            const int32_t *__restrict__ cand_cnt,
                                                            float *__restrict__ cand_u)
{
    const int64_t n = min((int64_t)*n_dev, n_max);
    const int K = p.K;
    for (int64_t u = blockIdx.x; u < n; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int64_t lbase = un.cand / K;
        for (int e = threadIdx.x; e < md.M * K; e += blockDim.x) {
            const int li = e / K, c = e - li * K;
            if (c >= cand_cnt[lbase + li]) continue;
            const int64_t o = un.cand + e;
            cand_u[o] = unary_fp32(md.f + (int64_t)li * p.F, sc.f + (int64_t)cand_idx[o] * p.F, p.F, p.lambda1);
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

// Units whose pruned optimum is infeasible, copied to `list` in their original (longest-first) order: the
// fallback keeps the batch's load balance. One CTA of 1024 threads scans the flags in blocks of 1024.
// `count` receives their number, `total` accumulates it across calls (read by hgm_prune_counters).
__global__ void __launch_bounds__(1024) collect_infeasible_kernel(const UnitResult *__restrict__ res,
                                                                  const Unit *__restrict__ units, int64_t n,
                                                                  Unit *__restrict__ list, int *__restrict__ count,
                                                                  unsigned long long *__restrict__ total)
{
    __shared__ int wsum[32];
    __shared__ int base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int64_t k0 = 0; k0 < n; k0 += 1024) {
        const int64_t k = k0 + tid;
        const bool f = k < n && res[k].z1 < 0;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int before = 0, all = 0;
        for (int w = 0; w < 32; ++w) {
            const int c = wsum[w];
            before += w < warp ? c : 0;
            all += c;
        }
        const int b0 = base;
        if (f) list[b0 + before + __popc(m & ((1u << lane) - 1))] = units[k];
        __syncthreads();
        if (tid == 0) base = b0 + all;
        __syncthreads();
    }
    if (tid == 0) {
        *count = base;
        atomicAdd(total, (unsigned long long)base);
    }
}

}  // namespace

cudaError_t launch_prop_fold_xy(float *rows, int64_t n, const float *xy, const float *w1c, int dp, float sign,
                                void *out_bf16, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n * H + 255) / 256, 8192);
    fold_xy_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, n, reinterpret_cast<const float2 *>(xy), w1c, dp, sign,
                                                     static_cast<__nv_bfloat16 *>(out_bf16));
    return cudaGetLastError();
}

cudaError_t launch_prop_score(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                              Params p, const PropInfer &pi, const int32_t *cand_idx, const int32_t *cand_cnt,
                              float *scores, int *status, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    if (p.K < 1 || p.K > 64) return cudaErrorInvalidValue;
    int kp_log2 = 0;
    while ((1 << kp_log2) < p.K) ++kp_log2;
    const size_t smem = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(prop_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    // two CTAs per SM: 2 x ~101 KB of shared memory, 2 x 256 of the SM's 512 TMEM columns
    const int64_t grid = std::min<int64_t>(n_units, (int64_t)sms * 2);
    prop_score_kernel<<<(unsigned)grid, 256, smem, st>>>(units, n_units, models, scenes, p, pi, kp_log2, cand_idx,
                                                         cand_cnt, scores, status);
    return cudaGetLastError();
}

cudaError_t launch_prop_prune(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                              Params p, const PropInfer &pi, const int32_t *cand_idx, const float *cand_u,
                              const int32_t *cand_cnt, float *scores, int32_t *out_idx, float *out_u,
                              int32_t *out_cnt, int *status, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    prof_begin(kProfPrune, st);
    cudaError_t e = launch_prop_score(units, n_units, models, scenes, p, pi, cand_idx, cand_cnt, scores, status, st);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>(n_units, (int64_t)1 << 20);
        prop_keep_kernel<<<(unsigned)blocks, 256, 0, st>>>(units, n_units, models, p, pi.keep, scores, cand_idx,
                                                           cand_u, cand_cnt, out_idx, out_u, out_cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && pi.rescore) {
        const int64_t blocks = std::min<int64_t>(n_units, (int64_t)1 << 20);
        prop_rescore_kernel<<<(unsigned)blocks, 256, 0, st>>>(units, n_units, models, scenes, p, pi.keep, out_idx,
                                                                  out_cnt, out_u);
        e = cudaGetLastError();
    }
    prof_end(kProfPrune, st);
    return e;
}

cudaError_t launch_rescore_units(const Unit *units, int64_t n_max, const int *n_dev, const ModelRec *models,
                                 const SceneRec *scenes, Params p, const int32_t *cand_idx, const int32_t *cand_cnt,
                                 float *cand_u, cudaStream_t st)
{
    if (n_max <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(n_max, (int64_t)sms * 8);
    rescore_units_kernel<<<(unsigned)grid, 256, 0, st>>>(units, n_max, n_dev, models, scenes, p, cand_idx, cand_cnt,
                                                         cand_u);
    return cudaGetLastError();
}

cudaError_t launch_derive_units(const Unit *in, int64_t n, int K, int keep, Unit *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    derive_units_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(in, n, K, keep, out);
    return cudaGetLastError();
}

cudaError_t launch_collect_infeasible(const UnitResult *res, const Unit *units, int64_t n, Unit *list, int *count,
                                      unsigned long long *total, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    collect_infeasible_kernel<<<1, 1024, 0, st>>>(res, units, n, list, count, total);
    return cudaGetLastError();
}

}  // namespace hgm
