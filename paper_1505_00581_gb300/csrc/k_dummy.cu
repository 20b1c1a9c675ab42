// k_dummy.cu -- the recursion with the dummy assignment of Eq. 2 (reading R5).
//
// Every candidate list C_i(o) gets one more slot, eps, after its real candidates (slot K of a table of
// L = K + 1 slots), with U(eps) = lambda1 W^d. A term that involves eps vanishes (Delta(i,j) if z_i or
// z_j is eps; D^g if any point of the triangle is), and a triple holding eps is feasible iff its real
// points, in chain order, are distinct, time-ordered and less than T frames apart. So the all-eps chain
// is always feasible and every offset has a finite optimum.
//
// One persistent CTA per unit, all tables in shared memory (L x L floats each): alpha_{i+1} and alpha_i
// (ping-pong), base(b, a) = U(a) + lambda2 Delta(a, b) + alpha_{i+1}(a, b) (eps rules applied), and the
// per-step directions P1(b, a) = A1 + theta(b->a), P2(b, a) = A2 + theta(a->b) (kept pairs only),
// R(a, c) = theta(a->c) (only for the a some row keeps, once the kept lists are built).
// Every open cell (b, c) has a best of at most thr(b): base(b, eps), since the triple (eps, b, c) is
// feasible and costs that alone, and base(b, a1) + max D^g when the row's smallest base a1 is feasible with
// every open c. A warp per row keeps the a with base <= thr(b) that may follow b and ranks them by
// (base, slot). Threads take groups of four consecutive c of one b (c fastest, so a warp shares b:
// broadcast reads of base, P1, P2) and walk b's kept a in that order until no open cell of the group can
// improve. The argmin slots go to a per-CTA global scratch, (M-2) x L x L bytes, and the CTA backtracks
// its own unit (Eq. 12); eps is reported as -2 in the assignment.
#include "hgm_internal.cuh"
#include "recurse_common.cuh"

namespace hgm {
namespace {

constexpr int kDummyThreads = 256;
constexpr int kL = kMaxK + 1;          // table side: up to 64 real slots + eps
constexpr int kTab = kL * kL;
constexpr int kRL = 68;                // row stride of R: four consecutive c of a row are one 16-byte load
constexpr float kGeoMax = 4.45f;       // > pi*sqrt(2) = 4.4429, bound of the FP32 D^g

struct DummySmem {
    float alpha[2][kTab];
    float base[kTab];                  // [b][a]
    float p1[kTab], p2[kTab];          // [b][a]
    alignas(16) float r[kL * kRL];     // [a][c], row stride kRL
    float2 xy[3][kL];                  // lists i (a), i-1 (b), i-2 (c)
    int t[3][kL], id[3][kL];
    float u[3][kL];
    uint8_t srt[kL][kMaxK];            // per row b: the kept real a by increasing base(b, a) (ties: lower slot)
    uint8_t kept[kL];                  // per row b: how many a srt[b] holds
    unsigned akept[2];                 // real a kept by some real row b (bits of slots 0-31, 32-63)
    int cnt[3];
    float ang[2];                      // the step's model angles A1, A2 (one thread computes them)
};
static_assert(2 * (sizeof(DummySmem) + 1024 + 128) <= 228 * 1024, "two CTAs per SM");

// (key, slot) order: smaller key first, then lower slot
__device__ __forceinline__ bool key_less(float ka, int sa, float kb, int sb)
{
    return ka < kb || (ka == kb && sa < sb);
}

struct DummyBest {
    float v;
    int j1, j2;
};

__device__ __forceinline__ bool dummy_better(float v, int j1, int j2, const DummyBest &o)
{
    if (v != o.v) return v < o.v;
    if (j1 != o.j1) return j1 < o.j1;
    return j2 < o.j2;
}

// kCount = true builds the accounting variant: identical work, plus a count of the (a, open cell) triples
// the walks evaluate, added to *evaluated (work accounting; not used on the timed path).
template <bool kCount>
__global__ void __launch_bounds__(kDummyThreads, 2) dummy_recurse_kernel(
    const Unit *__restrict__ units, int64_t n_units, const ModelRec *__restrict__ models,
    const SceneRec *__restrict__ scenes, Params p, float wd, const int32_t *__restrict__ cand_idx,
    const float *__restrict__ cand_u, const int32_t *__restrict__ cand_cnt, uint8_t *__restrict__ scratch,
    int64_t scratch_per_cta, float *__restrict__ energy, int32_t *__restrict__ assign,
    unsigned long long *__restrict__ evaluated)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DummySmem &sm = *reinterpret_cast<DummySmem *>(smem_raw);
    __shared__ DummyBest red[kDummyThreads / 32];
    const int K = p.K, L = K + 1, E = K;   // eps is slot K
    // e / L as one multiply-high: with m = ceil(2^32 / L), floor(e m / 2^32) = floor(e / L) for every
    // e < 2^32 / L (the error e (m - 2^32 / L) / 2^32 stays below 1 / L); the flat loops index e < 3 L^2
    const unsigned divL = 0xffffffffu / (unsigned)L + 1u;
    const float lam2 = p.lambda2, lam23 = __fmul_rn(p.lambda2, p.lambda3);
    const float ueps = __fmul_rn(p.lambda1, wd);
    const float gmax = lam23 * kGeoMax;
    const float inf = __int_as_float(0x7f800000);
    uint8_t *beta = scratch + (int64_t)blockIdx.x * scratch_per_cta;
    unsigned long long n_eval = 0;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int32_t *cidx = cand_idx + un.cand;
        const float *cu = cand_u + un.cand;
        const int32_t *ccnt = cand_cnt + un.cand / K;
        int cur = 0;
        for (int i = M - 1; i >= 2; --i) {
            // list buffers rotate with the chain index (list i in buffer i % 3): the first step loads the three
            // lists, every later step only list i - 2; slot s < cnt real, slot K eps
            const int sA = i % 3, sB = (i - 1) % 3, sC = (i - 2) % 3;
            const int nload = i == M - 1 ? 3 : 1, w0 = i == M - 1 ? 0 : 2;
            for (int e = threadIdx.x; e < nload * L; e += blockDim.x) {
                const int q = (int)__umulhi((unsigned)e, divL), s = e - q * L, li = i - (w0 + q);
                const int w = li % 3;
                const int n = ccnt[li];
                if (s < n) {
                    const int j = cidx[(int64_t)li * K + s];
                    sm.xy[w][s] = sc.xy[j];
                    sm.t[w][s] = sc.t[j];
                    sm.id[w][s] = j;
                    sm.u[w][s] = cu[(int64_t)li * K + s];
                } else if (s == E) {
                    sm.xy[w][s] = make_float2(0.f, 0.f);
                    sm.t[w][s] = 0;
                    sm.id[w][s] = -2;
                    sm.u[w][s] = ueps;
                }
                if (s == 0) sm.cnt[w] = n;
            }
            if (threadIdx.x == 0) {
                sm.akept[0] = 0u;
                sm.akept[1] = 0u;
                const float2 mi = md.xy[i], mj = md.xy[i - 1], mk = md.xy[i - 2];
                sm.ang[0] = signed_angle(mj, mi, mk);   // A1: at i-1, from ->i to ->i-2
                sm.ang[1] = signed_angle(mi, mj, mk);   // A2: at i, from ->i-1 to ->i-2
            }
            // base reads lists i and i - 1 only: after the first step they are in place already, so the list
            // being loaded (i - 2) and the base table share one barrier
            if (i == M - 1) __syncthreads();
            const int dt1 = md.t[i] - md.t[i - 1], dt2 = md.t[i - 1] - md.t[i - 2];
            const int na = sm.cnt[sA], nb = sm.cnt[sB];
            const float *an = sm.alpha[cur];
            const bool last = i == M - 1;
            // base(b, a); rows/columns of empty slots are never read
            for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
                const int b = (int)__umulhi((unsigned)e, divL), a = e - b * L;
                const bool ra = a < na, rb = b < nb;
                if ((ra || a == E) && (rb || b == E)) {
                    const float al = last ? 0.0f : an[a * L + b];   // alpha_{i+1}(z_i = a, z_{i-1} = b)
                    float bs;
                    if (ra && rb) bs = base_cost(sm.u[sA][a], lam2, dt1, sm.t[sA][a], sm.t[sB][b], al);
                    else bs = __fadd_rn(sm.u[sA][a], al);
                    sm.base[b * L + a] = bs;
                }
            }
            __syncthreads();
            const float A1 = sm.ang[0], A2 = sm.ang[1];
            const int nc = sm.cnt[sC];
            // branch and bound (exact): v(a, b, c) >= base(b, a), and no open cell of row b has a best above
            // thr(b). A warp per row keeps the a with base <= thr(b) that may follow b (any real a after eps)
            // and ranks them by (base, slot) by counting.
            {
                const unsigned full = 0xffffffffu;
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                for (int b = warp; b < L; b += kDummyThreads / 32) {
                    if (!(b < nb || b == E)) continue;
                    const bool rb = b < nb;
                    const float *brow = sm.base + b * L;
                    const int tb = rb ? sm.t[sB][b] : 0, ib = rb ? sm.id[sB][b] : -3;
                    float key[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int a = lane + 32 * h;
                        key[h] = a < na && (!rb || (sm.id[sA][a] != ib && sm.t[sA][a] >= tb)) ? brow[a] : inf;
                    }
                    float thr = brow[E];
                    if (rb) {
                        float m = key[0];
                        int s = lane;
                        if (key_less(key[1], lane + 32, m, s)) { m = key[1]; s = lane + 32; }
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            const float om = __shfl_xor_sync(full, m, off);
                            const int os = __shfl_xor_sync(full, s, off);
                            if (key_less(om, os, m, s)) { m = om; s = os; }
                        }
                        // the second bound can only matter below base(b, eps): skip its feasibility scan otherwise
                        if (m < inf && m + gmax + 1e-6f * fabsf(m) < thr) {
                            // a1 = s must be feasible with every open c and with (b, eps)
                            const int t1 = sm.t[sA][s], i1 = sm.id[sA][s];
                            bool bad = lane == 0 && p.T > 0 && t1 - tb >= p.T;
                            for (int c = lane; c < nc; c += 32) {
                                const int tc = sm.t[sC][c], ic = sm.id[sC][c];
                                const bool open = ic != ib && tc <= tb && (p.T <= 0 || tb - tc < p.T);
                                if (open && (i1 == ic || (p.T > 0 && t1 - tc >= p.T))) bad = true;
                            }
                            if (!__any_sync(full, bad)) thr = fminf(thr, m + gmax + 1e-6f * fabsf(m));
                        }
                    }
                    const bool k0 = key[0] < inf && key[0] <= thr, k1 = key[1] < inf && key[1] <= thr;
                    const unsigned m0 = __ballot_sync(full, k0), m1 = __ballot_sync(full, k1);
                    int r0 = 0, r1 = 0;
                    for (unsigned mm = m0; mm; mm &= mm - 1) {
                        const int l = __ffs(mm) - 1;
                        const float kk = __shfl_sync(full, key[0], l);
                        r0 += key_less(kk, l, key[0], lane);
                        r1 += key_less(kk, l, key[1], lane + 32);
                    }
                    for (unsigned mm = m1; mm; mm &= mm - 1) {
                        const int l = __ffs(mm) - 1;
                        const float kk = __shfl_sync(full, key[1], l);
                        r0 += key_less(kk, l + 32, key[0], lane);
                        r1 += key_less(kk, l + 32, key[1], lane + 32);
                    }
                    if (k0) sm.srt[b][r0] = (uint8_t)lane;
                    if (k1) sm.srt[b][r1] = (uint8_t)(lane + 32);
                    if (lane == 0) {
                        sm.kept[b] = (uint8_t)(__popc(m0) + __popc(m1));
                        if (rb) {   // the cells of a real row read R(a, c) of its kept a
                            if (m0) atomicOr(&sm.akept[0], m0);
                            if (m1) atomicOr(&sm.akept[1], m1);
                        }
                    }
                    // directions of the kept pairs of a real b, the only ones the cells read: lane r takes the
                    // kept a of rank r
                    if (rb) {
                        __syncwarp();
                        const int nk = __popc(m0) + __popc(m1);
                        const float2 xb = sm.xy[sB][b];
                        for (int r = lane; r < nk; r += 32) {
                            const int a = sm.srt[b][r];
                            sm.p1[b * L + a] = __fadd_rn(A1, direction(xb, sm.xy[sA][a]));
                            sm.p2[b * L + a] = __fadd_rn(A2, direction(sm.xy[sA][a], xb));
                        }
                    }
                }
            }
            __syncthreads();
            // R(a, c) = theta(a->c) for the a some real row keeps, where (a, c) can be feasible (with W^d small
            // most rows keep no a: their cells take eps without any direction)
            {
                const unsigned k0 = sm.akept[0], k1 = sm.akept[1];
                if (k0 | k1) {
                    for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
                        const int a2 = (int)__umulhi((unsigned)e, divL), c = e - a2 * L;
                        if (a2 >= na || c >= nc || !(((a2 < 32 ? k0 : k1) >> (a2 & 31)) & 1u)) continue;
                        if (sm.t[sC][c] <= sm.t[sA][a2] && !(p.T > 0 && sm.t[sA][a2] - sm.t[sC][c] >= p.T))
                            sm.r[a2 * kRL + c] = direction(sm.xy[sA][a2], sm.xy[sC][c]);
                    }
                }
            }
            __syncthreads();
            float *ac = sm.alpha[cur ^ 1];
            uint8_t *bt = beta + (int64_t)(i - 2) * L * L;
            // real cells (b, c) in groups of four consecutive c: one walk of b's base-sorted row serves the
            // group, and stops at the first base above every open cell's best (exact: v >= base)
            const int G = (nc + 3) >> 2;
            const unsigned divG = 0xffffffffu / (unsigned)max(G, 2) + 1u;   // e / G as for e / L
            for (int e = threadIdx.x; e < nb * G; e += blockDim.x) {
                const int b = G == 1 ? e : (int)__umulhi((unsigned)e, divG), c0 = 4 * (e - b * G);
                const int tb = sm.t[sB][b], ib = sm.id[sB][b];
                const float *brow = sm.base + b * L;
                const int nk = sm.kept[b];   // 0: every open cell of the group takes eps, no direction needed
                float best[4], q1[4];
                int arg[4], tcq[4], icq[4];
                bool open[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + q;
                    const bool inc = c < nc;
                    tcq[q] = inc ? sm.t[sC][c] : 0;
                    icq[q] = inc ? sm.id[sC][c] : -3;
                    open[q] = inc && icq[q] != ib && tcq[q] <= tb && (p.T <= 0 || tb - tcq[q] < p.T);
                    q1[q] = open[q] && nk > 0 ? direction(sm.xy[sB][b], sm.xy[sC][c]) : 0.0f;
                    best[q] = open[q] ? brow[E] : inf;   // (eps, b, c) is feasible with every open cell
                    arg[q] = open[q] ? E : 255;
                }
                const int nopen = (int)open[0] + (int)open[1] + (int)open[2] + (int)open[3];
                const unsigned long long q1a = pk2(q1[0], q1[1]), q1b = pk2(q1[2], q1[3]);
                const unsigned long long lamp = pk2(lam23, lam23);
                const uint8_t *order = sm.srt[b];
                for (int k = 0; k < nk; ++k) {
                    const int a = order[k];
                    const float ba = brow[a];
                    float bmax = -inf;
#pragma unroll
                    for (int q = 0; q < 4; ++q) bmax = fmaxf(bmax, open[q] ? best[q] : -inf);
                    if (ba > bmax) break;
                    if constexpr (kCount) n_eval += nopen;
                    const int ta = sm.t[sA][a], ia = sm.id[sA][a];   // kept: ia != ib, ta >= tb
                    const float p1 = sm.p1[b * L + a], p2 = sm.p2[b * L + a];
                    // R past the last c is never initialised: those lanes of v are discarded (open is false)
                    const float4 r4 = *reinterpret_cast<const float4 *>(sm.r + a * kRL + c0);
                    const unsigned long long bp = pk2(ba, ba), p1p = pk2(p1, p1), p2p = pk2(p2, p2);
                    float v[4];
                    triple_cost2(bp, p1p, p2p, q1a, pk2(r4.x, r4.y), lamp, v[0], v[1]);
                    triple_cost2(bp, p1p, p2p, q1b, pk2(r4.z, r4.w), lamp, v[2], v[3]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool ok = open[q] && ia != icq[q] && !(p.T > 0 && ta - tcq[q] >= p.T);
                        if (ok && (v[q] < best[q] || (v[q] == best[q] && a < arg[q]))) { best[q] = v[q]; arg[q] = a; }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + q;
                    if (c < nc) {
                        ac[b * L + c] = open[q] ? cell_alpha(best[q], lam2, dt2, tb, tcq[q]) : inf;
                        bt[b * L + c] = (uint8_t)(open[q] ? arg[q] : 255);
                    }
                }
            }
            // cells holding eps (row b = eps over every c, column c = eps over the real b): a triple holding
            // eps costs base(b, a) alone, so in ranked order the first feasible kept a is the smallest (lowest
            // slot among equals); eps (the last slot) only if below it. An a left out of row eps costs more
            // than base(eps, eps); for a real b either the same holds or a1, the first kept, is feasible with
            // (b, eps)
            for (int e = threadIdx.x; e < nc + 1 + nb; e += blockDim.x) {
                const int b = e <= nc ? E : e - (nc + 1);
                const int c = e < nc ? e : E;
                const bool rb = b < nb, rc = c < nc;
                const float *brow = sm.base + b * L;
                const uint8_t *order = sm.srt[b];
                const int tr = rc ? sm.t[sC][c] : (rb ? sm.t[sB][b] : 0);   // the other real point
                const int ir = rc ? sm.id[sC][c] : (rb ? sm.id[sB][b] : -3);
                const bool any = !rb && !rc;
                float best = inf;
                int arg = 255;
                const int nk = sm.kept[b];
                for (int k = 0; k < nk; ++k) {
                    const int a = order[k];
                    const int ta = sm.t[sA][a];
                    if (!any && (sm.id[sA][a] == ir || ta < tr || (p.T > 0 && ta - tr >= p.T))) continue;
                    best = brow[a];
                    arg = a;
                    break;
                }
                if (brow[E] < best) { best = brow[E]; arg = E; }
                ac[b * L + c] = best;
                bt[b * L + c] = (uint8_t)arg;
            }
            cur ^= 1;
            __syncthreads();
        }
        // Eq. 13 over (z_1 = j1, z_2 = j2) in C_1 + eps, C_2 + eps: U + U + alpha_3(j2, j1)
        const float *a3 = sm.alpha[cur];
        const int n0 = ccnt[0], n1 = ccnt[1];
        DummyBest mine{inf, 0x7fffffff, 0x7fffffff};
        for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
            const int j1 = (int)__umulhi((unsigned)e, divL), j2 = e - j1 * L;
            if (!((j1 < n0 || j1 == E) && (j2 < n1 || j2 == E))) continue;
            const float u1 = j1 == E ? ueps : cu[j1], u2 = j2 == E ? ueps : cu[(int64_t)K + j2];
            const float al = M == 2 ? 0.0f : a3[j2 * L + j1];
            const float v = __fadd_rn(__fadd_rn(u1, u2), al);
            if (v < inf && dummy_better(v, j1, j2, mine)) mine = DummyBest{v, j1, j2};
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            DummyBest o{__shfl_xor_sync(0xffffffffu, mine.v, off), __shfl_xor_sync(0xffffffffu, mine.j1, off),
                        __shfl_xor_sync(0xffffffffu, mine.j2, off)};
            if (dummy_better(o.v, o.j1, o.j2, mine)) mine = o;
        }
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            DummyBest best = red[0];
            for (int w = 1; w < kDummyThreads / 32; ++w)
                if (dummy_better(red[w].v, red[w].j1, red[w].j2, best)) best = red[w];
            int32_t *row = assign + un.out_a;
            if (best.v < inf) {
                int s2 = best.j1, s1 = best.j2;   // slots of z_{i-2}, z_{i-1}
                auto out = [&](int i, int s) {
                    row[md.perm[i]] = s == E ? -2 : sc.perm[cidx[(int64_t)i * K + s]];
                };
                out(0, s2);
                out(1, s1);
                for (int i = 2; i < M; ++i) {
                    const int sa = beta[(int64_t)(i - 2) * L * L + s1 * L + s2];
                    out(i, sa);
                    s2 = s1;
                    s1 = sa;
                }
                energy[un.out_e] = best.v;
            } else {
                for (int i = 0; i < M; ++i) row[i] = -1;
                energy[un.out_e] = inf;
            }
        }
        __syncthreads();   // tables, lists and the reduction slots are reused by the next unit
    }
    if constexpr (kCount) {
        if (n_eval) atomicAdd(evaluated, n_eval);
    }
}

}  // namespace

int64_t dummy_scratch_bytes(int K, int max_M, int grid)
{
    const int64_t L = K + 1;
    return (int64_t)grid * std::max(max_M - 2, 1) * L * L;
}

int dummy_grid()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 0;
    return sms * 2;
}

cudaError_t launch_recurse_dummy(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, float wd, const int32_t *cand_idx, const float *cand_u,
                                 const int32_t *cand_cnt, uint8_t *scratch, int max_M, int grid, float *energy,
                                 int32_t *assign, unsigned long long *evaluated, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    if (p.K > kMaxK) return cudaErrorInvalidValue;
    const size_t smem = sizeof(DummySmem);
    auto kern = evaluated ? dummy_recurse_kernel<true> : dummy_recurse_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t per_cta = (int64_t)std::max(max_M - 2, 1) * (p.K + 1) * (p.K + 1);
    const int g = (int)std::min<int64_t>(n_units, grid);
    prof_begin(kProfRecurse, st);
    kern<<<g, kDummyThreads, smem, st>>>(units, n_units, models, scenes, p, wd, cand_idx, cand_u, cand_cnt, scratch,
                                         per_cta, energy, assign, evaluated);
    e = cudaGetLastError();
    prof_end(kProfRecurse, st);
    return e;
}

}  // namespace hgm
