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
// lives in shared memory (Sec. 3.5's local-memory rows, extended to the whole
// alpha table and the geometry). Writing theta(p->q) = atan2(q-p) and A1, A2
// for the model's angles at i-1 and at i, the angle differences of Eq. 6 are
//   d1 = wrap(A1 + theta(b->a) - theta(b->c)),  d2 = wrap(A2 + theta(a->b) - theta(a->c))
// so that, with every pair-only term hoisted (Sec. 3.3's look-up idea applied
// to the geometry), a triple costs two subtractions, two circular folds, a
// squared norm, a square root and an FMA:
//   base(a,b) = U(a) + lambda2 Delta(i,i-1) + alpha_{i+1}(a,b),  p1(a,b) = wrap(A1 + theta(b->a))
//   v(a,b,c)  = base(a,b) + lambda2 lambda3 sqrt(d1^2 + d2^2)   [+ lambda2 Delta(i-1,i-2), after the min]
// Infeasible pairs are +inf (causality t'(c)<=t'(b)<=t'(a), closeness
// t'(a)-t'(c) < T, distinct points; Eqs. 7-8, Sec. 3.2's validity mask).
//
// Exact branch and bound: the geometric term is bounded, 0 <= D^g <= pi*sqrt(2),
// so v(a,b,c) >= base(a,b), and any a with base(a,b) > base(w,b) + lambda2
// lambda3 pi sqrt(2) (plus rounding slack) can never beat a feasible witness w.
// Per b, the witness is the a of smallest base; for the rare c where it is
// infeasible, the smallest base feasible with c raises the threshold. Only the
// kept a (about a quarter on the paper-shaped workloads) enter the triple
// loop, in increasing slot order with a strict '<', so the lowest slot still
// wins exact ties -- the result is bit-identical to the full minimisation.
//
// Work split per step (two CTA barriers): phase 1, warps build the kept lists
// of one b each; phase 2, the theta(a->c) rows of the kept a, then warp 0
// orders the b by decreasing kept count and lays out the tile table; phase 3,
// tiles of one b and CT consecutive c with t'(c) <= t'(b) are flattened across
// the CTA's threads in that order (similar loop lengths within a warp), each
// thread looping over the kept a of its b. The per-step model constants come
// from a table built at model creation, and the list C of the next step is
// fetched from global memory during phases 1-2 and stored in the buffer of the
// list A, which phase 3 no longer reads, so no step waits on a global load.
#include "recurse_common.cuh"

namespace hgm {
namespace {

constexpr float kInf = __builtin_huge_valf();
constexpr float kGeoMax = 4.45f;   // > pi*sqrt(2) = 4.4429, bound of the FP32 D^g

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <int KM>
struct List {
    float2 xy[KM];
    int32_t t[KM];
    float u[KM];
    int32_t idx[KM];
    int32_t n;
};

template <int KM, int NT>
struct Smem {
    static constexpr int RS = KM + 4;     // row stride of r (16-byte rows, bank skew)
    float2 fb[KM * KM];                   // per b: kept (base, p1) in increasing a, at b*KM + k
    float r[KM * RS];                     // theta(a->c) or +inf, at a*RS + c
    static constexpr int AS = KM + 1;     // row stride of alpha (conflict-free row and column access)
    float alpha[KM * AS];                 // alpha_{i+1}(a,b) at b*AS + a; alpha_i(b,c) written at c*AS + b
    uint8_t fs[KM * KM];                  // slot a of each kept entry
    uint8_t used[KM];                     // a kept for some b (its r row is needed)
    int32_t fn[KM];                       // number of kept a per b
    uint8_t tile_b[KM * KM / 4];          // b of every tile of the step (tiles of >= 4 cells)
    uint16_t tbase[KM];                   // first tile of b
    uint8_t tcount[KM];                   // tiles of b
    int32_t hist[KM + 1];                 // tiles per kept count (counting sort of the b), then bucket starts
    int32_t ntile;                        // tiles of the step
    List<KM> list[3];
    float4 geo[2];                        // model constants of step i at geo[i & 1]
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

// (value, slot) minimum with ties to the lower slot
__device__ __forceinline__ void argmin_merge(float &v, int &k, float ov, int ok)
{
    if (ov < v || (ov == v && ok < k)) { v = ov; k = ok; }
}

// kCount = true builds the accounting variant: identical work, plus a count of
// the (a, b, c) evaluations the triple loop performs (kept a x CT per tile).
template <int KM, int NT, int CT, bool kCount>
__global__ void __launch_bounds__(NT, (KM > 32 ? 3 : 4))
recurse_kernel(const Unit *__restrict__ units, int64_t n_units, const ModelRec *__restrict__ models,
               const SceneRec *__restrict__ scenes, Params p, const int32_t *__restrict__ cand_idx,
               const float *__restrict__ cand_u, const int32_t *__restrict__ cand_cnt, uint8_t *__restrict__ beta,
               UnitResult *__restrict__ res, int *__restrict__ work_counter, unsigned long long *__restrict__ evaluated)
{
    unsigned long long n_eval = 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<KM, NT> &sm = *reinterpret_cast<Smem<KM, NT> *>(smem_raw);
    constexpr int RS = Smem<KM, NT>::RS;
    constexpr int AS = Smem<KM, NT>::AS;
    constexpr int AQ = KM / 32;            // slots per lane in warp-wide passes
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = p.K;
    const int T = p.T;
    const float lam2 = p.lambda2;
    const float lam23 = p.lambda2 * p.lambda3;
    const float gmax = lam23 * kGeoMax;

    for (;;) {
        if (tid == 0) sm.unit = atomicAdd(work_counter, 1);
        __syncthreads();
        const int64_t u = sm.unit;
        if (u >= n_units) {
            if constexpr (kCount) atomicAdd(evaluated, n_eval);
            break;
        }
        const Unit un = units[u];
        const ModelRec md = models[un.model];
        const SceneRec sc = scenes[un.scene];
        const int M = md.M;
        const int32_t *cidx = cand_idx + un.cand;
        const float *cu = cand_u + un.cand;
        const int32_t *ccnt = cand_cnt + un.cand / K;
        uint8_t *ubeta = beta + un.beta;

        // alpha_{M+1} == 0 (Eq. 11); the three lists and the constants of the first step
        for (int e = tid; e < KM * AS; e += NT) sm.alpha[e] = 0.0f;
        for (int q = 1; q <= 3 && q <= M; ++q)
            load_list<KM>(sm.list[(M - q) % 3], sc, cidx + (int64_t)(M - q) * K, cu + (int64_t)(M - q) * K,
                          ccnt[M - q], tid, NT);
        if (tid < KM) sm.used[tid] = 0;
        if (tid == 0 && M >= 3) sm.geo[(M - 1) & 1] = md.geo[M - 1];
        __syncthreads();

        for (int i = M - 1; i >= 2; --i) {
            List<KM> &LA = sm.list[i % 3];
            List<KM> &LB = sm.list[(i - 1) % 3];
            List<KM> &LC = sm.list[(i - 2) % 3];
            const float4 g = sm.geo[i & 1];
            const float A1 = g.x, k2 = g.y;
            const int dt_ab = __float_as_int(g.z), dt_bc = __float_as_int(g.w);
            const int na = LA.n, nb = LB.n, nc = LC.n;

            // list C of the next step (chain index i-3): first half of the fetch
            const bool pf = i >= 3 && tid < K;
            int pf_n = 0, pf_j = -1;
            float pf_u = kInf;
            if (pf) {
                pf_n = ccnt[i - 3];
                pf_j = cidx[(int64_t)(i - 3) * K + tid];
                pf_u = cu[(int64_t)(i - 3) * K + tid];
            }

            // ---- phase 1: per b (one warp each) the kept a list and the tile count
            // per-lane data of the lane's a and c slots, shared by every b of the warp
            int la_t[AQ], la_i[AQ], lc_t[AQ], lc_i[AQ];
            float la_u[AQ];
#pragma unroll
            for (int q = 0; q < AQ; ++q) {
                const int a = lane + 32 * q;
                la_t[q] = LA.t[a];
                la_i[q] = LA.idx[a];
                la_u[q] = LA.u[a];
                lc_t[q] = a < nc ? LC.t[a] : 0x7fffffff;   // c outside the list never qualifies
                lc_i[q] = LC.idx[a];
            }
            for (int b = warp; b < KM; b += NW) {
                if (b >= nb) {
                    if (lane == 0) { sm.fn[b] = 0; sm.tcount[b] = 0; }
                    continue;
                }
                const float2 pb = LB.xy[b];
                const int tb = LB.t[b], ib = LB.idx[b];
                float base[AQ];
                float bv = kInf;
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    const int a = lane + 32 * q;
                    base[q] = kInf;
                    if (a < na && la_t[q] >= tb && la_i[q] != ib)
                        base[q] = base_cost(la_u[q], lam2, dt_ab, la_t[q], tb, sm.alpha[b * AS + a]);
                    bv = fminf(bv, base[q]);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) bv = fminf(bv, __shfl_xor_sync(0xffffffffu, bv, off));
                int bk = 0;   // witness: the lowest slot with the smallest base
#pragma unroll
                for (int q = AQ - 1; q >= 0; --q) {
                    const uint32_t hit = __ballot_sync(0xffffffffu, base[q] == bv);
                    if (hit) bk = __ffs(hit) - 1 + 32 * q;
                }
                // c with t'(c) <= t'(b) form a prefix of C: tiles cover it
                int ccount = 0;
#pragma unroll
                for (int q = 0; q < AQ; ++q) ccount += __popc(__ballot_sync(0xffffffffu, lc_t[q] <= tb));
                if (lane == 0) sm.tcount[b] = (uint8_t)((ccount + CT - 1) / CT);
                if (!(bv < kInf)) {
                    if (lane == 0) sm.fn[b] = 0;
                    continue;
                }
                float thr = bv + gmax + 1e-6f * bv;
                // cells (b,c) whose witness bk is infeasible: raise thr by their own best feasible base
                const int tw = LA.t[bk], iw = LA.idx[bk];
                uint32_t bad[AQ];
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    const bool bd = lc_t[q] <= tb && lc_i[q] != ib && ((T > 0 && tw - lc_t[q] >= T) || iw == lc_i[q]);
                    bad[q] = __ballot_sync(0xffffffffu, bd);
                }
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    while (bad[q]) {
                        const int c = __ffs(bad[q]) - 1 + 32 * q;
                        bad[q] &= bad[q] - 1;
                        const int tc = LC.t[c], ic = LC.idx[c];
                        float mv = kInf;
#pragma unroll
                        for (int qa = 0; qa < AQ; ++qa) {
                            if (!((T > 0 && la_t[qa] - tc >= T) || la_i[qa] == ic)) mv = fminf(mv, base[qa]);
                        }
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) mv = fminf(mv, __shfl_xor_sync(0xffffffffu, mv, off));
                        if (mv < kInf) thr = fmaxf(thr, mv + gmax + 1e-6f * mv);
                    }
                }
                // keep base <= thr, compacted in increasing a
                int kept = 0;
                float *fbf = reinterpret_cast<float *>(sm.fb + b * KM);
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    const int a = lane + 32 * q;
                    const bool keep = base[q] <= thr;
                    const uint32_t km = __ballot_sync(0xffffffffu, keep);
                    if (keep) {
                        const int pos = kept + __popc(km & lanemask_lt());
                        fbf[2 * pos] = base[q];
                        sm.fs[b * KM + pos] = (uint8_t)a;
                        sm.used[a] = 1;
                    }
                    kept += __popc(km);
                }
                __syncwarp();
                // p1 = A1 + theta(b->a) of the kept entries, one lane per entry
                for (int pos = lane; pos < kept; pos += 32) {
                    const float2 pa = LA.xy[sm.fs[b * KM + pos]];
                    fbf[2 * pos + 1] = wrap_pi(__fadd_rn(A1, direction(pb, pa)));
                }
                if (lane == 0) sm.fn[b] = kept;
            }
            __syncthreads();

            // list C of the next step: second half of the fetch (positions and frames)
            float2 pf_xy = make_float2(0.f, 0.f);
            int pf_t = 0x3fffffff;
            const bool pf_ok = pf && tid < pf_n;
            if (pf_ok) {
                pf_xy = sc.xy[pf_j];
                pf_t = sc.t[pf_j];
            }

            // ---- phase 2: theta(a->c) rows of the kept a; then warp 0 lays out the tile table
            if (tid == 32 && i >= 3) sm.geo[(i - 1) & 1] = md.geo[i - 1];
            for (int e = tid; e < na * KM; e += NT) {
                const int a = e / KM, c = e % KM;
                if (!sm.used[a]) continue;
                float r = kInf;
                if (c < nc) {
                    const int ta = LA.t[a], tc = LC.t[c];
                    // kept pairs have t'(c) <= t'(b) <= t'(a): entries with t'(c) > t'(a) are never read
                    if (tc <= ta && !(T > 0 && ta - tc >= T) && LA.idx[a] != LC.idx[c]) {
                        r = direction(LA.xy[a], LC.xy[c]);                   // theta(a->c)
                    }
                }
                sm.r[a * RS + c] = r;
            }
            if (warp == 0) {
                // tiles of b in decreasing kept count (counting sort; order inside a count is free):
                // the lanes of a warp then loop over similar numbers of a
                constexpr int HB = KM + 1, HE = (HB + 31) / 32;
                for (int k = lane; k < HB; k += 32) sm.hist[k] = 0;
                __syncwarp();
                int key[AQ], cnt[AQ];
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    const int b = lane + 32 * q;
                    cnt[q] = sm.tcount[b];
                    key[q] = KM - sm.fn[b];
                    if (cnt[q]) atomicAdd(&sm.hist[key[q]], cnt[q]);
                }
                __syncwarp();
                int loc[HE], sum = 0;
#pragma unroll
                for (int e = 0; e < HE; ++e) {
                    const int k = lane * HE + e;
                    loc[e] = k < HB ? sm.hist[k] : 0;
                    sum += loc[e];
                }
                int x = sum;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, off);
                    if (lane >= off) x += y;
                }
                int pre = x - sum;
#pragma unroll
                for (int e = 0; e < HE; ++e) {
                    const int k = lane * HE + e;
                    if (k < HB) sm.hist[k] = pre;
                    pre += loc[e];
                }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < AQ; ++q) {
                    if (cnt[q]) {
                        const int b = lane + 32 * q;
                        const int t0 = atomicAdd(&sm.hist[key[q]], cnt[q]);
                        sm.tbase[b] = (uint16_t)t0;
                        for (int t = 0; t < cnt[q]; ++t) sm.tile_b[t0 + t] = (uint8_t)b;
                    }
                }
                const int total = __shfl_sync(0xffffffffu, x, 31);
                if (lane == 0) sm.ntile = total;
            }
            __syncthreads();

            // list A is not read from here on: its buffer receives list C of the next step
            if (pf) {
                LA.idx[tid] = pf_ok ? pf_j : -1;
                LA.xy[tid] = pf_xy;
                LA.t[tid] = pf_t;
                LA.u[tid] = pf_ok ? pf_u : kInf;
                if (tid == 0) LA.n = pf_n;
            }
            if (i >= 3 && tid >= K && tid < KM) {
                LA.idx[tid] = -1;
                LA.xy[tid] = make_float2(0.f, 0.f);
                LA.t[tid] = 0x3fffffff;
                LA.u[tid] = kInf;
            }
            if (tid < KM) sm.used[tid] = 0;

            // ---- phase 3: tiles (b, CT consecutive c)
            const int ntile = sm.ntile;
            uint8_t *bstep = ubeta + (int64_t)(i - 2) * K * K;
            for (int tile = tid; tile < ntile; tile += NT) {
                const int b = sm.tile_b[tile];
                const int c0 = (tile - sm.tbase[b]) * CT;
                const float2 pb = LB.xy[b];
                const int tb = LB.t[b], ib = LB.idx[b];
                float q1[CT], best[CT];
                int arg[CT];
#pragma unroll
                for (int k = 0; k < CT; ++k) {
                    const int c = c0 + k;
                    const bool ok = c < nc && LC.t[c] <= tb && LC.idx[c] != ib;
                    q1[k] = ok ? direction(pb, LC.xy[c]) : kInf;   // theta(b->c)
                    best[k] = kInf;
                    arg[k] = kNoSlot;
                }
                const int nf = sm.fn[b];

                const float2 *fbb = sm.fb + b * KM;
                const uint8_t *fsb = sm.fs + b * KM;
                // cells in pairs: packed FP32x2 arithmetic, same roundings as triple_cost
                static_assert(CT % 4 == 0, "tiles of a multiple of 4 cells");
                unsigned long long q1p[CT / 2];
#pragma unroll
                for (int q = 0; q < CT / 2; ++q) q1p[q] = pk2(q1[2 * q], q1[2 * q + 1]);
                const unsigned long long lamp = pk2(lam23, lam23);
#pragma unroll 2
                for (int k = 0; k < nf; ++k) {
                    const float2 e = fbb[k];
                    const int a = fsb[k];
                    if constexpr (kCount) n_eval += CT;
                    const float p2 = __fadd_rn(e.y, k2);
                    const unsigned long long bp = pk2(e.x, e.x), p1p = pk2(e.y, e.y), p2p = pk2(p2, p2);
#pragma unroll
                    for (int q4 = 0; q4 < CT; q4 += 4) {
                        const float4 r4 = *reinterpret_cast<const float4 *>(&sm.r[a * RS + c0 + q4]);
                        float v[4];
                        triple_cost2(bp, p1p, p2p, q1p[q4 / 2], pk2(r4.x, r4.y), lamp, v[0], v[1]);
                        triple_cost2(bp, p1p, p2p, q1p[q4 / 2 + 1], pk2(r4.z, r4.w), lamp, v[2], v[3]);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (v[q] < best[q4 + q]) { best[q4 + q] = v[q]; arg[q4 + q] = a; }
                    }
                }
#pragma unroll
                for (int q = 0; q < CT; ++q) {
                    const int c = c0 + q;
                    if (c < nc) {
                        float al = kInf;
                        int bt = kNoSlot;
                        if (best[q] < kInf) {
                            al = cell_alpha(best[q], lam2, dt_bc, tb, LC.t[c]);
                            bt = arg[q];
                        }
                        sm.alpha[c * AS + b] = al;
                        bstep[b * K + c] = (uint8_t)bt;
                    }
                }
            }
            // cells (b, c) beyond the tiled prefix are infeasible
            for (int b = warp; b < nb; b += NW) {
                const int covered = sm.tcount[b] * CT;
                for (int c = covered + lane; c < nc; c += 32) {
                    sm.alpha[c * AS + b] = kInf;
                    bstep[b * K + c] = (uint8_t)kNoSlot;
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
                const int c = e / KM, b = e % KM;    // e = z1 * KM + z2: lexicographic order
                if (c < n0 && b < n1) argmin_merge(bv, bk, L0.u[c] + L1.u[b] + sm.alpha[c * AS + b], e);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                argmin_merge(bv, bk, __shfl_xor_sync(0xffffffffu, bv, off), __shfl_xor_sync(0xffffffffu, bk, off));
            if (lane == 0) { sm.red_v[warp] = bv; sm.red_k[warp] = bk; }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < NW; ++w) argmin_merge(bv, bk, sm.red_v[w], sm.red_k[w]);
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

template <int KM, int NT, int CT, bool kCount>
cudaError_t launch_recurse_t(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                             Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                             uint8_t *beta, UnitResult *res, int *work_counter, unsigned long long *evaluated,
                             cudaStream_t st)
{
    // three CTAs of 256 threads per SM: 3 x (shared memory + 1 KB reserved) <= 228 KB
    static_assert(KM != 64 || NT != 256 || 3 * (sizeof(Smem<KM, NT>) + 1024) <= 228 * 1024,
                  "recursion shared memory exceeds the three-CTA budget");
    auto kern = recurse_kernel<KM, NT, CT, kCount>;
    const size_t smem = sizeof(Smem<KM, NT>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > n_units) grid = n_units;
    if ((e = cudaMemsetAsync(work_counter, 0, sizeof(int), st)) != cudaSuccess) return e;
    prof_begin(kProfRecurse, st);
    kern<<<(unsigned)grid, NT, smem, st>>>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                                           work_counter, evaluated);
    prof_end(kProfRecurse, st);
    return cudaGetLastError();
}

template <bool kCount>
cudaError_t dispatch(int variant, const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                     Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt, uint8_t *beta,
                     UnitResult *res, int *work_counter, unsigned long long *evaluated, cudaStream_t st)
{
    if (p.K <= 32) {
        if (variant == 1)
            return launch_recurse_t<32, 128, 8, kCount>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt,
                                                        beta, res, work_counter, evaluated, st);
        return launch_recurse_t<32, 128, 4, kCount>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt,
                                                    beta, res, work_counter, evaluated, st);
    }
    if (variant == 1)
        return launch_recurse_t<64, 256, 8, kCount>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt,
                                                    beta, res, work_counter, evaluated, st);
    if (variant == 2)
        return launch_recurse_t<64, 128, 4, kCount>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt,
                                                    beta, res, work_counter, evaluated, st);
    return launch_recurse_t<64, 256, 4, kCount>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta,
                                                res, work_counter, evaluated, st);
}

int g_variant = 0;   // recursion variant: 0 = 4 c per tile, 1 = 8 c per tile, 2 = 4 c per tile on 128 threads

}  // namespace

namespace {
__global__ void model_geo_kernel(const float2 *__restrict__ xy, const int32_t *__restrict__ t, int M,
                                 float4 *__restrict__ geo)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i >= 2) {
            const float2 mi = xy[i], mj = xy[i - 1], mk = xy[i - 2];
            const float A1 = signed_angle(mj, mi, mk);   // at i-1, from ->i to ->i-2
            const float A2 = signed_angle(mi, mj, mk);   // at i, from ->i-1 to ->i-2
            g = make_float4(A1, wrap_pi(__fadd_rn(__fsub_rn(A2, A1), kPi)), __int_as_float(t[i] - t[i - 1]),
                            __int_as_float(t[i - 1] - t[i - 2]));
        }
        geo[i] = g;
    }
}
}  // namespace

cudaError_t launch_model_geo(const float2 *xy, const int32_t *t, int M, float4 *geo, cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    model_geo_kernel<<<(M + 127) / 128, 128, 0, st>>>(xy, t, M, geo);
    return cudaGetLastError();
}

int recurse_variant_count() { return 3; }
void set_recurse_variant(int v) { g_variant = (v >= 0 && v < 3) ? v : 0; }
int get_recurse_variant() { return g_variant; }

cudaError_t launch_recurse(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                           Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                           uint8_t *beta, UnitResult *res, int *work_counter, cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    if (p.K <= 16)   // short lists (pruned form): one warp per unit
        return launch_recurse_small(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res, st);
    return dispatch<false>(g_variant, units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                           work_counter, nullptr, st);
}

cudaError_t launch_recurse_count(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                                 uint8_t *beta, UnitResult *res, int *work_counter, unsigned long long *evaluated,
                                 cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    return dispatch<true>(g_variant, units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                          work_counter, evaluated, st);
}

}  // namespace hgm
