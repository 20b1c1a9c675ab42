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
// so v(a,b,c) >= base(a,b), and an a with base(a,b) > m(b,c) + lambda2 lambda3
// pi sqrt(2) (plus rounding slack), m(b,c) the smallest base among the a
// feasible with the cell, can never beat the cell's best. Any threshold at or
// above max_c m(b,c) + that bound is therefore exact. Per b the witness w is the
// a of smallest base, m(b,c) = base(w) wherever w is feasible with c; for the
// cells where it is not, m(b,c) is at most the runner-up's base when the
// runner-up is feasible with c; where neither the witness nor the runner-up is
// feasible with some c, no threshold is taken and every a of b is kept. (Which
// c rule them out is read off C by bisection: C is sorted by scene index, hence
// by time, so "too far in time" is a prefix and "same point" a lookup.) Only
// the kept a (about a third of the feasible ones on the batched workload) enter the
// triple loop, in increasing slot order with a strict '<', so the lowest slot
// still wins exact ties -- the result is bit-identical to the full minimisation.
//
// Work split per step (three CTA barriers): phase 1, NP threads per b (adjacent
// lanes, interleaved a) build the kept lists with pairwise shuffles only, while
// the other warps compute the theta(a->c) table; then every thread takes part in
// ordering the b by decreasing kept count and laying out the tile table; phase
// 3, tiles of one b and CT consecutive c with
// t'(c) <= t'(b) are flattened across the CTA's threads in that order (similar
// loop lengths within a warp), each thread looping over the kept a of its b.
// The per-step model constants come from a table built at model creation, and
// the list C of the next step is fetched from global memory during phase 2 and
// stored in the buffer of the list A, which phase 3 no longer reads, so no step
// waits on a global load. Argmin bytes are written for the tiled cells only, a
// tile's four at once: the cells past b's time prefix are never on a chain, so
// the backtrack never reads them.
#include "backtrack.cuh"
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

// Kept entry k of b sits at a per-row rotation of its slot, so that the rows of different b -- whose
// starts are multiples of 32 banks apart -- spread over the banks when several b are read or written
// at the same position (phase 1 writes, the triple loop's reads).
template <int KM>
__device__ __forceinline__ int fb_at(int b, int k) { return b * KM + ((k + b) & (KM - 1)); }
template <int KM>
__device__ __forceinline__ int fs_at(int b, int k) { return b * KM + ((k + 4 * b) & (KM - 1)); }

template <int KM>
struct alignas(16) List {   // 16-byte aligned arrays: tiles read four consecutive entries at once
    float2 xy[KM];
    int32_t t[KM];
    float u[KM];
    int32_t idx[KM];
    int32_t n;
};

template <int KM, int NT, int NP>
struct Smem {
    static constexpr int RS = KM + 4;     // row stride of r (16-byte rows, bank skew)
    float2 fb[KM * KM];                   // per b: kept (base, p1) in increasing a, at b*KM + k
    float r[KM * RS];                     // theta(a->c) or +inf, at a*RS + c
    // row stride of alpha: phase 1 reads row b at a = NP k + h with lanes (b, h); conflict-free when
    // AS = NP (mod 32) and odd multiples are avoided: 65 for one thread per b, 66 for two
    static constexpr int AS = KM + NP;
    float alpha[KM * AS];                 // alpha_{i+1}(a,b) at b*AS + a (then base(a,b)); alpha_i(b,c) at c*AS + b
    uint8_t fs[KM * KM];                  // slot a of each kept entry, | 0x80 when a lies at b's position
    uint8_t fn[KM];                       // number of kept a per b
    uint8_t tile_b[KM * KM / 4];          // b of every tile of the step (tiles of >= 4 cells)
    uint16_t tbase[KM];                   // first tile of b
    uint8_t tcount[KM];                   // tiles of b
    int32_t pw[KM];                       // per b: (sort key << 5) | tile count, key 0 for b without tiles
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
// kFused = true builds the self-contained variant used for the exact fallback
// of the pruned form: the number of units is read from n_dev (written by an
// earlier kernel, so nothing waits on the host), the argmin tables of a unit
// live in a per-CTA scratch block (beta + blockIdx.x * beta_cta, reused unit
// after unit), and the CTA backtracks its own unit and writes the energy and
// the assignment itself.
template <int KM, int NT, int CT, int NP, int UR, bool kCount, bool kFused>
__global__ void __launch_bounds__(NT, (KM > 32 ? 3 : 4))
recurse_kernel(const Unit *__restrict__ units, int64_t n_units, const ModelRec *__restrict__ models,
               const SceneRec *__restrict__ scenes, Params p, const int32_t *__restrict__ cand_idx,
               const float *__restrict__ cand_u, const int32_t *__restrict__ cand_cnt, uint8_t *__restrict__ beta,
               UnitResult *__restrict__ res, int *__restrict__ work_counter, unsigned long long *__restrict__ evaluated,
               const int *__restrict__ n_dev, int64_t beta_cta, float *__restrict__ energy_out,
               int32_t *__restrict__ assign_out)
{
    if constexpr (kFused) {
        const int64_t nd = *n_dev;
        n_units = nd < n_units ? nd : n_units;
    }
    unsigned long long n_eval = 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<KM, NT, NP> &sm = *reinterpret_cast<Smem<KM, NT, NP> *>(smem_raw);
    constexpr int RS = Smem<KM, NT, NP>::RS;
    constexpr int AS = Smem<KM, NT, NP>::AS;
    constexpr int AQ = KM / 32;            // slots per lane in warp-wide passes
    constexpr int NW = NT / 32;
    constexpr int P1 = KM * NP;            // threads building the kept lists (NP per b); the rest: theta table
    constexpr int AH = KM / NP;            // a (and c) slots per list-building thread
    static_assert(NP == 1 || NP == 2, "one or two threads per b");
    static_assert(P1 % 32 == 0 && NT - P1 >= KM, "thread split");
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
        uint8_t *ubeta = kFused ? beta + (int64_t)blockIdx.x * beta_cta : beta + un.beta;

        // alpha_{M+1} == 0 (Eq. 11); the three lists and the constants of the first step
        for (int e = tid; e < KM * AS; e += NT) sm.alpha[e] = 0.0f;
        for (int q = 1; q <= 3 && q <= M; ++q)
            load_list<KM>(sm.list[(M - q) % 3], sc, cidx + (int64_t)(M - q) * K, cu + (int64_t)(M - q) * K,
                          ccnt[M - q], tid, NT);
        if (tid == 0 && M >= 3) sm.geo[(M - 1) & 1] = md.geo[M - 1];
        __syncthreads();

        for (int i = M - 1; i >= 2; --i) {
            List<KM> &LA = sm.list[i % 3];
            List<KM> &LB = sm.list[(i - 1) % 3];
            List<KM> &LC = sm.list[(i - 2) % 3];
            const float4 g = sm.geo[i & 1];
            const float A1 = g.x, k2 = g.y;
            // p2 = p1 + k2 uses theta(a->b) = theta(b->a) + pi, which fails for a and b at the same position
            // (both directions are atan2(0, 0) = 0, reading R1): such entries (flagged in fs) take k2c
            const float k2c = wrap_pi(__fsub_rn(k2, kPi));
            const int dt_ab = __float_as_int(g.z), dt_bc = __float_as_int(g.w);
            const int na = LA.n, nb = LB.n, nc = LC.n;

            // list C of the next step (chain index i-3) is fetched by the theta-table threads
            const int pfi = tid - P1;
            const bool pf = i >= 3 && pfi >= 0 && pfi < K;
            int pf_n = 0, pf_j = -1;
            float pf_u = kInf;
            float2 pf_xy = make_float2(0.f, 0.f);
            int pf_t = 0x3fffffff;
            bool pf_ok = false;

            if (tid < P1) {
                // ---- phase 1: the kept a list of b, NP threads per b (lanes h of a pair; a = NP k + h)
                const int b = tid / NP, h = tid % NP;
                const bool inb = b < nb;
                float2 pb = make_float2(0.f, 0.f);
                int tb = 0, ib = -1;
                if (inb) { pb = LB.xy[b]; tb = LB.t[b]; ib = LB.idx[b]; }
                float *arow = sm.alpha + b * AS;
                // smallest and second-smallest base (value, slot) over all feasible a
                float m1 = kInf, m2 = kInf;
                int s1 = 1 << 20, s2 = 1 << 20;
                // the a with t'(a) >= t'(b) form a suffix of list A (time order): the slots before it are never
                // feasible with b and are neither evaluated nor read below (k0: first k that can reach it)
                int k0 = 0;
                if (inb) {
                    int lo = 0, hi = na;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (LA.t[mid] < tb) lo = mid + 1;
                        else hi = mid;
                    }
                    k0 = lo / NP;
                }
                if (inb) {
#pragma unroll 4
                    for (int k = k0; k < AH; ++k) {
                        const int a = NP * k + h;
                        // slots past the list hold t = 0x3fffffff, idx = -1, u = inf: never feasible with b
                        const int ta = LA.t[a];
                        float bs = kInf;
                        if (a < na && ta >= tb && LA.idx[a] != ib)
                            bs = base_cost(LA.u[a], lam2, dt_ab, ta, tb, arow[a]);
                        arow[a] = bs;   // base(a,b) replaces alpha_{i+1}(a,b): read once, by this thread
                        if (bs < m1) { m2 = m1; s2 = s1; m1 = bs; s1 = a; }
                        else if (bs < m2) { m2 = bs; s2 = a; }
                    }
                }
                if constexpr (NP == 2) {
                    // merge the pair's (value, slot) top-2 lists; ties go to the lower slot
                    const float om1 = __shfl_xor_sync(0xffffffffu, m1, 1), om2 = __shfl_xor_sync(0xffffffffu, m2, 1);
                    const int os1 = __shfl_xor_sync(0xffffffffu, s1, 1), os2 = __shfl_xor_sync(0xffffffffu, s2, 1);
                    if (om1 < m1 || (om1 == m1 && os1 < s1)) {
                        if (m1 < om2 || (m1 == om2 && s1 < os2)) { m2 = m1; s2 = s1; }
                        else { m2 = om2; s2 = os2; }
                        m1 = om1; s1 = os1;
                    } else if (om1 < m2 || (om1 == m2 && os1 < s2)) {
                        m2 = om1; s2 = os1;
                    }
                }
                const float bv = m1;
                // c with t'(c) <= t'(b) form a prefix of C (time order): its length by binary search
                int ccount = 0;
                if (inb) {
                    int lo = 0, hi = nc;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (LC.t[mid] <= tb) lo = mid + 1;
                        else hi = mid;
                    }
                    ccount = lo;
                }
                const bool live = inb && bv < kInf && ccount > 0;
                // cells (b,c) where the witness s1 is infeasible: their best base is the second smallest over
                // the a feasible with c -- exactly m2 when the runner-up s2 is feasible with c; otherwise
                // (rare) every a is kept
                bool anybad = false, loose = false;
                if (live) {
                    // C is in increasing scene index, hence in increasing time: the c with t'(c) <= x form a
                    // prefix, and a point's slot in C is found by bisection. The cells of b's own point are
                    // infeasible and never count; the witness and the runner-up are feasible with b, so their
                    // points differ from b's.
                    const int tw = LA.t[s1], iw = LA.idx[s1];
                    const bool has2 = m2 < kInf;
                    const int t2 = has2 ? LA.t[s2] : 0, i2 = has2 ? LA.idx[s2] : -2;
                    auto count_le = [&](int x) {
                        int lo = 0, hi = ccount;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (LC.t[mid] <= x) lo = mid + 1;
                            else hi = mid;
                        }
                        return lo;
                    };
                    auto slot_of = [&](int j) {
                        int lo = 0, hi = ccount;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (LC.idx[mid] < j) lo = mid + 1;
                            else hi = mid;
                        }
                        return lo < ccount && LC.idx[lo] == j ? lo : -1;
                    };
                    const int pbs = slot_of(ib);
                    const int nT = T > 0 ? count_le(tw - T) : 0;                  // c too far from the witness
                    const int pw = slot_of(iw);                                   // c at the witness's point
                    anybad = nT - (pbs >= 0 && pbs < nT ? 1 : 0) > 0 || pw >= 0;
                    if (anybad) {
                        if (!has2) {
                            loose = true;
                        } else {
                            // a c that rules out both: too far from both, or at one's point and too far from
                            // the other
                            const int nT2 = T > 0 ? count_le(min(tw, t2) - T) : 0;
                            const int p2 = slot_of(i2);
                            loose = nT2 - (pbs >= 0 && pbs < nT2 ? 1 : 0) > 0 || (p2 >= 0 && p2 < nT) ||
                                    (pw >= 0 && T > 0 && t2 - tw >= T);
                        }
                    }
                }
                float thr = bv + gmax + 1e-6f * bv;
                if (anybad) thr = !loose && m2 < kInf ? fmaxf(thr, m2 + gmax + 1e-6f * m2) : kInf;
                // keep base <= thr, compacted in increasing a: positions from the pair's kept masks
                unsigned long long mk = 0;
                if (live) {
#pragma unroll 8
                    for (int k = k0; k < AH; ++k) {
                        const float bs = arow[NP * k + h];   // +inf for a past the list
                        if (bs < kInf && bs <= thr) mk |= 1ull << k;
                    }
                }
                unsigned long long pmk = 0;
                if constexpr (NP == 2) pmk = __shfl_xor_sync(0xffffffffu, (unsigned)mk, 1);
                const int kept = __popcll(mk) + __popcll(pmk);
                float *fbf = reinterpret_cast<float *>(sm.fb);
                for (unsigned long long m = mk; m; m &= m - 1) {
                    const int k = __ffsll((long long)m) - 1;
                    const int a = NP * k + h;
                    int pos = __popcll(mk & ((1ull << k) - 1));
                    if constexpr (NP == 2) pos += __popcll(pmk & ((h ? 2ull << k : 1ull << k) - 1));
                    const int at = fb_at<KM>(b, pos);
                    const float2 pa = LA.xy[a];
                    fbf[2 * at] = arow[a];
                    sm.fs[fs_at<KM>(b, pos)] = (uint8_t)(a | (pa.x == pb.x && pa.y == pb.y ? 0x80 : 0));
                    fbf[2 * at + 1] = wrap_pi(__fadd_rn(A1, direction(pb, pa)));   // p1 = A1 + theta(b->a)
                }
                // tiles in decreasing kept count, then increasing b (the lanes of a warp then loop over
                // similar numbers of a): b's first tile = sum of the tile counts of the b ranked before it
                const int nt_b = inb ? (ccount + CT - 1) / CT : 0;
                const int fnb = live ? kept : 0;
                const int key = nt_b > 0 ? ((fnb + 1) << 8) | (255 - b) : 0;
                if (h == 0) {
                    sm.fn[b] = (uint8_t)fnb;
                    sm.tcount[b] = (uint8_t)nt_b;
                    sm.pw[b] = (key << 5) | nt_b;
                }
            } else {
                // ---- phase 2 (concurrent): theta(a->c) for every a and the c with t'(c) <= t'(a)
                if (pf) {
                    pf_n = ccnt[i - 3];
                    pf_j = cidx[(int64_t)(i - 3) * K + pfi];
                    pf_u = cu[(int64_t)(i - 3) * K + pfi];
                }
                if (tid == P1 && i >= 3) sm.geo[(i - 1) & 1] = md.geo[i - 1];
                {
                    // two threads per c, interleaved a. A kept a of a cell (b, c) has t'(a) >= t'(b) >= t'(c), so
                    // only the rows from the first a with t'(a) >= t'(c) are read; entries of c past the list
                    // belong to cells whose theta(b->c) is +inf, so their value is never used either
                    const int q = tid - P1, c = q >> 1, h2 = q & 1;
                    if (c < nc) {
                        const int tc = LC.t[c], ic = LC.idx[c];
                        const float2 pc = LC.xy[c];
                        int lo = 0, hi = na;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (LA.t[mid] < tc) lo = mid + 1;
                            else hi = mid;
                        }
                        for (int a = lo + h2; a < na; a += 2) {
                            const int ta = LA.t[a];
                            float r = kInf;
                            if (!(T > 0 && ta - tc >= T) && LA.idx[a] != ic) r = direction(LA.xy[a], pc);   // theta(a->c)
                            sm.r[a * RS + c] = r;
                        }
                    }
                }
                pf_ok = pf && pfi < pf_n;
                if (pf_ok) {
                    pf_xy = sc.xy[pf_j];
                    pf_t = sc.t[pf_j];
                }
            }
            __syncthreads();

            // tile layout, by every thread (NT / KM per b): b's first tile = the tile count of the b ranked
            // before it (decreasing kept count, then increasing b)
            {
                constexpr int RP = NT / KM;
                static_assert(RP >= 1 && RP <= 32 && (RP & (RP - 1)) == 0, "threads per b in the ranking");
                const int b = tid / RP, part = tid % RP;
                const int wb = sm.pw[b], key = wb >> 5, nt_b = wb & 31;
                int before = 0, total = 0;
                for (int b2 = part; b2 < KM; b2 += RP) {
                    const int w = sm.pw[b2];
                    total += w & 31;
                    if ((w >> 5) > key) before += w & 31;
                }
#pragma unroll
                for (int off = 1; off < RP; off <<= 1) {
                    before += __shfl_xor_sync(0xffffffffu, before, off);
                    total += __shfl_xor_sync(0xffffffffu, total, off);
                }
                if (part == 0) sm.tbase[b] = (uint16_t)before;
                for (int t = part; t < nt_b; t += RP) sm.tile_b[before + t] = (uint8_t)b;
                if (tid == 0) sm.ntile = total;
            }

            // list A is not read from here on: its buffer receives list C of the next step
            if (pf) {
                LA.idx[pfi] = pf_ok ? pf_j : -1;
                LA.xy[pfi] = pf_xy;
                LA.t[pfi] = pf_t;
                LA.u[pfi] = pf_ok ? pf_u : kInf;
                if (pfi == 0) LA.n = pf_n;
            }
            if (i >= 3 && pfi >= K && pfi < KM) {
                LA.idx[pfi] = -1;
                LA.xy[pfi] = make_float2(0.f, 0.f);
                LA.t[pfi] = 0x3fffffff;
                LA.u[pfi] = kInf;
            }

            __syncthreads();   // the tile layout is complete

            // ---- phase 3: tiles (b, CT consecutive c)
            const int ntile = sm.ntile;
            uint8_t *bstep = ubeta + (int64_t)(i - 2) * K * K;
            // tiles in decreasing kept count, dealt to the threads back and forth (round r: thread t takes
            // tile r NT + t for even r, r NT + NT - 1 - t for odd r) so that per-thread sums even out
            for (int r0 = 0; r0 < ntile; r0 += NT) {
                const int tile = r0 + (((r0 / NT) & 1) ? NT - 1 - tid : tid);
                if (tile >= ntile) continue;
                const int b = sm.tile_b[tile];
                const int c0 = (tile - sm.tbase[b]) * CT;
                const float2 pb = LB.xy[b];
                const int tb = LB.t[b], ib = LB.idx[b];
                float q1[CT], best[CT];
                int arg[CT], tcq[CT];
#pragma unroll
                for (int q4 = 0; q4 < CT; q4 += 4) {   // the tile's cells of list C, four at a time
                    const int4 t4 = *reinterpret_cast<const int4 *>(&LC.t[c0 + q4]);
                    const int4 i4 = *reinterpret_cast<const int4 *>(&LC.idx[c0 + q4]);
                    const float4 xa = *reinterpret_cast<const float4 *>(&LC.xy[c0 + q4]);
                    const float4 xb = *reinterpret_cast<const float4 *>(&LC.xy[c0 + q4 + 2]);
                    const int tv[4] = {t4.x, t4.y, t4.z, t4.w}, iv[4] = {i4.x, i4.y, i4.z, i4.w};
                    const float2 xv[4] = {make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
                                          make_float2(xb.z, xb.w)};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int c = c0 + q4 + k;
                        const bool ok = c < nc && tv[k] <= tb && iv[k] != ib;
                        q1[q4 + k] = ok ? direction(pb, xv[k]) : kInf;   // theta(b->c)
                        tcq[q4 + k] = tv[k];
                        best[q4 + k] = kInf;
                        arg[q4 + k] = kNoSlot;
                    }
                }
                const int nf = sm.fn[b];
                // cells in pairs: packed FP32x2 arithmetic, same roundings as triple_cost
                static_assert(CT % 4 == 0, "tiles of a multiple of 4 cells");
                unsigned long long q1p[CT / 2];
#pragma unroll
                for (int q = 0; q < CT / 2; ++q) q1p[q] = pk2(q1[2 * q], q1[2 * q + 1]);
                const unsigned long long lamp = pk2(lam23, lam23);
#pragma unroll UR
                for (int k = 0; k < nf; ++k) {
                    const float2 e = sm.fb[fb_at<KM>(b, k)];
                    const int fa = sm.fs[fs_at<KM>(b, k)];
                    const int a = fa & 0x7f;
                    if constexpr (kCount) n_eval += CT;
                    const float p2 = __fadd_rn(e.y, (fa & 0x80) ? k2c : k2);
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
                // argmin bytes of the tile's cells, four at a time (c0 is a multiple of 4, and K, the row
                // stride, is a multiple of 4 whenever a tile reaches past c0 + 3: the packed store is used
                // only then)
                uint32_t packed[CT / 4];
#pragma unroll
                for (int q4 = 0; q4 < CT / 4; ++q4) packed[q4] = 0;
#pragma unroll
                for (int q = 0; q < CT; ++q) {
                    const int c = c0 + q;
                    float al = kInf;
                    int bt = kNoSlot;
                    if (best[q] < kInf) {
                        al = cell_alpha(best[q], lam2, dt_bc, tb, tcq[q]);
                        bt = arg[q];
                    }
                    if (c < nc) sm.alpha[c * AS + b] = al;
                    packed[q / 4] |= (uint32_t)bt << (8 * (q % 4));
                }
                const bool aligned = (K & 3) == 0;
#pragma unroll
                for (int q4 = 0; q4 < CT / 4; ++q4) {
                    const int c = c0 + 4 * q4;
                    if (aligned && c + 3 < K) {
                        *reinterpret_cast<uint32_t *>(bstep + b * K + c) = packed[q4];
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (c + q < nc) bstep[b * K + c + q] = (uint8_t)(packed[q4] >> (8 * q));
                    }
                }
            }
            // cells (b, c) beyond the tiled prefix are infeasible: the backtrack never reads their argmin (a
            // chain's cells are feasible) and the next step never reads their alpha (the pair (b, c) is
            // infeasible there); only the initial pair search of Eq. 13 reads every cell of the last step
            if (i == 2) {
                for (int b = warp; b < nb; b += NW) {
                    const int covered = sm.tcount[b] * CT;
                    for (int c = covered + lane; c < nc; c += 32) sm.alpha[c * AS + b] = kInf;
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
                if constexpr (kFused) backtrack_unit(un, md, sc, K, cidx, ubeta, r, energy_out, assign_out);
                else res[u] = r;
            }
            __syncthreads();
        }
    }
}

constexpr int kFusedPerSm = 3;   // CTAs per SM of the fused variant (its argmin scratch is per CTA)

struct FusedArgs {
    const int *n_dev = nullptr;
    int64_t beta_cta = 0;
    float *energy = nullptr;
    int32_t *assign = nullptr;
};

template <int KM, int NT, int CT, int NP, int UR, bool kCount, bool kFused>
cudaError_t launch_recurse_t(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                             Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                             uint8_t *beta, UnitResult *res, int *work_counter, unsigned long long *evaluated,
                             const FusedArgs &fa, cudaStream_t st)
{
    // three CTAs of 256 threads per SM: 3 x (shared memory + 1 KB reserved) <= 228 KB
    static_assert(KM != 64 || NT != 256 || 3 * (sizeof(Smem<KM, NT, NP>) + 1024) <= 228 * 1024,
                  "recursion shared memory exceeds the three-CTA budget");
    auto kern = recurse_kernel<KM, NT, CT, NP, UR, kCount, kFused>;
    const size_t smem = sizeof(Smem<KM, NT, NP>);
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
    if (kFused) {   // the per-CTA scratch was sized for sms * kFusedPerSm CTAs
        grid = std::min<int64_t>((int64_t)sms * kFusedPerSm, n_units);
    }
    kern<<<(unsigned)grid, NT, smem, st>>>(units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta, res,
                                           work_counter, evaluated, fa.n_dev, fa.beta_cta, fa.energy, fa.assign);
    prof_end(kProfRecurse, st);
    return cudaGetLastError();
}

template <bool kCount, bool kFused>
cudaError_t dispatch(int variant, const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                     Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt, uint8_t *beta,
                     UnitResult *res, int *work_counter, unsigned long long *evaluated, const FusedArgs &fa,
                     cudaStream_t st)
{
#define HGM_RECURSE(KM_, NT_, CT_, NP_, UR_)                                                                      \
    return launch_recurse_t<KM_, NT_, CT_, NP_, UR_, kCount, kFused>(units, n_units, models, scenes, p, cand_idx,  \
                                                                     cand_u, cand_cnt, beta, res, work_counter,   \
                                                                     evaluated, fa, st)
    if (p.K <= 32) {
        if (variant == 1) HGM_RECURSE(32, 128, 8, 2, 2);
        if (variant == 2) HGM_RECURSE(32, 128, 4, 2, 4);
        HGM_RECURSE(32, 128, 4, 2, 2);
    }
    if (variant == 1) HGM_RECURSE(64, 256, 8, 2, 2);
    if (variant == 2) HGM_RECURSE(64, 256, 4, 2, 4);
    HGM_RECURSE(64, 256, 4, 2, 2);
#undef HGM_RECURSE
}

int g_variant = 0;   // recursion variant: 0 = 4 c per tile, 1 = 8 c per tile, 2 = 4 c per tile, triple loop unrolled by 4

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

cudaError_t preload_recurse()
{
    cudaFuncAttributes a;
    const void *kerns[] = {(const void *)recurse_kernel<32, 128, 8, 2, 2, false, false>,
                           (const void *)recurse_kernel<32, 128, 4, 2, 4, false, false>,
                           (const void *)recurse_kernel<32, 128, 4, 2, 2, false, false>,
                           (const void *)recurse_kernel<64, 256, 8, 2, 2, false, false>,
                           (const void *)recurse_kernel<64, 256, 4, 2, 4, false, false>,
                           (const void *)recurse_kernel<64, 256, 4, 2, 2, false, false>};
    for (const void *k : kerns) {
        cudaError_t e = cudaFuncGetAttributes(&a, k);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
    return dispatch<false, false>(g_variant, units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta,
                                  res, work_counter, nullptr, FusedArgs{}, st);
}

int64_t recurse_fused_scratch(int K, int max_M)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return -1;
    const int64_t per = ((int64_t)std::max(max_M - 2, 1) * K * K + 255) / 256 * 256;
    return (int64_t)sms * kFusedPerSm * per;
}

cudaError_t launch_recurse_fused(const Unit *units, int64_t n_max, const int *n_dev, const ModelRec *models,
                                 const SceneRec *scenes, Params p, const int32_t *cand_idx, const float *cand_u,
                                 const int32_t *cand_cnt, uint8_t *scratch, int max_M, float *energy,
                                 int32_t *assign, int *work_counter, cudaStream_t st)
{
    if (n_max <= 0) return cudaSuccess;
    FusedArgs fa;
    fa.n_dev = n_dev;
    fa.beta_cta = ((int64_t)std::max(max_M - 2, 1) * p.K * p.K + 255) / 256 * 256;
    fa.energy = energy;
    fa.assign = assign;
    return dispatch<false, true>(0, units, n_max, models, scenes, p, cand_idx, cand_u, cand_cnt, scratch, nullptr,
                                 work_counter, nullptr, fa, st);
}

cudaError_t launch_recurse_count(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                                 uint8_t *beta, UnitResult *res, int *work_counter, unsigned long long *evaluated,
                                 cudaStream_t st)
{
    if (n_units <= 0) return cudaSuccess;
    return dispatch<true, false>(g_variant, units, n_units, models, scenes, p, cand_idx, cand_u, cand_cnt, beta,
                                 res, work_counter, evaluated, FusedArgs{}, st);
}

}  // namespace hgm
