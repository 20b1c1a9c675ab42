/*
 * hgm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the chain
 * hypergraph matching of Lombardi, Wolf, Celiktutan and Sankur, "Activity
 * recognition from videos with parallel hypergraph matching on GPUs"
 * (arXiv 1505.00581): the energy of Sec. 2 (Eqs. 1-6) simplified to a
 * second-order chain (Sec. 2.2, Eq. 9), its exact backward min-sum recursion
 * (Eq. 10) with initialisation (Eq. 11), argmin tables and backtracking
 * (Eq. 12) and the initial pair search (Eq. 13), under the causality and
 * temporal-closeness assumptions (Sec. 2.1, Eqs. 7-8). Two candidate
 * domains: per time offset with windowed, capped lists (the batched form),
 * and the whole-block problem of the paper itself, where every scene node is
 * a candidate of every model node (Sec. 2.2, Sec. 3).
 *
 * It is the parity reference for the CUDA library and shares no code with
 * it. Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it. Nothing here is tuned: every term is evaluated directly
 * from its definition, per triple, in double precision.
 *
 * Readings where the paper is silent or ambiguous (each also listed in the
 * design notes):
 *  R1 angles: a(i,j,k) is the signed angle at vertex j from edge j->i to edge
 *     j->k, computed as wrap(theta(j->k) - theta(j->i)) with
 *     theta(p->q) = atan2(qy-py, qx-px) on spatial coordinates only and
 *     atan2(0,0) = 0; wrap(x) = x - 2*pi*rint(x/(2*pi)). The circular
 *     difference of two angles is wrap(a - a').
 *  R2 roles: hyperedge (i,j,k) = (i, i-1, i-2); D^t = Delta(i,i-1) +
 *     Delta(i-1,i-2); lambda1 multiplies U, lambda2 multiplies D^t +
 *     lambda3 D^g (Eq. 1 with Eq. 3).
 *  R3 feasibility of (z_i, z_{i-1}, z_{i-2}) = (a,b,c): t'(c) <= t'(b) <=
 *     t'(a), t'(a) - t'(c) < T (T <= 0 means no closeness limit), and a, b, c
 *     pairwise distinct scene points.
 *  R4 candidates of model point i at offset o: scene points whose frame lies
 *     in [t_i+o-w, t_i+o+w]; if more than K, the K with smallest U (ties to
 *     the lower scene index); listed in ascending scene index. Keeping K is
 *     an integer decision taken on floating point, so it is taken on an FP32
 *     key that both sides compute identically (or_rank_key): d_k = a_k - b_k
 *     in FP32, s = fma(d_k, d_k, s) for k = 0..F-1 in order, then
 *     lambda1 * sqrt(s), each step rounded to nearest FP32. The energy itself
 *     uses the FP64 U.
 *  R6 ties: the argmin over z_i keeps the lowest candidate slot; the initial
 *     pair keeps the lexicographically lowest (slot of z_1, then of z_2).
 *  R5 dummy assignment (Eq. 2), off unless or_ctx_set_dummy gives W^d >= 0:
 *     every list gets one extra slot eps (after the real candidates, so ties
 *     prefer a real point) with U(eps) = W^d (times lambda1, as every U here).
 *     A term that involves eps vanishes: Delta(i,j) is 0 if z_i or z_j is eps,
 *     D^g is 0 if any point of the triangle is eps. A triple holding eps is
 *     feasible iff its real points, in chain order, are distinct, ordered in
 *     time and span less than T frames. eps is the scene index OR_EPS (-2).
 *
 * Scene and model arrays given to this file are already stably sorted by
 * frame (the Python wrapper does that); indices below are sorted indices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

typedef struct {
    int M, S, F, nframes;
    const double *mx, *my, *mf; const int *mt;   /* model, sorted by t */
    const double *sx, *sy, *sf; const int *st;   /* scene, sorted by t */
    double lambda1, lambda2, lambda3;
    int T, window, K;
    int *frame_start;                            /* minnode table, nframes+1 */
    double wd;                                   /* dummy cost W^d; < 0: no dummy assignment */
} or_ctx;

#define OR_EPS (-2)

/* ---- construction ---------------------------------------------------- */

or_ctx *or_ctx_create(int M, const double *mx, const double *my, const int *mt, const double *mf,
                      int S, const double *sx, const double *sy, const int *st, const double *sf,
                      int F, int nframes, double lambda1, double lambda2, double lambda3,
                      int T, int window, int K)
{
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!c) return NULL;
    c->M = M; c->S = S; c->F = F; c->nframes = nframes;
    c->mx = mx; c->my = my; c->mt = mt; c->mf = mf;
    c->sx = sx; c->sy = sy; c->st = st; c->sf = sf;
    c->lambda1 = lambda1; c->lambda2 = lambda2; c->lambda3 = lambda3;
    c->T = T; c->window = window; c->K = K;
    c->wd = -1.0;
    /* minnode(f) (Sec. 3.4): first sorted scene index whose frame is >= f. */
    c->frame_start = (int *)malloc(sizeof(int) * (size_t)(nframes + 1));
    if (!c->frame_start) { free(c); return NULL; }
    int n = 0;
    for (int f = 0; f <= nframes; ++f) {
        while (n < S && st[n] < f) ++n;
        c->frame_start[f] = n;
    }
    return c;
}

/* Enables the dummy assignment with cost W^d (wd >= 0) or disables it (wd < 0). */
void or_ctx_set_dummy(or_ctx *c, double wd)
{
    c->wd = wd;
}

void or_ctx_destroy(or_ctx *c)
{
    if (!c) return;
    free(c->frame_start);
    free(c);
}

/* ---- energy terms ---------------------------------------------------- */

/* U of Eq. 2 (non-dummy branch), with lambda1 of Eq. 1 absorbed as in Eq. 9. */
double or_unary(const or_ctx *c, int i, int j)
{
    double s = 0.0;
    for (int k = 0; k < c->F; ++k) {
        double d = c->mf[(size_t)i * c->F + k] - c->sf[(size_t)j * c->F + k];
        s += d * d;
    }
    return c->lambda1 * sqrt(s);
}

/* FP32 ranking key of reading R4 (same value as the FP32 U of the CUDA
 * path by construction: fixed component order, fused multiply-add, IEEE
 * square root). The descriptors are FP32 values widened to double, so the
 * casts below are exact. */
float or_rank_key(const or_ctx *c, int i, int j)
{
    float s = 0.0f;
    for (int k = 0; k < c->F; ++k) {
        float d = (float)c->mf[(size_t)i * c->F + k] - (float)c->sf[(size_t)j * c->F + k];
        s = fmaf(d, d, s);
    }
    return (float)c->lambda1 * sqrtf(s);
}

static double wrap_angle(double x)
{
    return x - 2.0 * OR_PI * rint(x / (2.0 * OR_PI));
}

static double direction(double px, double py, double qx, double qy)
{
    return atan2(qy - py, qx - px);
}

/* Signed angle at vertex v from edge v->p to edge v->q (reading R1). */
static double angle_at(double vx, double vy, double px, double py, double qx, double qy)
{
    return wrap_angle(direction(vx, vy, qx, qy) - direction(vx, vy, px, py));
}

/* U of model point i assigned to z (Eq. 2 with both branches, lambda1 absorbed). */
static double unary_z(const or_ctx *c, int i, int z)
{
    return z == OR_EPS ? c->lambda1 * c->wd : or_unary(c, i, z);
}

/* Delta of Eq. 5 for model pair (i,j) assigned to scene pair (zi,zj); 0 if either is eps. */
static double delta_t(const or_ctx *c, int i, int j, int zi, int zj)
{
    if (zi == OR_EPS || zj == OR_EPS) return 0.0;
    return fabs((double)(c->mt[i] - c->mt[j]) - (double)(c->st[zi] - c->st[zj]));
}

/* D^g of Eq. 6 for model triangle (i, i-1, i-2) and scene triangle (a,b,c). */
double or_geo(const or_ctx *c, int i, int a, int b, int cc)
{
    if (a == OR_EPS || b == OR_EPS || cc == OR_EPS) return 0.0;
    /* first row: angle at the middle vertex j = i-1 of triangle (i,j,k) */
    double am1 = angle_at(c->mx[i - 1], c->my[i - 1], c->mx[i], c->my[i], c->mx[i - 2], c->my[i - 2]);
    double as1 = angle_at(c->sx[b], c->sy[b], c->sx[a], c->sy[a], c->sx[cc], c->sy[cc]);
    /* second row: a(j,i,k), the angle at vertex i of triangle (j,i,k) */
    double am2 = angle_at(c->mx[i], c->my[i], c->mx[i - 1], c->my[i - 1], c->mx[i - 2], c->my[i - 2]);
    double as2 = angle_at(c->sx[a], c->sy[a], c->sx[b], c->sy[b], c->sx[cc], c->sy[cc]);
    double d1 = wrap_angle(am1 - as1);
    double d2 = wrap_angle(am2 - as2);
    return sqrt(d1 * d1 + d2 * d2);
}

/* D of Eqs. 3-4 with lambda2 absorbed (Eq. 9): model triple (i,i-1,i-2) -> (a,b,c). */
double or_triple(const or_ctx *c, int i, int a, int b, int cc)
{
    double dt = delta_t(c, i, i - 1, a, b) + delta_t(c, i - 1, i - 2, b, cc);
    return c->lambda2 * (dt + c->lambda3 * or_geo(c, i, a, b, cc));
}

/* Causality (Eq. 7), closeness (Eq. 8) and distinctness, reading R3. */
int or_feasible(const or_ctx *c, int a, int b, int cc)
{
    if (a == OR_EPS || b == OR_EPS || cc == OR_EPS) {
        /* the real points of the triple, newest first (chain order a, b, c) */
        int p[3], n = 0;
        if (a != OR_EPS) p[n++] = a;
        if (b != OR_EPS) p[n++] = b;
        if (cc != OR_EPS) p[n++] = cc;
        for (int k = 0; k + 1 < n; ++k)
            for (int l = k + 1; l < n; ++l)
                if (p[k] == p[l]) return 0;
        for (int k = 0; k + 1 < n; ++k)
            if (!(c->st[p[k + 1]] <= c->st[p[k]])) return 0;
        if (n >= 2 && c->T > 0 && !(c->st[p[0]] - c->st[p[n - 1]] < c->T)) return 0;
        return 1;
    }
    if (a == b || b == cc || a == cc) return 0;
    if (!(c->st[cc] <= c->st[b] && c->st[b] <= c->st[a])) return 0;
    if (c->T > 0 && !(c->st[a] - c->st[cc] < c->T)) return 0;
    return 1;
}

/* E(z) of Eq. 9 for a full assignment z[0..M-1] (sorted scene indices);
 * +inf if some triple is infeasible. */
double or_energy(const or_ctx *c, const int *z)
{
    double e = 0.0;
    for (int i = 0; i < c->M; ++i) e += unary_z(c, i, z[i]);
    for (int i = 2; i < c->M; ++i) {
        if (!or_feasible(c, z[i], z[i - 1], z[i - 2])) return INFINITY;
        e += or_triple(c, i, z[i], z[i - 1], z[i - 2]);
    }
    return e;
}

/* ---- candidate lists (reading R4) ------------------------------------ */

typedef struct { float key; double u; int j; } cand_t;

static int cmp_u_then_index(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->j > b->j) - (a->j < b->j);
}

static int cmp_index(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    return (a->j > b->j) - (a->j < b->j);
}

/* Candidates of model point i at offset o. Writes up to K sorted scene
 * indices to idx and their U to u; returns the count. */
int or_candidates(const or_ctx *c, int i, int o, int *idx, double *u)
{
    int lo = c->mt[i] + o - c->window, hi = c->mt[i] + o + c->window;
    if (lo < 0) lo = 0;
    if (hi > c->nframes - 1) hi = c->nframes - 1;
    if (lo > hi) return 0;
    int j0 = c->frame_start[lo], j1 = c->frame_start[hi + 1];
    int n = j1 - j0;
    if (n <= 0) return 0;
    cand_t *all = (cand_t *)malloc(sizeof(cand_t) * (size_t)n);
    for (int k = 0; k < n; ++k) {
        all[k].j = j0 + k;
        all[k].key = or_rank_key(c, i, j0 + k);
        all[k].u = or_unary(c, i, j0 + k);
    }
    qsort(all, (size_t)n, sizeof(cand_t), cmp_u_then_index);
    int keep = n < c->K ? n : c->K;
    qsort(all, (size_t)keep, sizeof(cand_t), cmp_index);
    for (int k = 0; k < keep; ++k) { idx[k] = all[k].j; u[k] = all[k].u; }
    free(all);
    return keep;
}

/* Whole-block candidates (the paper's own formulation, Sec. 2.2 and Sec. 3:
 * z_i ranges over every scene node, restricted only by the constraints of
 * Eqs. 7-8): C_i = all S scene points in ascending index, for every i.
 * Writes S indices to idx and the U of model point i to u; returns S. */
int or_block_candidates(const or_ctx *c, int i, int *idx, double *u)
{
    for (int j = 0; j < c->S; ++j) { idx[j] = j; u[j] = or_unary(c, i, j); }
    return c->S;
}

/* ---- exact recursion (Eqs. 10-13) ------------------------------------ */

/* Solves the chain problem over the given candidate lists: list i holds cnt[i]
 * sorted scene indices at cand[i*Kc ..] with their U at cu[i*Kc ..]. Outputs
 * the minimal energy (or +inf), the assignment z[0..M-1] as sorted scene
 * indices (-1 when infeasible), and optionally the number of feasible
 * (z_i, z_{i-1}, z_{i-2}) triples visited. Returns 0, or -1 on allocation
 * failure. */
static int solve_lists(const or_ctx *c, int Kc, const int *cand, const double *cu, const int *cnt,
                       double *energy, int *z, int64_t *n_triples)
{
    const int M = c->M, K = Kc;
    double *alpha_next = (double *)malloc(sizeof(double) * (size_t)K * K);
    double *alpha_cur = (double *)malloc(sizeof(double) * (size_t)K * K);
    int *beta = (int *)malloc(sizeof(int) * (size_t)M * K * K);
    if (!alpha_next || !alpha_cur || !beta) {
        free(alpha_next); free(alpha_cur); free(beta);
        return -1;
    }
    int64_t triples = 0;
    int feasible = 1;
    for (int i = 0; i < M; ++i)
        if (cnt[i] == 0) feasible = 0;
    for (int i = 0; i < M; ++i) z[i] = -1;
    *energy = INFINITY;
    if (feasible) {
        /* alpha_{M+1} == 0: alpha_next[ja*K + jb] holds alpha_{i+1}(z_i = slot ja, z_{i-1} = slot jb). */
        for (size_t k = 0; k < (size_t)K * K; ++k) alpha_next[k] = 0.0;
        for (int i = M - 1; i >= 2; --i) {          /* 0-based i is the paper's i+1 */
            const int *Ci = cand + (size_t)i * K, *Cb = cand + (size_t)(i - 1) * K, *Cc = cand + (size_t)(i - 2) * K;
            const double *Ui = cu + (size_t)i * K;
            for (int jb = 0; jb < cnt[i - 1]; ++jb) {
                for (int jc = 0; jc < cnt[i - 2]; ++jc) {
                    double best = INFINITY;
                    int arg = -1;
                    const int b = Cb[jb], cc = Cc[jc];
                    /* R3 between two real points b and c alone (distinct, t'(c) <= t'(b), t'(b) - t'(c) < T)
                     * is implied by the feasibility of any (a, b, c): when it fails, no a is tried */
                    const int bc_ok = b == OR_EPS || cc == OR_EPS ||
                                      (b != cc && c->st[cc] <= c->st[b] && !(c->T > 0 && c->st[b] - c->st[cc] >= c->T));
                    for (int ja = 0; bc_ok && ja < cnt[i]; ++ja) {
                        int a = Ci[ja];
                        if (!or_feasible(c, a, b, cc)) continue;
                        ++triples;
                        double v = Ui[ja] + or_triple(c, i, a, b, cc) + alpha_next[(size_t)ja * K + jb];
                        if (v < best) { best = v; arg = ja; }
                    }
                    alpha_cur[(size_t)jb * K + jc] = best;
                    beta[((size_t)i * K + jb) * K + jc] = arg;
                }
            }
            double *tmp = alpha_next; alpha_next = alpha_cur; alpha_cur = tmp;
        }
        /* alpha_next now holds alpha_3(z_2 = slot jb, z_1 = slot jc). Eq. 13: */
        double best = INFINITY;
        int b1 = -1, b2 = -1;
        for (int j1 = 0; j1 < cnt[0]; ++j1) {
            for (int j2 = 0; j2 < cnt[1]; ++j2) {
                double v = cu[j1] + cu[K + j2] + alpha_next[(size_t)j2 * K + j1];
                if (v < best) { best = v; b1 = j1; b2 = j2; }
            }
        }
        if (b1 >= 0 && isfinite(best)) {
            /* Eq. 12: z_i = beta_i(z_{i-1}, z_{i-2}) */
            int *slot = (int *)malloc(sizeof(int) * (size_t)M);
            if (!slot) {
                free(alpha_next); free(alpha_cur); free(beta);
                return -1;
            }
            slot[0] = b1; slot[1] = b2;
            for (int i = 2; i < M; ++i) slot[i] = beta[((size_t)i * K + slot[i - 1]) * K + slot[i - 2]];
            for (int i = 0; i < M; ++i) z[i] = cand[(size_t)i * K + slot[i]];
            free(slot);
            *energy = best;
        }
    }
    if (n_triples) *n_triples = triples;
    free(alpha_next); free(alpha_cur); free(beta);
    return 0;
}

/* Builds the lists of offset o (block != 0: the whole-block lists) with
 * capacity *Kc; the caller frees cand, cu and cnt. */
static int build_lists(const or_ctx *c, int block, int o, int **cand, double **cu, int **cnt, int *Kc)
{
    const int dummy = c->wd >= 0.0;
    const int M = c->M, K = (block ? (c->S > 0 ? c->S : 1) : c->K) + dummy;
    *Kc = K;
    *cand = (int *)malloc(sizeof(int) * (size_t)M * K);
    *cu = (double *)malloc(sizeof(double) * (size_t)M * K);
    *cnt = (int *)malloc(sizeof(int) * (size_t)M);
    if (!*cand || !*cu || !*cnt) {
        free(*cand); free(*cu); free(*cnt);
        return -1;
    }
    for (int i = 0; i < M; ++i) {
        int n = block ? or_block_candidates(c, i, *cand + (size_t)i * K, *cu + (size_t)i * K)
                      : or_candidates(c, i, o, *cand + (size_t)i * K, *cu + (size_t)i * K);
        if (dummy) {   /* eps after the real candidates (R5) */
            (*cand)[(size_t)i * K + n] = OR_EPS;
            (*cu)[(size_t)i * K + n] = unary_z(c, i, OR_EPS);
            ++n;
        }
        (*cnt)[i] = n;
    }
    return 0;
}

/* Solves one offset (windowed, capped lists). See solve_lists for outputs. */
int or_match_offset(const or_ctx *c, int o, double *energy, int *z, int64_t *n_triples)
{
    int *cand, *cnt, Kc;
    double *cu;
    if (build_lists(c, 0, o, &cand, &cu, &cnt, &Kc)) return -1;
    int rc = solve_lists(c, Kc, cand, cu, cnt, energy, z, n_triples);
    free(cand); free(cu); free(cnt);
    return rc;
}

/* Solves the whole-block problem (every scene point a candidate of every
 * model point, no offset). See solve_lists for outputs. */
int or_match_block(const or_ctx *c, double *energy, int *z, int64_t *n_triples)
{
    int *cand, *cnt, Kc;
    double *cu;
    if (build_lists(c, 1, 0, &cand, &cu, &cnt, &Kc)) return -1;
    int rc = solve_lists(c, Kc, cand, cu, cnt, energy, z, n_triples);
    free(cand); free(cu); free(cnt);
    return rc;
}

/* Runs or_match_offset over offsets[0..n-1]; energy[n], z[n*M]. */
int or_match_offsets(const or_ctx *c, const int *offsets, int n, double *energy, int *z, int64_t *n_triples)
{
    for (int k = 0; k < n; ++k) {
        int rc = or_match_offset(c, offsets[k], energy + k, z + (size_t)k * c->M, n_triples ? n_triples + k : NULL);
        if (rc) return rc;
    }
    return 0;
}

/* ---- brute force ----------------------------------------------------- */

/* Enumerates every z with z_i in C_i(o) and returns min E(z) (Eq. 9) and the
 * first minimiser in lexicographic slot order. n_ties receives the number of
 * assignments whose energy is within tol of the minimum. Intended for tiny
 * inputs only (product of list sizes up to ~1e6). Returns -1 if the product
 * exceeds max_assignments. */
static int bruteforce_lists(const or_ctx *c, int block, int o, double tol, int64_t max_assignments,
                            double *energy, int *z, int64_t *n_ties)
{
    const int M = c->M;
    int *cand, *cnt, K;
    double *cu;
    if (build_lists(c, block, o, &cand, &cu, &cnt, &K)) return -1;
    int *slot = (int *)calloc((size_t)M, sizeof(int));
    int *zz = (int *)malloc(sizeof(int) * (size_t)M);
    double prod = 1.0;
    for (int i = 0; i < M; ++i) prod *= (double)cnt[i];
    for (int i = 0; i < M; ++i) z[i] = -1;
    *energy = INFINITY;
    *n_ties = 0;
    if (prod > (double)max_assignments) {
        free(cand); free(cu); free(cnt); free(slot); free(zz);
        return -1;
    }
    if (prod == 0.0) {
        free(cand); free(cu); free(cnt); free(slot); free(zz);
        return 0;
    }
    /* pass 1: minimum and first minimiser; pass 2: count near-ties */
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < M; ++i) slot[i] = 0;
        for (;;) {
            for (int i = 0; i < M; ++i) zz[i] = cand[(size_t)i * K + slot[i]];
            double e = or_energy(c, zz);
            if (pass == 0) {
                if (e < *energy) { *energy = e; memcpy(z, zz, sizeof(int) * (size_t)M); }
            } else if (isfinite(*energy) && e <= *energy + tol) {
                ++*n_ties;
            }
            int i = M - 1;
            while (i >= 0) {
                if (++slot[i] < cnt[i]) break;
                slot[i] = 0;
                --i;
            }
            if (i < 0) break;
        }
    }
    if (!isfinite(*energy)) for (int i = 0; i < M; ++i) z[i] = -1;
    free(cand); free(cu); free(cnt); free(slot); free(zz);
    return 0;
}

int or_bruteforce(const or_ctx *c, int o, double tol, int64_t max_assignments,
                  double *energy, int *z, int64_t *n_ties)
{
    return bruteforce_lists(c, 0, o, tol, max_assignments, energy, z, n_ties);
}

/* Brute force of the whole-block problem (every scene point a candidate). */
int or_bruteforce_block(const or_ctx *c, double tol, int64_t max_assignments,
                        double *energy, int *z, int64_t *n_ties)
{
    return bruteforce_lists(c, 1, 0, tol, max_assignments, energy, z, n_ties);
}
