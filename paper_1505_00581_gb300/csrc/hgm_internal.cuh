// hgm_internal.cuh -- shared declarations of libhgm's host runtime and kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "hgm.h"

namespace hgm {

constexpr int kMaxK = 64;          // candidate cap supported by the kernels
constexpr int kNoSlot = 255;       // beta entry of a cell without a feasible z_i
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

// Device-resident model (points sorted stably by frame).
struct ModelDev {
    int32_t M, F;
    float2 *xy;          // [M]
    int32_t *t;          // [M]
    float *f;            // [M*F]
    int32_t *perm;       // [M] caller index of sorted point k
    float4 *geo;         // [M] per chain step i >= 2: (A1, k2, t_i - t_{i-1}, t_{i-1} - t_{i-2}) (ints as bits)
};

// Device-resident scene (points sorted stably by frame) with its minnode table.
struct SceneDev {
    int32_t S, F, n_frames;
    float2 *xy;          // [S]
    int32_t *t;          // [S]
    float *f;            // [S*F]
    int32_t *frame_start;  // [n_frames+1], minnode of Sec. 3.4
    int32_t *perm;       // [S] caller index of sorted point k
};

// Per-model record the kernels read (device array indexed by model slot).
struct ModelRec {
    const float2 *xy;
    const int32_t *t;
    const int32_t *perm;
    int32_t M;
    int32_t urow;        // first row of this model in the unary table
    const float *f;      // sorted descriptors, row stride Params::F (used to re-score in FP32)
    const float4 *geo;   // per-step model constants of the recursion (ModelDev::geo)
};

// Per-scene record the kernels read.
struct SceneRec {
    const float2 *xy;
    const int32_t *t;
    const int32_t *frame_start;
    const int32_t *perm;
    const float *U;      // unary table block of this scene: [R x upitch]
    int64_t upitch;      // row pitch of U in floats (>= S)
    int32_t S, n_frames;
    const float *f;      // sorted descriptors, row stride Params::F
    const __nv_bfloat16 *pq;   // proposal network: W1b f'_j + position terms per point of the block, BF16
                               // [.. x 128] (pruned mode only)
    int64_t ucol0;       // first sorted scene point of the U / pq blocks (a segment of the scene)
};

// One matching problem: a (model, scene, offset) triple.
struct Unit {
    int32_t model, scene, offset, pad;
    int64_t cand;        // base of this unit's candidate lists (entries), M*K
    int64_t beta;        // base of this unit's argmin tables (bytes), (M-2)*K*K
    int64_t out_e;       // index into the energy output
    int64_t out_a;       // index into the assignment output
};

// Result of the recursion for one unit, consumed by the backtrack kernel.
struct UnitResult {
    float energy;
    int32_t z1, z2;      // slots of z_1 and z_2 in C_1, C_2 (-1 if infeasible)
    int32_t pad;
};

struct Params {
    float lambda1, lambda2, lambda3;
    int32_t T, window, K;
    int32_t F = 0;       // descriptor row stride (padded width)
    int32_t rescore = 0; // 0, or: recompute the U of the `rescore` smallest candidates per list in FP32
    float dummy = -1.0f; // W^d of the dummy assignment (k_dummy.cu), < 0: none
    int32_t max_window = 1 << 30;   // scene points of a typical candidate window of the call (host estimate from
                                    // the scenes' mean density; longer windows are still selected, from memory)
};

constexpr int kRescore = 8;   // candidates per list re-scored in FP32 by the BF16 precision mode

enum ProfKernel { kProfUnary = 0, kProfSelect = 1, kProfRecurse = 2, kProfBacktrack = 3, kProfPrune = 4, kProfCount = 5 };

// Proposal network operands for the pruning kernel (device pointers into the weights).
struct PropInfer {
    const __nv_bfloat16 *Pb;   // [R x 128]: W1a f_i + b1 - W1c (x_i, y_i) / 100 per model row, rounded to BF16
    const float *W2, *b2, *w3, *b3;
    const float *w1c;    // W1 columns 2F..2F+2 (row stride dp)
    int dp;
    float inv_window;    // 1 / max(w, 1)
    int keep;            // candidates kept per list
    int rescore;         // 1: kept candidates' U recomputed in FP32 (precision mode)
};
// Scores every candidate (scores [n_lists x K] scratch) and keeps the pi.keep best per list.
// Per-step model constants of the recursion: geo[i] = (A1, k2, dt_ab, dt_bc) for i >= 2 (zero for i < 2),
// A1 = signed angle at i-1 (->i to ->i-2), k2 = wrap(A2 - A1 + pi) with A2 the angle at i (->i-1 to ->i-2).
cudaError_t launch_model_geo(const float2 *xy, const int32_t *t, int M, float4 *geo, cudaStream_t st);
// rows[r][h] += sign * (W1c[h][0] x_r + W1c[h][1] y_r) / 100 (the first layer's position terms), r < n;
// with out_bf16 non-null the sums go there as BF16 and rows is left unchanged.
cudaError_t launch_prop_fold_xy(float *rows, int64_t n, const float *xy, const float *w1c, int dp, float sign,
                                void *out_bf16, cudaStream_t st);
// The proposal network's logit of every candidate of every list (scores [n_lists x K], -inf for empty slots).
cudaError_t launch_prop_score(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                              Params p, const PropInfer &pi, const int32_t *cand_idx, const int32_t *cand_cnt,
                              float *scores, int *status, cudaStream_t st);
cudaError_t launch_prop_prune(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                              Params p, const PropInfer &pi, const int32_t *cand_idx, const float *cand_u,
                              const int32_t *cand_cnt, float *scores, int32_t *out_idx, float *out_u,
                              int32_t *out_cnt, int *status, cudaStream_t st);
cudaError_t launch_derive_units(const Unit *in, int64_t n, int K, int keep, Unit *out, cudaStream_t st);
// Precision mode: FP32 unary cost of every candidate of the fallback units' full lists (count on the device).
cudaError_t launch_rescore_units(const Unit *units, int64_t n_max, const int *n_dev, const ModelRec *models,
                                 const SceneRec *scenes, Params p, const int32_t *cand_idx, const int32_t *cand_cnt,
                                 float *cand_u, cudaStream_t st);
cudaError_t launch_collect_infeasible(const UnitResult *res, const Unit *units, int64_t n, Unit *list, int *count,
                                      unsigned long long *total, cudaStream_t st);

// ---- kernel launchers (each checks its own launch error) --------------------
cudaError_t launch_unary(const float *A, int R, const float *B, int S, int F, float lambda1, float *U,
                         int ldu, cudaStream_t st);
// k_rowdot.cu: BF16 tensor-core products.
cudaError_t launch_sqnorm_bf16(const float *X, int64_t n, int ld, int F, float *out, cudaStream_t st);
// scratch: device memory of at least unary_bf16_scratch_bytes(R, S, F) for the BF16 copies of the operands
// the TMA-staged kernel reads (with less, or F > 256, the operands are staged by the threads instead).
size_t unary_bf16_scratch_bytes(int R, int64_t S, int F);
cudaError_t launch_unary_bf16(const float *model, int R, const float *scene, int S, int F, int ld,
                              const float *mnorm, const float *snorm, float lambda1, float *U, int64_t ldu,
                              int *status, void *scratch, size_t scratch_bytes, cudaStream_t st);
cudaError_t launch_rowdot_plain(const float *X, int64_t nrows, int ldx, const float *W, int ncols, int ldw, int F,
                                const float *bias, float *Y, int64_t ldy, int *status, cudaStream_t st);
cudaError_t launch_select(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                          Params p, int max_M, int32_t *cand_idx, float *cand_u, int32_t *cand_cnt,
                          cudaStream_t st);
cudaError_t launch_recurse(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                           Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                           uint8_t *beta, UnitResult *res, int *work_counter, cudaStream_t st);
// k_recurse_small.cu: warp-per-unit recursion for lists of at most 16 candidates.
cudaError_t launch_recurse_small(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                                 uint8_t *beta, UnitResult *res, cudaStream_t st);
// Tile variant of the recursion kernel used by launch_recurse (autotuned): 0..count-1.
int recurse_variant_count();
void set_recurse_variant(int v);
int get_recurse_variant();
// Same as launch_recurse, additionally adding the number of (a, b, c) evaluations of
// the triple loop to *evaluated (work accounting; not used on the timed path).
// Fused recursion + backtrack for the exact fallback of the pruned form: the unit count is read from n_dev
// (at most n_max), argmin tables live in per-CTA scratch of recurse_fused_scratch(K, max_M) bytes, and
// energies / assignments are written directly. No host synchronisation.
int64_t recurse_fused_scratch(int K, int max_M);
cudaError_t launch_recurse_fused(const Unit *units, int64_t n_max, const int *n_dev, const ModelRec *models,
                                 const SceneRec *scenes, Params p, const int32_t *cand_idx, const float *cand_u,
                                 const int32_t *cand_cnt, uint8_t *scratch, int max_M, float *energy,
                                 int32_t *assign, int *work_counter, cudaStream_t st);
cudaError_t launch_recurse_count(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, const int32_t *cand_idx, const float *cand_u, const int32_t *cand_cnt,
                                 uint8_t *beta, UnitResult *res, int *work_counter, unsigned long long *evaluated,
                                 cudaStream_t st);
cudaError_t launch_backtrack(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                             Params p, const int32_t *cand_idx, const uint8_t *beta, const UnitResult *res,
                             float *energy, int32_t *assign, cudaStream_t st);
cudaError_t launch_count(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                         Params p, const int32_t *cand_idx, const int32_t *cand_cnt, int64_t *triples,
                         cudaStream_t st);

// Load the device code of a kernel family now (the runtime otherwise loads code at first use), so that a later
// call allocates nothing for it: the kernels hgm_match_noalloc launches.
cudaError_t preload_unary();
cudaError_t preload_select();
cudaError_t preload_recurse();
cudaError_t preload_recurse_small();
cudaError_t preload_backtrack();

// Profiling hooks (api.cu).
// k_block.cu: the whole-block problem (every scene point a candidate, no offsets).
struct BlockGeo {            // band tables of one scene (see k_block.cu)
    const int32_t *lo;       // [S] first point of b's band
    const int64_t *cs;       // [S+1] first cell of b's band
    const int32_t *cellb;    // [cells] owner b of each cell
    const float *dirf;       // [cells] theta(b->c)
    const float *dirb;       // [cells] theta(c->b)
    int64_t cells;
};
struct BlockUnit {
    int32_t model, scene;
    int64_t beta;            // first argmin entry (uint16) of this unit: (M-2) x cells
    int64_t out_e, out_a;    // energy index, first assignment element
};
cudaError_t launch_block_geo(const float2 *xy, int S, const int32_t *lo, const int64_t *cs, int64_t cells,
                             int32_t *cellb, float *dirf, float *dirb, cudaStream_t st);
int64_t block_smem_cells();   // largest band table (cells) whose two copies fit one CTA's shared memory
// scratch == nullptr: tables in shared memory (max_cells <= block_smem_cells()); else per-CTA global scratch
// of 2 x max_cells floats for grid_global CTAs.
cudaError_t launch_block_recurse(const BlockUnit *units, int n_units, const ModelRec *models, const SceneRec *scenes,
                                 const BlockGeo *geos, Params p, int64_t max_cells, uint16_t *beta, float *scratch,
                                 int grid_global, float *energy, int32_t *assign, cudaStream_t st);

// k_dummy.cu: the recursion with the dummy assignment eps (fused backtrack; per-CTA argmin scratch).
// evaluated != NULL runs the accounting variant, which adds its evaluated triples to *evaluated.
int dummy_grid();
int64_t dummy_scratch_bytes(int K, int max_M, int grid);
cudaError_t launch_recurse_dummy(const Unit *units, int64_t n_units, const ModelRec *models, const SceneRec *scenes,
                                 Params p, float wd, const int32_t *cand_idx, const float *cand_u,
                                 const int32_t *cand_cnt, uint8_t *scratch, int max_M, int grid, float *energy,
                                 int32_t *assign, unsigned long long *evaluated, cudaStream_t st);

void prof_begin(int kernel, cudaStream_t st);
void prof_end(int kernel, cudaStream_t st);

constexpr uint32_t kModelMagic = 0x4d4f444cu;   // "MODL"
constexpr uint32_t kSceneMagic = 0x53434e45u;   // "SCNE"
constexpr uint32_t kPlanMagic = 0x504c414eu;    // "PLAN"

}  // namespace hgm

// Handle layouts (opaque to callers of include/hgm.h).
struct hgm_model {
    uint32_t magic;
    hgm::ModelDev d;
    int32_t F_user;
    std::vector<int32_t> t_sorted;   // host copy of sorted frames
    std::vector<int32_t> perm;       // host copy of the order
    // frames that anchor the offset range o = -span_t1 .. F_s-1-span_tM: the model's own first and last
    // frames, or for a chain of a multi-point model the whole model's (so that every chain shares its range)
    int32_t span_t1 = 0, span_tM = 0;
    // independent-chains split (built on first use for chain_n chains; released with the model)
    mutable int32_t chain_n = 0;
    mutable std::vector<hgm_model *> chains;        // the chains with >= 3 points, in chain order
    mutable std::vector<int32_t> chain_map;         // concatenated chain points -> caller index in this model
};

struct hgm_scene {
    uint32_t magic;
    hgm::SceneDev d;
    int32_t F_user;
    std::vector<int32_t> perm;
    std::vector<int32_t> fs_host;    // host copy of the minnode table (segment planning)
};

namespace hgm {
// api.cu: sets the thread's hgm_last_error() message and returns s.
hgm_status set_error(hgm_status s, const char *msg);
bool valid_model(const hgm_model *m);
bool valid_scene(const hgm_scene *s);
// api.cu: the parameter check shared by the matching entry points (HGM_EINVAL / HGM_EUNSUPPORTED + message).
hgm_status check_match_params(const hgm_params *p);
// api.cu: the points 2w+1 consecutive frames of the scene hold on average (a typical candidate window).
int32_t typical_window_points(const hgm_scene *s, int window);
// noalloc.cu: looks up (once per device) the device address of the fixed scratch of hgm_match_noalloc on the
// current device, which makes the runtime load the code that holds the scratch, and so create it, now.
hgm_status noalloc_prepare();
}  // namespace hgm
