/*
 * hgm.h -- C ABI of libhgm: exact chain hypergraph matching of space-time
 * interest points on one GB300 GPU (sm_103a).
 *
 * The library solves, for every scene time offset, the matching problem of
 * Lombardi, Wolf, Celiktutan and Sankur, "Activity recognition from videos
 * with parallel hypergraph matching on GPUs" (arXiv 1505.00581): the model
 * points, ordered by frame, form a second-order chain hypergraph (Sec. 2.1);
 * each is assigned a scene point so as to minimise
 *     E(z) = sum_i U(z_i) + sum_{i>=3} D(z_i, z_{i-1}, z_{i-2})          (Eq. 9)
 * with U the weighted descriptor distance (Eq. 2, lambda1 absorbed) and D the
 * weighted temporal + angle distortion of the triangle (Eqs. 3-6, lambda2 and
 * lambda3 absorbed), under causality and temporal closeness (Eqs. 7-8). The
 * minimum is exact: the backward min-sum recursion of Eq. 10 with its
 * initialisation (Eq. 11), argmin tables and backtracking (Eq. 12) and the
 * initial pair search (Eq. 13).
 *
 * Problem statement per call (Sec. 2): matching is done one (model, scene)
 * pair at a time; hgm_match_batch runs many pairs in one pass. For a pair,
 * the offsets are o = -t_1 .. F_s-1-t_M (the shifted model lies inside the
 * scene; t_1/t_M are the model's first/last frames, F_s the scene's frame
 * count). At offset o, model point i may only take one of its candidates
 * C_i(o): the scene points whose frame lies in [t_i+o-w, t_i+o+w]; when more
 * than K qualify, the K with the smallest U (ties: lower scene index in the
 * stably time-sorted scene), listed by ascending scene index.
 *
 * Conventions shared by every entry point
 *  - Every function returns an hgm_status; nothing aborts. On failure
 *    hgm_last_error() returns a message (thread-local, valid until the next
 *    call on the same thread).
 *  - "stream" is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream. Device work is ordered on that stream. The library's shared
 *    workspace is ordered across streams: each call's work waits for the
 *    previous call's, whatever stream that was on (plans and stream objects
 *    own their buffers; calls on one stream object must not overlap).
 *  - A pointer documented "host or device" may be either; the library asks
 *    the CUDA driver which. Host outputs make the call synchronous on the
 *    stream; device outputs leave it asynchronous.
 *  - Point arrays are row-major: xy is n x 2 float (x, y), t is n int32 frame
 *    indices, desc is n x F float. The library copies them; the caller keeps
 *    ownership of its buffers. Handles own device memory until hgm_destroy.
 *  - Indices returned to the caller are the caller's own point indices
 *    (positions in the arrays given to hgm_create_*), not sorted ones,
 *    except where an entry point says "sorted".
 *  - An offset at which some C_i(o) is empty or no chain is feasible is not
 *    an error: its energy is +inf and its assignment row is all -1.
 */
#ifndef HGM_H
#define HGM_H

#include <stdint.h>

#if defined(__GNUC__)
#define HGM_API __attribute__((visibility("default")))
#else
#define HGM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hgm_model hgm_model;
typedef struct hgm_scene hgm_scene;
typedef struct hgm_prop hgm_prop;
typedef struct hgm_plan hgm_plan;
typedef struct hgm_stream hgm_stream;

typedef enum {
    HGM_OK = 0,
    HGM_EINVAL = 1,         /* invalid argument (shape, range, NULL, non-finite data) */
    HGM_ENOMEM = 2,         /* device or host allocation failed */
    HGM_ECUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
    HGM_ETIMEOUT = 4,       /* a bounded device-side wait gave up */
    HGM_EUNSUPPORTED = 5    /* valid request outside what this library implements (e.g. K > 64) */
} hgm_status;

/* Matching parameters. Defaults (hgm_default_params) are the paper's weights
 * lambda1 = 0.6, lambda2 = 0.2, lambda3 = 5 and T = 10 frames (Sec. 4), with
 * window w = 3 and cap K = 64. */
typedef struct {
    float lambda1;      /* weight of U (Eq. 1) */
    float lambda2;      /* weight of D (Eq. 1) */
    float lambda3;      /* weight of D^g inside D (Eq. 3) */
    int32_t T;          /* temporal closeness limit in frames (Eq. 8): a triple (a,b,c) needs
                           t'(a) - t'(c) < T; T <= 0 means no limit */
    int32_t window;     /* candidate window half-width w in frames, >= 0 */
    int32_t K;          /* candidate cap, 1..64 (1..255 is valid; > 64 is HGM_EUNSUPPORTED) */
    int32_t precision;  /* 0 = FP32 exact path; 1 = unary table as a BF16 tensor-core contraction
                           (|a|^2 + |b|^2 - 2 a.b, FP32 accumulation) with the 8 smallest candidates
                           of every list re-scored from the FP32 descriptors */
    int32_t offset_lo;  /* restrict offsets to [offset_lo, offset_hi] (inclusive); */
    int32_t offset_hi;  /* INT32_MIN / INT32_MAX (the defaults) mean all offsets */
    const struct hgm_prop *prune;  /* NULL: exact path. Else the proposal network keeps the `keep` best
                                      candidates of every list (ties: lower slot) before the recursion; units
                                      whose pruned optimum is infeasible are re-solved on the full lists. */
    int32_t keep;       /* candidates kept per list when pruning, 1..K (default 8) */
    int32_t refine;     /* with pruning: per (model, scene) pair, the `refine` offsets of lowest pruned
                           energy are solved again without pruning (same precision mode), so a pair's
                           minimum over offsets is the unpruned one whenever its offset is among them.
                           0 (default) = off; 0..65535. Not available in plans (HGM_EUNSUPPORTED). */
    float dummy_cost;   /* W^d of Eq. 2: >= 0 adds the dummy assignment eps to every candidate list (model
                           point not found; U(eps) = W^d, terms involving eps vanish, a triple holding
                           eps must order its real points in time within T); eps is reported as -2 in
                           assignments. < 0 (default -1) = off. HGM_EUNSUPPORTED with pruning and in the
                           whole-block, streaming and no-allocation forms. */
} hgm_params;

/* Fills *p with the defaults above (prune = NULL, keep = 8, refine = 0). */
HGM_API void hgm_default_params(hgm_params *p);

/* Creates a model from M points (host or device pointers; copied). The chain
 * order is the points' stable order by frame (Sec. 2.1: the hypergraph links
 * each point to its two frame-wise predecessors). M >= 3 (Eq. 9 needs one
 * triangle), 1 <= F <= 4096, frames >= 0, all values finite; else
 * HGM_EINVAL. The first model or scene created on a device also creates the
 * fixed 64 MiB scratch of hgm_match_noalloc there (HGM_ECUDA if that fails). */
HGM_API hgm_status hgm_create_model(const float *xy, const int32_t *t, const float *desc, int32_t M, int32_t F,
                            void *stream, hgm_model **out);

/* Creates a scene from S points (host or device pointers; copied). The scene
 * is stored stably sorted by frame with its minnode table (Sec. 3.4: first
 * point of every frame). n_frames is the scene length F_s (frames are
 * 0..F_s-1); n_frames <= 0 means max(t)+1. S >= 0 (an empty scene has no
 * feasible offset), frames in [0, F_s), values finite; else HGM_EINVAL.
 * Creates the scratch of hgm_match_noalloc as hgm_create_model does. */
HGM_API hgm_status hgm_create_scene(const float *xy, const int32_t *t, const float *desc, int32_t S, int32_t F,
                            int32_t n_frames, void *stream, hgm_scene **out);

/* Releases a model, scene, proposal-network, plan or stream handle and its device
 * memory. NULL is a no-op.
 * Work on the handle must be complete (or ordered before on the stream the
 * handle was used on) -- the call synchronises the device first. */
HGM_API void hgm_destroy(void *handle);

/* Message for the last failed call on this thread ("" if none). */
HGM_API const char *hgm_last_error(void);

/* Number of offsets and the first one for a (model, scene, params) triple,
 * host only, no device work. */
HGM_API hgm_status hgm_offsets(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                       int32_t *n_offsets, int32_t *first_offset);

/* Solves every offset of one (model, scene) pair (Eqs. 10-13).
 *  energy [n_offsets] float (host or device, or NULL): minimal E per offset,
 *         +inf where infeasible.
 *  assign [n_offsets x M] int32 (host or device, or NULL): row k is the
 *         optimal assignment at offset first_offset + k; column i is the
 *         caller's model point i, the value the caller's scene index (or -1).
 *  n_offsets / first_offset (host, may be NULL) receive the offset range.
 * With both outputs NULL only the offset range is computed. */
HGM_API hgm_status hgm_match(const hgm_model *model, const hgm_scene *scene, const hgm_params *params, void *stream,
                     int32_t *n_offsets, int32_t *first_offset, float *energy, int32_t *assign);

/* Output layout of a batch of n_models x n_scenes pairs; pair p = m*n_scenes + s.
 * All arrays host, caller-allocated:
 *  first_offset [n_pairs]        first offset of pair p
 *  energy_start [n_pairs + 1]    pair p's energies occupy energy[energy_start[p] .. energy_start[p+1])
 *  assign_start [n_pairs + 1]    pair p's assignment rows (M_m int32 each) start at assign[assign_start[p]]
 * Any of them may be NULL. */
HGM_API hgm_status hgm_batch_layout(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                            int32_t n_scenes, const hgm_params *params, int32_t *first_offset,
                            int64_t *energy_start, int64_t *assign_start);

/* Solves every offset of every (model, scene) pair in one pass: the unit
 * list (model, scene, offset) is ordered by decreasing model size and run by
 * persistent kernels, in chunks bounded by the workspace budget. Scenes whose
 * unary table (model points x scene points x 4 bytes) exceeds the budget are
 * cut into offset segments (each with the frames its windows reach), solved
 * group by group; results do not depend on the segmentation.
 * energy (host or device, or NULL) and assign (host or device, or NULL) use
 * the layout of hgm_batch_layout. */
HGM_API hgm_status hgm_match_batch(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                           int32_t n_scenes, const hgm_params *params, void *stream, float *energy,
                           int32_t *assign);

/* The "independent chains" variant for models with several points per frame
 * (Sec. 4, multiple points per frame, method 2; Table 4): the model's points
 * are split into single-point chains -- chain k takes the point of
 * within-frame rank k (ranked by the caller's index) of every model frame
 * that has one -- each chain with at least 3 points is solved as its own
 * model (Eqs. 10-13) over the whole model's offset range (the same offsets
 * as hgm_match), and the matching distance at an offset is the mean of the
 * chain energies, summed in chain order in FP32 (+inf where any chain is
 * infeasible). energy [n_offsets], assign [n_offsets x M] (host or device,
 * or NULL): each model point gets its chain's optimal scene point (-1 for
 * points of chains shorter than 3, and for the whole row where a chain is
 * infeasible). n_chains in 1..255; HGM_EINVAL if no chain of the model has
 * 3 points. The split is kept on the model handle (rebuilt when n_chains
 * changes; the first call for a model and n_chains synchronises the stream).
 * params apply to every chain as in hgm_match_batch (precision, pruning and
 * the dummy assignment included; the refinement is not applied).
 * Completion as for hgm_match. */
HGM_API hgm_status hgm_match_chains(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                                    int32_t n_chains, void *stream, int32_t *n_offsets, int32_t *first_offset,
                                    float *energy, int32_t *assign);

/* hgm_match_chains for every (model, scene) pair of a batch in one pass: all
 * chains of all models are run as one hgm_match_batch, then combined per pair.
 * energy and assign use the layout of hgm_batch_layout for the same models,
 * scenes and params. Completion as for hgm_match_batch. */
HGM_API hgm_status hgm_match_chains_batch(const hgm_model *const *models, int32_t n_models,
                                          const hgm_scene *const *scenes, int32_t n_scenes,
                                          const hgm_params *params, int32_t n_chains, void *stream, float *energy,
                                          int32_t *assign);

/* The whole-block problem: the paper's own formulation (Sec. 2.2 and Sec. 3),
 * with no time offsets and no candidate windows. Every scene point is a
 * candidate of every model point; only the constraints of Eqs. 7-8 (reading
 * R3: t'(z_{i-2}) <= t'(z_{i-1}) <= t'(z_i), t'(z_i) - t'(z_{i-2}) < T,
 * distinct points) restrict the chain. The recursion (Eqs. 10-13) runs over
 * the band of the trellis these constraints leave (Sec. 3.3), its loop bounds
 * taken from the minnode table (Sec. 3.5). One result per (model, scene)
 * pair, pair q = m * n_scenes + s:
 *  energy [n_models x n_scenes] (host or device, or NULL): the minimum of
 *      Eq. 9, +inf if no chain is feasible;
 *  assign (host or device, or NULL): for pair q, M_m entries starting at
 *      sum of M over the earlier pairs; the caller scene index of each caller
 *      model point, -1 where infeasible.
 * params: lambda1..3 and T are used (T <= 0: no closeness limit); window, K
 * and the offset range are ignored. HGM_EUNSUPPORTED for precision 1 or
 * pruning, or if more than 65535 scene points lie within T frames of one
 * frame (the argmin tables hold 16-bit offsets); HGM_ENOMEM if the argmin
 * tables, (M-2) x cells x 2 bytes per pair, do not fit. Completion as for
 * hgm_match_batch (asynchronous with device outputs). */
HGM_API hgm_status hgm_match_block(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                                   int32_t n_scenes, const hgm_params *params, void *stream, float *energy,
                                   int32_t *assign);

/* Streaming blocks (Sec. 4: for continuous video the scene is cut into
 * blocks of about 60 frames, each matched whole against every model as it
 * arrives). A stream keeps the models' rows, the band and argmin tables and
 * pinned staging buffers between blocks, all sized at creation for blocks of
 * up to max_points points, so a block costs one upload, six kernel launches
 * and the read-back of its results, and hgm_stream_match never allocates
 * device or pinned memory.
 * hgm_stream_create: models (handles; they must outlive the stream), params
 * as for hgm_match_block, block_frames >= 1 (frames of one block),
 * max_points >= 1 (the largest block; the band tables are sized for
 * max_points^2 cells, the argmin tables for sum(M - 2) x max_points^2 16-bit
 * entries). HGM_ENOMEM if those do not fit. Release with hgm_destroy. */
HGM_API hgm_status hgm_stream_create(const hgm_model *const *models, int32_t n_models, const hgm_params *params,
                                     int32_t block_frames, int32_t max_points, void *stream, hgm_stream **out);

/* Matches one block: n points (xy n x 2, t n with frames in [0, block_frames)
 * relative to the block's first frame, desc n x F; host or device) against
 * every model as hgm_match_block does for one scene. energy [n_models] and
 * assign [sum of M] (host or device, or NULL) follow hgm_match_block's
 * layout; assignments are indices into this call's point arrays. With host
 * outputs the call returns when the results are there (HGM_EINVAL if a
 * descriptor was non-finite); with device outputs it is asynchronous. Blocks
 * that overlap (e.g. 60 frames every 30) are separate calls. A block of more
 * than the stream's max_points points is HGM_EUNSUPPORTED. */
HGM_API hgm_status hgm_stream_match(hgm_stream *s, const float *xy, const int32_t *t, const float *desc, int32_t n,
                                    void *stream, float *energy, int32_t *assign);

/* Completion: hgm_match and hgm_match_batch return once their work is queued
 * on `stream` when both outputs are device pointers and no tensor-core kernel
 * runs (precision 0, no pruning); with a host output, precision 1 or pruning
 * they return after the work has finished, so that HGM_ETIMEOUT (a bounded
 * tensor-core wait gave up) can be reported. */

/* Plans (the batch driver's replay form; the paper's one-launch-per-step
 * OpenCL driver has no counterpart): the work of hgm_match_batch for fixed
 * models, scenes, params and device outputs is laid out once -- segment
 * groups, unit lists in decreasing model size, workspace -- and recorded as a
 * CUDA graph that hgm_plan_run replays with a single launch.
 * hgm_plan_create runs the batch once (sizing pass; results are written) and
 * records a second pass without executing it. energy / assign must be device
 * pointers (or NULL) in the hgm_batch_layout order. The model, scene and
 * proposal-network handles and the outputs must outlive the plan: the graph
 * holds their device addresses (their contents, e.g. retrained weights, may
 * change between runs). The plan owns its workspace, so plans and ordinary
 * calls do not share buffers. Release with hgm_destroy.
 * HGM_EINVAL: bad arrays, params or host outputs. */
HGM_API hgm_status hgm_plan_create(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                                   int32_t n_scenes, const hgm_params *params, float *energy, int32_t *assign,
                                   void *stream, hgm_plan **out);

/* Replays the plan on `stream` (asynchronous: one graph launch). */
HGM_API hgm_status hgm_plan_run(hgm_plan *plan, void *stream);

/* Waits for `stream` and reports HGM_ETIMEOUT if a bounded tensor-core wait
 * gave up in a replay since the last run was issued. */
HGM_API hgm_status hgm_plan_check(hgm_plan *plan, void *stream);

/* ---- learned candidate proposal ---------------------------------------------- */

/* The paper has no learned component; this small network is layered on the
 * exact method as a pruning stage. For descriptors of width F it scores a
 * candidate scene point j of model point i at offset o from
 *   x = [f_i (F), f'_j (F), (x'_j - x_i)/100, (y'_j - y_i)/100, (t'_j - t_i - o)/w]   (d_in = 2F + 3)
 * as z3 = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 (hidden width 128), keep
 * score sigmoid(z3). Every contraction runs in BF16 on the tensor cores with
 * FP32 accumulation; weights, gradients and Adam moments are FP32.
 * Weights cross the ABI in one host array, in this order: W1 [128 x d_in]
 * row-major, b1 [128], W2 [128 x 128], b2 [128], w3 [128], b3 [1]
 * (hgm_prop_size(F) floats). hgm_destroy releases a handle. */
HGM_API hgm_status hgm_prop_create(int32_t F, const float *weights /* host or NULL: He init from seed */,
                                   uint64_t seed, hgm_prop **out);
HGM_API int64_t hgm_prop_size(int32_t F);
HGM_API hgm_status hgm_prop_get(const hgm_prop *prop, float *weights /* host */, int64_t *step /* or NULL */);
/* Replaces the weights (host array) and resets the Adam moments; step is the
 * optimizer step count to resume from. */
HGM_API hgm_status hgm_prop_set(hgm_prop *prop, const float *weights, int64_t step);
/* Logits z3 [B] (device) of the rows of X [B x d_in] (device, row-major). */
HGM_API hgm_status hgm_prop_forward(hgm_prop *prop, const float *X, int32_t B, void *stream, float *logits);
/* Mean binary cross-entropy of labels y [B] (device, 0/1) and its gradient
 * with respect to every weight, in the weight order above (host array). */
HGM_API hgm_status hgm_prop_gradients(hgm_prop *prop, const float *X, const float *y, int32_t B, void *stream,
                                      float *loss /* host, or NULL */, float *grad /* host */);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on batch
 * (X, y); loss (host or device float, or NULL) receives the batch loss before
 * the step. Asynchronous on the stream when loss is NULL or a device pointer. */
HGM_API hgm_status hgm_prop_train_step(hgm_prop *prop, const float *X, const float *y, int32_t B, float lr,
                                       void *stream, float *loss);

/* ---- tuning ---------------------------------------------------------------- */

/* The recursion kernel (Eq. 10) comes in tile variants that differ only in how
 * the work is split (0: 4 z_{i-2} cells per thread, 1: 8 cells per thread,
 * 2: 4 cells per thread with half the threads per unit); results are
 * identical. hgm_autotune times every variant on this batch restricted to
 * offsets [max(offset_lo, 0), +sample_offsets) (full pipeline, CUDA events,
 * best of two after a warm-up), makes the fastest the process-wide choice and
 * returns it; ms_per_variant (host, may be NULL) receives each variant's time
 * (3 entries). hgm_set_recurse_variant restores
 * a cached choice. */
HGM_API hgm_status hgm_autotune(const hgm_model *const *models, int32_t n_models, const hgm_scene *const *scenes,
                                int32_t n_scenes, const hgm_params *params, void *stream, int32_t sample_offsets,
                                int32_t *best_variant, float *ms_per_variant);
HGM_API hgm_status hgm_set_recurse_variant(int32_t variant);
HGM_API int32_t hgm_get_recurse_variant(void);

/* ---- matching without device allocation --------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory while they run: a real-time video loop
 * that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause, or a host framework that reserves all GPU memory at start-up.
 * Same result as hgm_match for one (model, scene) pair and all its offsets
 * (params->offset_lo/hi respected) on the FP32 exact path, but every
 * intermediate (unary table, candidate lists, argmin tables, unit records)
 * lives in one fixed 64 MiB scratch array compiled into the library. Offsets
 * are processed in chunks that fit the scratch. No cudaMalloc, cudaFree or
 * allocating library call is made.
 *  energy [n_offsets] float, assign [n_offsets x M] int32: DEVICE pointers
 *         (the layout of hgm_match; n_offsets from hgm_offsets).
 * When the scratch appears: the first hgm_create_model or hgm_create_scene on
 * a device creates it there (by looking up its device address, which loads
 * the library code that holds it) and it stays until the process exits. So
 * create the handles on a device before reserving its memory for other uses
 * and before any stream capture; hgm_match_noalloc itself then neither
 * allocates nor loads anything.
 * Errors: params are checked as by hgm_match (HGM_EINVAL for invalid values);
 * then HGM_EUNSUPPORTED, with a message, for the options this entry point
 * leaves out: precision != 0, dummy_cost >= 0, prune != NULL, refine > 0.
 * HGM_EUNSUPPORTED (with the byte counts in the message) also when one offset
 * of this pair does not fit the scratch -- the unary table alone needs
 * M x S x 4 bytes; HGM_EINVAL for host outputs or bad handles.
 * All calls share the scratch and it keeps the last call's contents: calls
 * whose GPU work may overlap (other streams, other threads) race and must be
 * serialised by the caller. */
HGM_API hgm_status hgm_match_noalloc(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                                     void *stream, float *energy, int32_t *assign);

/* Workspace budget in bytes for one segment group's unary table and for one
 * chunk's candidate lists and argmin tables (0 = automatic: a third of the
 * free device memory, at most 24 GiB). */
HGM_API hgm_status hgm_set_workspace_budget(int64_t bytes);

/* ---- kernel-level entry points (used by the parity tests) -------------- */

/* Stable frame order of a handle's points: perm[k] = caller index of the
 * k-th point in sorted order (host, n entries). */
HGM_API hgm_status hgm_model_order(const hgm_model *model, int32_t *perm);
HGM_API hgm_status hgm_scene_order(const hgm_scene *scene, int32_t *perm);

/* The unary table of Sec. 3.3: U[i*S + j] = lambda1 * ||f_i - f'_j|| for
 * sorted model point i and sorted scene point j, FP32, components summed in
 * order with fused multiply-add and an IEEE square root (the same value as
 * the candidate ranking key). U: device, M x S floats. */
HGM_API hgm_status hgm_unary(const hgm_model *model, const hgm_scene *scene, float lambda1, void *stream, float *U);

/* The same table in the precision mode: U[i*S + j] = lambda1 * sqrt(max(0,
 * |f~_i|^2 + |f~'_j|^2 - 2 f~_i . f~'_j)) with f~ the BF16-rounded descriptors,
 * products accumulated in FP32 on the tensor cores (tcgen05). U: device,
 * M x S floats. Synchronous; HGM_ETIMEOUT if a bounded tensor-core wait gave up. */
HGM_API hgm_status hgm_unary_bf16(const hgm_model *model, const hgm_scene *scene, float lambda1, void *stream,
                                  float *U);

/* Candidate lists for offsets first..first+n-1 (all must be valid offsets):
 *  idx [n x M x K] int32 (device): sorted scene indices of C_i(o) in
 *      ascending order, -1 after the last one; i is the sorted model index.
 *  cnt [n x M] int32 (device): |C_i(o)|.
 *  cost [n x M x K] float (device, or NULL): the unary cost of each
 *      candidate as the recursion receives it, +inf after the last one. With
 *      precision 1 the lists are ranked on the BF16 table and the 8 smallest
 *      of each list (ties: lower slot) carry their FP32 cost, computed as
 *      hgm_unary computes it (the same bits); the others keep the BF16 value. */
HGM_API hgm_status hgm_candidates(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                          int32_t first, int32_t n, void *stream, int32_t *idx, int32_t *cnt, float *cost);

/* The proposal network's logit for every candidate of offsets first..first+n-1
 * of one pair, as the pruning pass computes it: the first layer from the
 * per-point projections P and Q (position terms folded in), layer 2 on the
 * tensor cores with BF16 operands and FP32 accumulation, relu, output layer in
 * FP32. Candidates are those of hgm_candidates (params->prune is ignored; prop
 * is used). scores [n x M x K] float (device): slot c of list (offset, sorted
 * model index i); -inf for empty slots. HGM_EUNSUPPORTED if K > 64,
 * HGM_ETIMEOUT if a bounded tensor-core wait gave up. Synchronous. The paper
 * has no learned pruning; this checks the pruning pass's scores. */
HGM_API hgm_status hgm_prop_scores(const hgm_prop *prop, const hgm_model *model, const hgm_scene *scene,
                                   const hgm_params *params, int32_t first, int32_t n, void *stream, float *scores);

/* Feasible (z_i, z_{i-1}, z_{i-2}) triples of the recursion at each offset
 * (the work Sec. 2.2 counts as O(S M T^2) after pruning):
 * triples [n] int64 (device). Used to state algorithmic work. */
HGM_API hgm_status hgm_count_triples(const hgm_model *model, const hgm_scene *scene, const hgm_params *params,
                             int32_t first, int32_t n, void *stream, int64_t *triples);

/* The FP32 two-argument arctangent the recursion kernel uses for the angle
 * tables of Eq. 6 (reading R1: atan2(0,0) = 0), applied elementwise:
 * out[k] = atan2(y[k], x[k]). y, x, out: device arrays of n floats. A test
 * hook, so that the function's error bound can be checked against FP64. */
HGM_API hgm_status hgm_atan2_f32(const float *y, const float *x, int64_t n, void *stream, float *out);

/* Test hook for the bounded waits of the tensor-core kernels: one warp waits,
 * with the same bounded mbarrier poll, on a barrier that nothing completes,
 * gives up after `polls` polls (1..2^20) and sets *status (device int32) to 1;
 * the context stays usable. Asynchronous on `stream`. */
HGM_API hgm_status hgm_debug_timeout(uint32_t polls, void *stream, int32_t *status);

/* C = bf16(A) * bf16(B)^T, FP32 accumulation on the 5th-generation tensor cores
 * (tcgen05.mma, accumulator in tensor memory): A [M x K], B [N x K], C [M x N],
 * row-major FP32 device arrays; K a multiple of 16 in 16..256. A test hook
 * that pins the shared-memory operand layout and the descriptors used by the
 * BF16 kernels. *status (device int, caller-zeroed) becomes 1 if a bounded
 * wait for the tensor core gave up (C is then incomplete). */
HGM_API hgm_status hgm_gemm_bf16(const float *A, const float *B, int32_t M, int32_t N, int32_t K, void *stream,
                                 float *C, int32_t *status);

/* ---- profiling ----------------------------------------------------------- */

/* on = 1: every launch of the kernels below is bracketed by CUDA events on
 * its stream and its duration accumulated:
 *   0 = unary distance, 1 = candidate selection, 2 = recursion, 3 = backtrack,
 *   4 = proposal-network pruning.
 * hgm_profile_read synchronises on the recorded events and returns, per
 * kernel, total milliseconds and launch count since the last reset.
 * on = 2: batch calls instead run the accounting variant of the recursion
 * kernel (same results), which adds the number of (z_i, z_{i-1}, z_{i-2})
 * evaluations its triple loop performs to a counter read by
 * hgm_profile_evaluated. on = 0: off. */
HGM_API hgm_status hgm_profile_enable(int32_t on);
/* Reads (and with reset != 0, then clears) the evaluation counter of on = 2. */
HGM_API hgm_status hgm_profile_evaluated(int64_t *evaluated, int32_t reset);
/* Units solved on the pruned lists and units re-solved on the full lists
 * (fallback) by batch calls with pruning, since the last reset. */
HGM_API hgm_status hgm_prune_counters(int64_t *pruned_units, int64_t *fallback_units, int32_t reset);
/* Units solved again by the refinement (hgm_params.refine) since the last reset. */
HGM_API hgm_status hgm_refine_counter(int64_t *refined_units, int32_t reset);
HGM_API hgm_status hgm_profile_read(double *ms, int64_t *launches, int32_t n_kernels);
HGM_API hgm_status hgm_profile_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* HGM_H */
