/*
 * gve.h -- C ABI of libgve: fixed-budget Gaussian volume encoding on one
 * B300 GPU (sm_103a), after arxiv 2608.14112 ("Fixed-Budget Gaussian Volume
 * Encoding with Structure-Aware Allocation").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.   Arguments named *_dev are device pointers (cudaMalloc, torch,
 *             or any allocator of the calling process on the context's
 *             device); every other pointer is a host pointer.  The caller
 *             owns every buffer it passes.  The context owns its scratch
 *             (pair lists, sort buffers, partial sums), grown on demand.
 * Streams.    `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *             default stream).  Calls are stream-ordered and asynchronous
 *             unless they return a host value (stats, feasible_max, pair
 *             counts), in which case they synchronise `stream` first.
 * Field.      float32 [nz][ny][nx], x fastest; voxel (i,j,k) has its centre
 *             at the voxel-index position (i,j,k) (Sec. III-B).  Values are
 *             expected normalised to [0,1] (Sec. III-B).
 * Primitive.  12 float32 per Gaussian, 48 bytes (Sec. III-J, Eq. 7):
 *             [mu_x mu_y mu_z, log s_0 log s_1 log s_2, q_w q_x q_y q_z,
 *              a, w_logit] -- the unconstrained parameters of Eq. 2
 *             (log-scales, quaternion normalised in every evaluation,
 *             w = sigmoid(w_logit)); 16-byte aligned.
 * Errors.     Every entry point returns a gve_status; nothing aborts or
 *             throws across the ABI.  gve_last_error() gives a message.
 *             Invalid arguments are rejected before any launch.
 * Counts.     At most 2^24 (16,777,216) primitives per call; grid axes up to
 *             2^14 (16,384) voxels for evaluation and refinement (the float32
 *             margins of the brick cover hold for coordinates below 2^14) and
 *             2^24 for allocation, with fewer than 2^31 bricks.
 * Threads.    A context may be used by one host thread at a time.
 */
#ifndef GVE_H
#define GVE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GVE_API __attribute__((visibility("default")))
#else
#define GVE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GVE_OK = 0,
    GVE_E_INVALID = 1,    /* bad argument (null pointer, size, option)            */
    GVE_E_BUDGET = 2,     /* infeasible budget; *feasible_max holds the largest
                             feasible one (Sec. V-B)                               */
    GVE_E_NOMEM = 3,      /* device scratch could not be allocated                 */
    GVE_E_CUDA = 4,       /* a CUDA runtime call failed                            */
    GVE_E_TIMEOUT = 5,    /* a bounded device-side wait gave up                    */
    GVE_E_CAPACITY = 6,   /* pair buffer overflow that survived the internal retry */
    GVE_E_INTERNAL = 7    /* device-side consistency check failed                  */
} gve_status;

typedef struct { int32_t nx, ny, nz; } gve_dims;

/* Field evaluation options (Sec. III-C, Eq. 3).
 * trunc_k    truncation radius in standard deviations: a pair is kept when its
 *            squared Mahalanobis distance is below trunc_k^2 (paper: 5).
 *            The keep decision is taken in float32 by a fixed chain of fused
 *            multiply-adds on float32 coefficients of -0.5*log2(e)*Sigma^-1.
 * rho0       density floor of Eq. 3 (paper: 0.05).
 * normalized 1 = Eq. 3 (sum w a G / max(sum w G, rho0)); 0 = plain sum w a G.
 * brick      brick edge B in voxels for binning: 4, 8 or 16 (8 by default).
 * gaussians_per_block  Gaussian records the evaluator stages per shared-memory
 *            chunk: 32 or 64, 0 = 64.  B and this value change speed only,
 *            never results (a tuning knob, see gve_autotune).                */
typedef struct {
    float trunc_k;
    float rho0;
    int32_t normalized;
    int32_t brick;
    int32_t gaussians_per_block;
} gve_eval_opts;

/* Allocation options (Sec. III-E, Table III).
 * detail_frac  share of the budget drawn in proportion to |grad V| (0.55).
 * occ_thresh   occupancy threshold: voxels with V > occ_thresh (0.02).
 * w0           initial weight w = sigmoid(w_logit) of every Gaussian (0.1).
 * seed         seed of the Philox4x32-10 streams of the draws and jitter.   */
typedef struct {
    double detail_frac;
    double w0;
    float occ_thresh;
    int32_t reserved;     /* set to 0 */
    uint64_t seed;
} gve_alloc_opts;

/* Refinement schedule (Sec. III-E).  One iteration = evaluate every voxel,
 * mean squared error, analytic gradient, one Adam step on all 12N values.
 * mask_thresh  < 0: plain MSE over all voxels; >= 0: only voxels with
 *              V > mask_thresh contribute to the loss (Eq. 6 mask).
 * step0        Adam step counter before the first iteration (0 = fresh).  */
typedef struct {
    int32_t iters;
    float lr, beta1, beta2, eps;
    float mask_thresh;
    int32_t step0;
    gve_eval_opts eval;
} gve_schedule;

/* Host-side summary of a refinement. */
typedef struct {
    double loss_first;     /* loss at the starting parameters                 */
    double loss_last;      /* loss of the last iteration (before its update)  */
    double sse_final;      /* unmasked sum of squared errors after the last
                              update (one extra evaluation)                    */
    double psnr_final;     /* 10 log10(M / sse_final)  (Sec. IV-C)            */
    int64_t brick_pairs;   /* (brick, Gaussian) pairs of the final evaluation */
    int64_t launches;      /* kernels launched by the call                    */
    int32_t iters_done;
    int32_t retries;       /* pair-capacity regrowths during the call         */
    float ms_total;        /* device time of the call (CUDA events)           */
    float ms_brick;        /* device time of the brick evaluator, summed over
                              the iterations (events on the call's stream)     */
    float ms_bin;          /* device time of preparation and binning, summed  */
    float ms_fwd;          /* device time of the brick evaluator's forward
                              phase alone: the final evaluation after the last
                              update (a forward-only launch of the same
                              kernel); 0 when that evaluation was replayed    */
} gve_stats;

/* Summary of an allocation. */
typedef struct {
    int64_t n_occupied, n_eligible, n_detail, n_coverage;
    double gbar;           /* median |grad V| over occupied voxels            */
    double h_detail, h_coverage;   /* group seed spacings (Sec. III-E)        */
} gve_alloc_info;

typedef struct gve_ctx gve_ctx;

/* Context on CUDA device `device`.  Creates no stream; allocates scratch
 * lazily.  *out is NULL on failure.  A context's scratch serves one call at a
 * time: calls on one context from several threads, or overlapping on several
 * streams, must be serialised by the caller (one context per stream). */
GVE_API gve_status gve_ctx_create(gve_ctx** out, int device);
/* Frees the context's scratch (synchronises the device first). NULL is ok. */
GVE_API void gve_ctx_destroy(gve_ctx* ctx);
/* Static description of a status code. */
GVE_API const char* gve_status_str(gve_status s);
/* Message of the last failing call on ctx (never NULL). */
GVE_API const char* gve_last_error(const gve_ctx* ctx);

/* Analytic fixed-budget allocation (Sec. III-E, Table I stages S1a-S1e,
 * Eq. 4).  Draws Nd = floor(detail_frac*budget + 1/2) distinct occupied voxels
 * with |grad V| > 0 with probability proportional to |grad V| (Efraimidis-
 * Spirakis keys), and budget - Nd distinct occupied voxels uniformly; jitters
 * each centre in [-1/2,1/2)^3; orients and shapes each Gaussian from the 7^3
 * structure tensor at its voxel; a = trilinear V(mu); w = w0.
 *   field_dev    [nz][ny][nx] float32 (read only).
 *   prims_dev    [budget][12] float32 output, detail seeds first.
 *   feasible_max host, optional: on GVE_E_BUDGET the largest feasible
 *                budget (Sec. V-B); on success the budget itself.
 *   info         host, optional summary.
 * Synchronises `stream` (the feasibility check reads two counts).
 * Returns GVE_E_BUDGET without writing prims_dev when the field cannot
 * support the budget.  The draws select on 32-bit surrogates of their keys
 * and compute the full keys (FP64 for the detail draw) only near the
 * threshold; the seeds are those of a draw over every voxel's full key
 * (the environment variable GVE_TEST_DRAW_FULL, for tests, forces that
 * draw). */
GVE_API gve_status gve_allocate(gve_ctx* ctx, const float* field_dev, gve_dims dims, int64_t budget,
                        const gve_alloc_opts* opts, float* prims_dev, int64_t* feasible_max,
                        gve_alloc_info* info, void* stream);

/* Field of Eq. 3 at every voxel centre.
 *   prims_dev     [n][12] float32.
 *   field_out_dev [nz][ny][nx] float32 output. */
GVE_API gve_status gve_evaluate(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                        const gve_eval_opts* opts, float* field_out_dev, void* stream);

/* Loss and gradient at the current parameters, no update (Sec. III-E, V-D).
 *   field_dev       target V, [nz][ny][nx].
 *   grad_prims_dev  [n][12] float32 output: dL/d(raw record), L = masked
 *                   sum of squared errors / (nx ny nz).
 *   sse_dev         [2] double output: {masked SSE, unmasked SSE}; may be
 *                   NULL. */
GVE_API gve_status gve_loss_grad(gve_ctx* ctx, const float* prims_dev, int64_t n, const float* field_dev,
                         gve_dims dims, const gve_eval_opts* opts, float mask_thresh,
                         float* grad_prims_dev, double* sse_dev, void* stream);

/* Backward of gve_evaluate for an arbitrary upstream gradient dL/dVtilde
 * (the autograd form): recomputes the field per brick, nothing is saved
 * between the calls.
 *   grad_field_dev  [nz][ny][nx] float32 upstream gradient.
 *   grad_prims_dev  [n][12] float32 output. */
GVE_API gve_status gve_backward(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                        const gve_eval_opts* opts, const float* grad_field_dev,
                        float* grad_prims_dev, void* stream);

/* Fixed-budget refinement (Sec. III-E): sched->iters iterations of
 * evaluate -> MSE -> gradient -> Adam on all primitives; no densification,
 * pruning or count change.
 *   prims_dev       [n][12] float32, updated in place.
 *   field_dev       target V.
 *   adam_state_dev  [2][n][12] float32 first and second moments, updated in
 *                   place (zero them for a fresh run); NULL = the context
 *                   keeps zero-initialised moments for this call only.
 *   loss_trace_dev  [iters] double output of per-iteration losses, or NULL.
 *   stats           host, optional; filling it synchronises `stream`.
 * Pair capacity overflow is detected on the device; the affected iterations
 * leave the parameters untouched and are replayed after the scratch grows. */
GVE_API gve_status gve_refine(gve_ctx* ctx, float* prims_dev, int64_t n, const float* field_dev,
                      gve_dims dims, const gve_schedule* sched, float* adam_state_dev,
                      double* loss_trace_dev, gve_stats* stats, void* stream);

/* One volume of a batch: its target field and its number of primitives. */
typedef struct {
    const float* field_dev;   /* [nz][ny][nx] float32 */
    gve_dims dims;
    int64_t n;                /* primitives of this volume */
} gve_volume;

/* Allocation of a batch (the batched form, Sec. III-E per volume): volume
 * v's vols[v].n Gaussians are allocated, exactly as gve_allocate with opts
 * would allocate them on that volume alone, into rows [off_v, off_v + n_v)
 * of prims_dev (volumes in order, concatenated; off_v = sum of the earlier
 * n).  The volumes run concurrently: up to 8 host threads, each with its own
 * internal context (scratch of about 12 bytes per voxel of the largest
 * volume it takes) and stream, largest volumes first; the caller's stream
 * waits for all of them.  infos (host, optional) [nvol] receives each
 * volume's summary.  Returns the first failing volume's status in volume
 * order (gve_last_error names the volume), e.g. GVE_E_BUDGET when its field
 * cannot support its budget; 1 <= nvol <= 32. */
GVE_API gve_status gve_allocate_batch(gve_ctx* ctx, int32_t nvol, const gve_volume* vols,
                                      const gve_alloc_opts* opts, float* prims_dev, gve_alloc_info* infos,
                                      void* stream);

/* Batched refinement of many volumes of uneven shapes (the batched encode
 * form; each volume is refined exactly as gve_refine would, Sec. III-E).
 * The records of all volumes are concatenated in prims_dev ([sum n][12],
 * volume order); adam_state_dev is [2][sum n][12] or NULL; loss_trace_dev is
 * [iters][nvol] or NULL; psnr_out is host [nvol] or NULL (final PSNR of each
 * volume).  One iteration of all volumes is captured once as a CUDA graph
 * (one branch per volume) and replayed; the Adam step lives on the device.
 * 1 <= nvol <= 32.  Synchronises `stream`. */
GVE_API gve_status gve_refine_batch(gve_ctx* ctx, int32_t nvol, const gve_volume* vols, float* prims_dev,
                                    const gve_schedule* sched, float* adam_state_dev,
                                    double* loss_trace_dev, double* psnr_out, gve_stats* stats,
                                    void* stream);

/* Autotuner of the evaluator's launch shape for a batch (nvol = 1 for one
 * volume): times one loss-and-gradient pass, without any update, for each
 * brick edge in {4, 8, 16} and each gaussians_per_block in {32, 64}, and
 * writes the fastest into *opts (other fields unchanged).  ms_out (host,
 * optional) receives the 6 timings in that order (brick-major).
 * Synchronises `stream`. */
GVE_API gve_status gve_autotune(gve_ctx* ctx, int32_t nvol, const gve_volume* vols, const float* prims_dev,
                                gve_eval_opts* opts, float* ms_out, void* stream);

/* ---- learned proposal (the learned-proposal form) --------------------------
 * A small MLP maps each allocated Gaussian's local structure statistics to a
 * correction of its initial amplitude and log-scales; plain allocation (an
 * all-zero last layer) is its fallback and refinement judges it.  The model
 * is one caller-owned float32 device buffer of GVE_MLP_FLOATS words: FP32
 * master parameters [0, P), Adam moments [P, 3P), feature mean and inverse
 * standard deviation [3P, 3P+32), BF16 copies of the parameters packed two
 * per word [3P+32, 3P+32+P/2), P = GVE_MLP_PARAMS, parameter order
 * W1[64][16] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4].
 * The network's input is clamp((x - mean) * istd, -6, 6) per feature.
 * Forward passes use the BF16 copies with FP32 accumulation; GELU is the
 * erf form.  Outputs: (delta a, delta log s0, delta log s1, delta log s2). */
#define GVE_MLP_PARAMS 9668
#define GVE_MLP_FLOATS 33870

/* 16 features per Gaussian from the field and its allocated record (seed
 * voxel = round(mu)): log(1 + lambda_k/(343 gbar^2)) of the 7^3 structure
 * tensor (3, ascending), |grad V|/gbar (capped at 10), mean, standard
 * deviation, min and max of V over the 5^3 window, the 3 log-scales, a,
 * the detail-seed flag (index < n_detail), the occupied fraction (V >
 * occ_thresh) of the 5^3 window, the eigengap (lambda_2 - lambda_1)/lambda_3,
 * V at the seed.  features_dev: [n][16] float32 output. */
GVE_API gve_status gve_proposal_features(gve_ctx* ctx, const float* field_dev, gve_dims dims,
                                         const float* prims_dev, int64_t n, int64_t n_detail, float gbar,
                                         float occ_thresh, float* features_dev, void* stream);
/* Y[rows][4] = MLP(X[rows][16]); save (optional) receives the three hidden
 * pre-activations [rows][3][64] for a backward pass. */
GVE_API gve_status gve_mlp_forward(gve_ctx* ctx, const float* model_dev, const float* X_dev, int64_t rows,
                                   float* Y_dev, float* save_dev, void* stream);
/* Gradient of the mean squared error mean_{rows,4}(MLP(X) - target)^2 with
 * respect to the P parameters (dP_dev, [P] float32, overwritten); loss_dev
 * (optional, device double) receives the loss. */
GVE_API gve_status gve_mlp_grad(gve_ctx* ctx, const float* model_dev, const float* X_dev,
                                const float* target_dev, int64_t rows, float* dP_dev, double* loss_dev,
                                void* stream);
/* One Adam step (bias-corrected, 1-based step) on the master parameters;
 * refreshes the BF16 copies. */
GVE_API gve_status gve_mlp_adam(gve_ctx* ctx, float* model_dev, const float* dP_dev, float lr, float beta1,
                                float beta2, float eps, int32_t step, void* stream);
/* Rounds the master parameters into the BF16 copies (after loading a model). */
GVE_API gve_status gve_mlp_quantise(gve_ctx* ctx, float* model_dev, void* stream);
/* prims[i]: a += delta a, log s += delta log s from MLP(features[i]), the
 * log-scales clamped to [log 0.3, log(max(nx,ny,nz)/16)] (the allocator's
 * scale caps, logarithms in double rounded once to float), so a zero
 * correction leaves an allocation unchanged.  Rows with a non-finite output
 * are left unchanged. */
GVE_API gve_status gve_proposal_apply(gve_ctx* ctx, const float* model_dev, const float* features_dev,
                                      float* prims_dev, int64_t n, gve_dims dims, void* stream);
/* End-to-end gradient of the proposal: with prims_corrected = the output of
 * gve_proposal_apply and grad_prims = dL/dprims at those records (from
 * gve_loss_grad), writes (accumulate = 0) or adds (accumulate != 0) dL/dtheta
 * [GVE_MLP_PARAMS] float32 into dP_dev.  The clamp of the log-scales passes
 * no gradient where it was active.  n >= 1. */
GVE_API gve_status gve_proposal_backward(gve_ctx* ctx, const float* model_dev, const float* features_dev,
                                         const float* prims_corrected_dev, const float* grad_prims_dev,
                                         int64_t n, gve_dims dims, int32_t accumulate, float* dP_dev,
                                         void* stream);

/* Input standardisation of the network from its training features X
 * [rows][16] (rows >= 1): the column means and sample spreads in FP64 (two
 * passes, a fixed summation order) go into the model's mean and inverse
 * spread, a feature whose spread is at most 1e-3 (1 + |mean|) getting
 * inverse spread 0 (it carries nothing to learn from). */
GVE_API gve_status gve_mlp_standardise(gve_ctx* ctx, float* model_dev, const float* X_dev, int64_t rows,
                                       void* stream);
/* Training targets of the proposal from an allocation and its refinement:
 * T[i] = refined minus allocated (a, log s0, log s1, log s2) of record i
 * (prims0_dev, prims1_dev [n][12]; T_dev [n][4], 16-byte aligned). */
GVE_API gve_status gve_proposal_targets(gve_ctx* ctx, const float* prims0_dev, const float* prims1_dev, int64_t n,
                                        float* T_dev, void* stream);
/* Divides each column of a target matrix T_dev [rows][4] (in place,
 * 16-byte aligned) by its sample spread over the rows (FP64, at least
 * 1e-6), the spreads written to scale_dev (device float[4]). */
GVE_API gve_status gve_mlp_scale_targets(gve_ctx* ctx, float* T_dev, int64_t rows, float* scale_dev, void* stream);
/* Multiplies output k of the network's last layer (W4 row k and b4[k]) by
 * scale_dev[k] and refreshes the BF16 copies: a network trained on targets
 * divided by those spreads then predicts the targets themselves. */
GVE_API gve_status gve_mlp_fold_output_scale(gve_ctx* ctx, float* model_dev, const float* scale_dev, void* stream);

/* Pre-encoding structure statistics (Sec. V-F, Table VI) of a device field
 * (float32, [nz][ny][nx], device memory, not modified).  Host output
 * out[5] = {occupancy (V > 0.02), share of the occupied voxels' float32
 * |grad V| mass held by the ceil(n_occ / 10) largest, S(1), S(16),
 * S(1) / S(16)} with S(l) the mean over the axes longer than l of the mean
 * (V(x + l e) - V(x))^2 over all voxel pairs (FP64).  The paper names but
 * does not define S; this second-order structure function is the reading.
 * stage_ms (host, nullable, [4]) receives the device time in ms of the
 * first sweep, of the second sweep with the exact select and of the whole
 * pass, then the number of kernels the call launched.
 * One stencil sweep of the field, which also keeps each voxel's gradient
 * bits in the context (4 bytes per voxel, held until the context is
 * destroyed), then one streaming sweep of those bits; synchronises `stream`.
 * GVE_E_INVALID on null pointers, non-positive sizes or an axis above 2^24. */
GVE_API gve_status gve_structure_stats(gve_ctx* ctx, const float* field_dev, gve_dims dims, double* out,
                                       double* stage_ms, void* stream);

/* ---- stratified-sample refinement (Sec. III-F, Table III) ------------------
 * The paper's training regime: each iteration fits the field at S jittered
 * points drawn by value class -- floor(0.35 S + 1/2) from voxels with
 * V > 0.4, floor(0.40 S + 1/2) from occupied mid-range voxels
 * (0.02 < V <= 0.4), the rest uniformly from the grid (a class without
 * voxels hands its share to the uniform draw).  Sample j of iteration t uses
 * the Philox4x32-10 words of counter (j, t, 4, 'GVE1') under key `seed`:
 * voxel = the floor(x0 count / 2^32)-th of its class (ascending voxel
 * order), point p = c + u with u_k = (x_{k+1} >> 8) 2^-24 - 1/2 rounded to
 * float32, target = trilinear V(p) (FP64, edge-clamped) rounded to float32.
 * Eq. 3 is evaluated at p with the same float32 keep test as at voxel
 * centres; the loss is (1/S) sum_s 1[v_s > occ] (Vt(p_s) - v_s)^2 (occ =
 * schedule mask_thresh, 0.02 when negative).  S <= 8192; grids of fewer than
 * 2^32 voxels; normalized evaluation only. */

/* The points of iteration `iter`: pts_out [S][4] float32 (x, y, z, target),
 * 16-byte aligned; vox_out [S] int64 voxel indices or NULL. */
GVE_API gve_status gve_draw_samples(gve_ctx* ctx, const float* field_dev, gve_dims dims, int64_t S,
                                    uint64_t seed, uint32_t iter, float* pts_out_dev, int64_t* vox_out_dev,
                                    void* stream);
/* The full objective (Sec. III-F): L = L_val + lambda_rho L_rho + lambda_sm
 * L_sm + lambda_anc L_anc + lambda_aniso L_aniso + lambda_cap L_cap.  The
 * paper names the five regularisers and their purpose but gives neither
 * formulas nor weights; the forms are these readings:
 *   L_rho   = (1/S) sum_s 1[v_s > occ] (rho(p_s) - 1)^2, rho = sum w G (the
 *             denominator of Eq. 3 before the floor): density toward one
 *             over occupied space, from both sides;
 *   L_sm    = (1/S) sum_s (rho(p_s) - rho(p'_s))^2, p'_s the partner of p_s:
 *             u = (x >> 8) 2^-24 - 1/2 per axis from the Philox4x32-10 words
 *             of counter (s, t, 5, 'GVE1'), p' = clamp(p + 2 radius u, 0,
 *             n - 1) in float32; its weight decays geometrically from
 *             lambda_sm to lambda_sm_end over anneal_iters iterations;
 *   L_anc   = (1/N) sum_i (a_i - V(mu_i))^2, V trilinear (float32,
 *             edge-clamped); the gradient flows into a_i only;
 *   L_aniso = (1/N) sum_i sum_{j<k} relu(|l_ij - l_ik| - ln aniso_max)^2
 *             over the log-scales l (elongation bounded at aniso_max : 1);
 *   L_cap   = (1/N) sum_i sum_j relu(l_ij - ln s_hi)^2 + relu(ln s_lo -
 *             l_ij)^2 (s_hi <= 0: the allocator's cap, longest axis / 16).
 * With lambda_sm > 0 the partners double the points: S <= 4096.  A NULL
 * option pointer means the value term alone. */
typedef struct {
    float lambda_rho;
    float lambda_sm, lambda_sm_end;
    int32_t anneal_iters;
    float lambda_anc, lambda_aniso, lambda_cap;
    float partner_radius;  /* voxels */
    float aniso_max;
    float s_lo, s_hi;      /* voxels */
} gve_reg_opts;

/* Smoothness partners of caller-given points pts [S][4] for iteration
 * `iter`: out [S][4] = (x', y', z', -1) (no target), 16-byte aligned. */
GVE_API gve_status gve_draw_partners(gve_ctx* ctx, const float* pts_dev, int64_t S, gve_dims dims, uint64_t seed,
                                     uint32_t iter, float radius, float* out_dev, void* stream);

/* Eq. 3, the sampled objective and (grad_out != NULL) its gradient [n][12]
 * at caller-given points pts [S][4] (x, y, z, target), followed by their S
 * partners when reg->lambda_sm > 0 (the weight of this step).  field_dev is
 * needed when lambda_anc > 0.  loss_dev (device double: L), terms_dev
 * (device double[6]: L_val, L_rho, L_sm, L_anc, L_aniso, L_cap unweighted)
 * and vt_out [S] (Vt per sample) are optional. */
GVE_API gve_status gve_sample_loss_grad(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                                        const gve_eval_opts* opts, const float* pts_dev, int64_t S,
                                        float occ_thresh, const gve_reg_opts* reg, const float* field_dev,
                                        float* grad_out_dev, double* loss_dev, double* terms_dev,
                                        float* vt_out_dev, void* stream);
/* sched->iters iterations of draw (and partners) -> sampled objective and
 * gradient -> Adam on every primitive (iteration index sched->step0 + t
 * selects the points, the smoothness weight and the bias correction).
 * reg (nullable) adds the regularisers.  adam_state and loss_trace_dev as
 * for gve_refine (the trace receives the objective per iteration).  stats
 * (optional) adds one full-grid evaluation after the last step for
 * sse_final / psnr_final; ms_total is the iterations' time, ms_brick its
 * draw, search (with the keep coefficients, computed only for Gaussians
 * whose box holds candidate points), loss and gradient share, ms_bin 0 (the
 * chain rule and Adam are the rest). */
GVE_API gve_status gve_refine_sampled(gve_ctx* ctx, float* prims_dev, int64_t n, const float* field_dev,
                                      gve_dims dims, const gve_schedule* sched, int64_t S, uint64_t seed,
                                      const gve_reg_opts* reg, float* adam_state_dev, double* loss_trace_dev,
                                      gve_stats* stats, void* stream);

/* ---- mixture-field ray marcher (Sec. III-A, rendering of the encoded set)
 * Rendering applies a transfer function T = (c_T, alpha_T) to the value Eq. 3
 * returns at sample positions along each camera ray and composites the
 * samples front to back; grad Vt, available in closed form at the sample,
 * shades it.  Nothing is rendered through a graphics API: the image is a
 * device buffer.
 *
 * Camera, in voxel coordinates (voxel centres at integers, the volume box is
 * [-0.5, n - 0.5] per axis): the ray through pixel (i, j) (column i, row j,
 * row 0 at the top) has direction forward + sx right + sy up, normalised,
 * with sx = ((2i + 1) / W - 1) tan_half_fovy (W / H) and sy = (1 - (2j + 1) /
 * H) tan_half_fovy; ray setup and sample positions are float32 in that
 * written order (no contraction).  Samples sit at t = tmin + (k + 1/2) step
 * inside the box (tmin = max(entry, 0)). */
typedef struct {
    float eye[3];
    float right[3], up[3], forward[3];
    float tan_half_fovy;
    int32_t width, height;
} gve_camera;

/* Render options.
 *   step       sample spacing along the ray in voxels, >= 1/64, and at most
 *              65,536 samples across the box diagonal.
 *   term       stop a ray once its transmittance falls below term (0 = off).
 *   ref_step   spacing the table's opacities refer to: a sample's opacity is
 *              1 - (1 - alpha)^(step / ref_step).
 *   background RGB seen through the remaining transmittance.
 *   shade      0: emission-absorption; 1: headlight shading with the normal
 *              n = grad Vt / max(|grad Vt|, gfloor): colour c (ka + kd |n.l|)
 *              + ks |n.l|^shininess, l the direction towards the eye.
 *   tf_dev     [tf_n][4] float32 RGBA table over V in [0, 1] (device memory,
 *              linear interpolation, values clamped to [0, 1]); tf_n >= 2. */
typedef struct {
    float step, term, ref_step;
    float background[3];
    int32_t shade;
    float ka, kd, ks, shininess, gfloor;
    const float* tf_dev;
    int32_t tf_n;
} gve_render_opts;

/* Builds the renderer's lists for a primitive set (once per set; the set may
 * change afterwards, the context keeps its own copy of the coefficients):
 * cells of 8^3 voxels, each listing, in Gaussian order, every Gaussian whose
 * conservative truncation box (the same margins as the sampled refinement)
 * overlaps the cell's continuous extent and whose inflated ellipsoid is not
 * separated from the cell by the plane through the direction to the cell's
 * centre (so no kept sample is lost).  prims_dev [n][12] float32,
 * 16-byte aligned.  Synchronises `stream`.  GVE_E_INVALID for bad sizes,
 * alignment or options, GVE_E_CAPACITY beyond 2^32 pairs. */
GVE_API gve_status gve_render_prepare(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                                      const gve_eval_opts* opts, void* stream);

/* Renders the prepared set: image_dev [height][width][4] float32 RGBA
 * (premultiplied colour plus background, alpha = 1 - transmittance).
 * kept_pairs (host, nullable) receives the kept (sample, Gaussian) pairs,
 * the algorithmic work of the frame, and tested_pairs (host, nullable) the
 * pairs the march tested (list lengths times samples); either synchronises.
 * GVE_E_INVALID without a prepared set, for a non-finite camera, bad
 * options, more than 2^28 pixels or more than 524,280 rows. */
GVE_API gve_status gve_render(gve_ctx* ctx, const gve_camera* cam, const gve_render_opts* opts, float* image_dev,
                              int64_t* kept_pairs, int64_t* tested_pairs, void* stream);

/* Brick binning introspection: the (brick, Gaussian) pairs that evaluation
 * uses, sorted by brick key (z-major brick index) and then by Gaussian index,
 * and per-brick [start, end) ranges.
 *   counts_dev   [n] uint32 output: pairs per Gaussian.
 *   keys_dev, gids_dev  [cap] uint32 outputs.
 *   masks_dev    [cap] uint8 output or NULL: the evaluator's sub-brick cover
 *                of each pair (bit = y half + 2 * z quarter of the B x B/2 x
 *                B/4 sub-bricks), a superset of the sub-bricks holding kept
 *                voxels.
 *   ranges_dev   [2][nbricks] uint32 output (starts, then ends; 0,0 = empty).
 *   n_pairs      host output: number of pairs (synchronises).  If it exceeds
 *                cap, nothing is written and GVE_E_CAPACITY is returned. */
GVE_API gve_status gve_bin(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                   const gve_eval_opts* opts, uint32_t* counts_dev, uint32_t* keys_dev,
                   uint32_t* gids_dev, uint8_t* masks_dev, int64_t cap, uint32_t* ranges_dev,
                   int64_t* n_pairs, void* stream);

/* Number of kept (voxel, Gaussian) pairs of the truncated field -- the
 * algorithmic work of one evaluation -- and the candidate pairs the brick
 * evaluator visits.  Host outputs; synchronises. */
GVE_API gve_status gve_count_pairs(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                           const gve_eval_opts* opts, int64_t* kept_pairs,
                           int64_t* candidate_pairs, void* stream);

/* Kept (voxel, Gaussian) pairs of one evaluation, listed (for checking the
 * keep decision pair by pair): pairs_dev [cap] uint64 output, each entry
 * (voxel index << 24) | Gaussian index, voxel index = (z ny + y) nx + x, in
 * no particular order.  n_pairs (host) receives the number of kept pairs;
 * when it exceeds cap only cap entries are written and GVE_E_CAPACITY is
 * returned.  Grids of at most 2^40 voxels.  Synchronises `stream`. */
GVE_API gve_status gve_kept_pairs(gve_ctx* ctx, const float* prims_dev, int64_t n, gve_dims dims,
                                  const gve_eval_opts* opts, uint64_t* pairs_dev, int64_t cap, int64_t* n_pairs,
                                  void* stream);

/* Stage P of the encoder (Sec. III-B): out = (V - min) / (max - min) over the
 * whole field, in float32 with one correctly rounded subtraction and one
 * correctly rounded division per voxel (a constant field maps to 0).
 *   field_dev  [nz][ny][nx] float32 input.
 *   out_dev    [nz][ny][nx] float32 output; may equal field_dev (in place).
 *   minmax     host, optional [2]: the field's float32 minimum and maximum
 *              (the header of an encoding keeps them to undo the scaling).
 * Returns GVE_E_INVALID without writing out_dev when a value is not finite.
 * Synchronises `stream` (the extremes are read before the scaling pass). */
GVE_API gve_status gve_normalize(gve_ctx* ctx, const float* field_dev, gve_dims dims, float* out_dev, float* minmax,
                                 void* stream);

/* Throughput microbenchmark of the pipes the evaluator runs on (no paper
 * counterpart; it measures the roofline's denominators on the running GPU):
 * kind 0 = scalar float32 FMA, 1 = packed float32x2 FMA (counted as two
 * operations), 2 = SFU ex2.approx.  One launch of 8 CTAs x 256 threads per
 * SM, each thread running 8 independent chains for iters x 16 steps; timed
 * with CUDA events on `stream`.  ops_per_s (host) receives lane-operations
 * per second, ms_out (host, optional) the kernel time.  Synchronises. */
GVE_API gve_status gve_peak_bench(int32_t kind, int64_t iters, double* ops_per_s, float* ms_out, void* stream);

/* Field evaluation that allocates no memory -- an addition for callers that
 * cannot call cudaMalloc (a memory pool or arena that owns the device, a
 * fixed device footprint after start-up, no allocator locks on the call
 * path); the paper has no counterpart.  Same arguments and result as
 * gve_evaluate, without a context.  All scratch lives in one fixed
 * file-scope device array of the library (about 7 MB, held by every GPU
 * that loads the library until the process exits).
 *   prims_dev      [n][12] float32, n <= GVE_NOALLOC_MAX_PRIMS.
 *   dims           at most GVE_NOALLOC_MAX_BRICKS bricks of 8^3, axes up to
 *                  2^14 voxels.
 *   opts           brick must be 8; gaussians_per_block 0, 32 or 64.
 *   field_out_dev  [nz][ny][nx] float32 output.
 * prims_dev and field_out_dev must be memory of the current device (the
 * array and the launches are the current device's); GVE_E_INVALID otherwise.
 * Returns GVE_E_INVALID for sizes beyond the limits (before any launch), and
 * GVE_E_CAPACITY when the (brick, Gaussian) pair count, found on the device,
 * exceeds GVE_NOALLOC_MAX_PAIRS, or the binning's (tile, Gaussian) pairs
 * (tiles of 4^3 bricks) exceed 16 x GVE_NOALLOC_MAX_PRIMS (the output is then
 * not written).  The call
 * synchronises `stream` to read that count.  The first call on a device
 * resolves the array's address with that device current; make it before any
 * stream capture (a cudaDeviceReset invalidates the resolved address).  All
 * calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. */
#define GVE_NOALLOC_MAX_PRIMS 8192
#define GVE_NOALLOC_MAX_BRICKS 32768
#define GVE_NOALLOC_MAX_PAIRS 524288
GVE_API gve_status gve_evaluate_noalloc(const float* prims_dev, int64_t n, gve_dims dims,
                                        const gve_eval_opts* opts, float* field_out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GVE_H */
