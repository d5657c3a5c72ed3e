/*
 * bmf.h -- C ABI of libbmf.so: the BPMF Gibbs sweep and posterior propagation (PP) of
 * Qin et al., "Distributed Bayesian Matrix Factorization with Limited Communication"
 * (arXiv 1703.00734), on one GB300 GPU.
 *
 * Model (Section 2.1): Y (N x D) partially observed, y_nd ~ N(x_n^T w_d, 1/tau) on observed
 * entries (Eqs. 2-3), x_n ~ N(mu_X, Lambda_X^{-1}), w_d ~ N(mu_W, Lambda_W^{-1}) (Eqs. 4a/4b),
 * Normal-Wishart hyperpriors on (mu_X, Lambda_X) and (mu_W, Lambda_W) with tau fixed
 * (Section 5.1).  The Gibbs sweep draws the hyperparameters, then every x_n given W, then every
 * w_d given X.  PP (Section 3.2, Algorithm 1) splits the rows into I and the columns into J
 * blocks; stage 1 samples subset (0,0), stage 2 the subsets sharing its rows or columns with
 * the stage-1 posterior as prior, stage 3 the rest with the stage-2 posteriors as priors; each
 * subset posterior is summarised per row by moment matching (Section 4.1) and the summaries
 * are combined by Eq. 14 with the eigenvalue correction of Algorithm 2.
 *
 * Conventions (the paper does not fix them; the library and any checker follow these):
 *  - Gaussian draws: precision P = L L^T (lower Cholesky, positive diagonal), x = mu + L^{-T} z.
 *  - Wishart(W, nu) draws: Bartlett decomposition on the lower Cholesky L of W:
 *    Lambda = (L A)(L A)^T, A lower triangular, A_kk = sqrt(c_k), c_k ~ chi^2(nu - k)
 *    (k = 0..K-1), A_kl ~ N(0,1) for k > l.
 *  - Hyperparameter posterior: centred scatter matrix (Section 5.1 footnote):
 *    [W*]^{-1} = W0^{-1} + N Sbar + (beta0 N / (beta0 + N)) (mu0 - xbar)(mu0 - xbar)^T,
 *    beta* = beta0 + N, nu* = nu0 + N, mu* = (beta0 mu0 + N xbar) / beta*;
 *    mu ~ N(mu*, (beta* Lambda)^{-1}).
 *  - Sweep order: (mu_X, Lambda_X) | X, (mu_W, Lambda_W) | W, then X | W, then W | X, then
 *    (sampled noise) the noise precisions | X, W: tau_d ~ Gamma(a0 + n_d / 2, b0 + SSE_d / 2)
 *    with SSE_d the squared residuals of column d's entries (one precision: the subset's
 *    entries and summed SSE), drawn as c / (2 b0 + SSE) from a chi-square variate c.  The row
 *    conditionals weight entry (n, d) by tau_d, the column conditional of w_d takes tau_d.
 *  - Ordering (Section 5.2): BMF_ORDER_DECREASING sorts rows (columns) by decreasing number
 *    of training observations, ties by original index; row_bounds/col_bounds are given in
 *    that order.  Subset (i, j) (0-based) has id s = i*J + j and stage 1 if i = j = 0,
 *    stage 2 if exactly one of i, j is 0, stage 3 otherwise.
 *  - Propagated priors (Algorithm 1, Section 5.1): in stage 2, subset (i,0) uses the stage-1
 *    posterior of W^(0) and draws hyperparameters for X^(i); subset (0,j) uses the stage-1
 *    posterior of X^(0) and draws hyperparameters for W^(j).  In stage 3, subset (i,j) uses
 *    the posterior of X^(i) from (i,0) and of W^(j) from (0,j) and draws no hyperparameters.
 *    A propagated factor starts its chain at the propagated mean.
 *  - Moment matching: over the retained samples (sweep t, counted from 1 within a subset's
 *    chain, is retained when t > burnin and (t - burnin - 1) % thin == 0):
 *    mu = mean, Sigma = E[x x^T] - mu mu^T (1/S normaliser), Lambda = Sigma^{-1}.  It needs
 *    S >= K + 1 retained samples (a full-rank Sigma); fewer fail with BMF_E_STATE.
 *  - Dominant-mode and mixture summaries (Section 4.1, PP DM / PP GMM; summary != MM): the
 *    retained samples of each row are clustered by lambda-means (one cluster at the first
 *    sample; each round visits the samples in order and gives each to the nearest centre,
 *    lowest index on ties, unless every squared distance exceeds lambda, when it opens a
 *    cluster at itself; centres then move to their means and empty clusters are dropped; until
 *    no assignment changes, at most 100 rounds).  DM fits one Gaussian (mean, inverse of the 1/n
 *    covariance) to the largest cluster; GMM one to each of the C largest clusters with at
 *    least K + 1 samples (ties: lowest index), weights by size.  A row without such a cluster
 *    takes one Gaussian over all samples.  DM propagates and aggregates its Gaussian; GMM
 *    propagates the mixture (before each draw of a row the component with the largest
 *    pi_c N(x; mu_c, Lambda_c^{-1}) at the row's current value is its prior; its chain starts at
 *    the mixture mean) and aggregates the pooled moments, mean and inverse of
 *    sum_c pi_c (Lambda_c^{-1} + (mu_c - m)(mu_c - m)^T).
 *  - Aggregation (Eq. 14, Algorithm 2): for X^(i) submodel "(1)" is subset (i,0) and the
 *    others are (i,j), j >= 1; for W^(j) it is (0,j) and (i,j), i >= 1.  A difference
 *    Lambda^(j) - Lambda^(1) that is not positive definite (FP64 Cholesky pivot <= 0) gets
 *    |lambda_min| + eps added to its diagonal, eps = eps_rel * max(1, mean diag Lambda^(1)).
 *  - Prediction (Section 5.2): y_hat = offset + mu*_x^T mu*_w with the aggregated posterior
 *    means (for a 1 x 1 grid: the means of the retained samples); offset is the training mean
 *    when cfg.center = 1, else 0.
 *
 * Draw buffers (bmf_draws): for each sweep of a batch (the subsets of one stage, or one
 * subset), in this order:
 *    for each subset of the batch in id order: an X block then a W block of K(K+3)/2 numbers
 *      each: c[K] (chi-square variates, dof nu0 + n - k for k = 0..K-1, where n is the number
 *      of rows of that factor block in the subset), the K(K-1)/2 below-diagonal normals row by
 *      row (k = 1..K-1, l = 0..k-1), z_mu[K].  The block of a propagated factor is present and
 *      ignored.
 *    then z for every X row of the batch (subsets in id order, rows in local order), K each;
 *    then z for every W row of the batch, K each;
 *    then (sampled noise) for each subset in id order its noise chi-square variates: one per
 *      column in local order with dof 2 a0 + the column's entries in the subset, or one with
 *      dof 2 a0 + the subset's entries.
 *  Consecutive sweeps follow each other.
 *
 * Device generator (draws == NULL).  The library then computes the same buffer on the GPU from
 * the counter-based generator Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key
 * (cfg.seed, 0) and counter (index, t, tag, attempt), where t is the 1-based sweep number of
 * the subset's chain and tag = subset id * 256 + factor (0 = X, 1 = W) * 16 + kind:
 *    kind 3, z of a factor block: element r K + k (local row r) is element e of a normal
 *      stream; kind 2, the K(K-1)/2 + K normals of a hyperparameter block, likewise.  Element
 *      e of a normal stream comes from call (e / 4, t, tag, 0): words 0, 1 give elements 4q,
 *      4q + 1 and words 2, 3 elements 4q + 2, 4q + 3 by Box-Muller, r cos(2 pi u2) and
 *      r sin(2 pi u2) with r = sqrt(-2 ln u1), u1 = ((w >> 11) + 1) 2^-53, u2 = (w >> 11) 2^-53;
 *    kind 1, chi-square variate k of a block: 2 Gamma(dof / 2) by Marsaglia & Tsang (ACM TOMS
 *      2000), attempt j on counter (k, t, tag, j) with the candidate normal from words 0, 1
 *      (cosine), the acceptance uniform u1 of word 2 and, when dof < 2, the factor
 *      U^(2 / dof) with U = u1 of word 3 (the shape-below-one boost).  64 rejections in a row
 *      fail the call with BMF_E_CUDA (probability below 1e-80);
 *    kind 4, noise chi-square variate k of a subset (factor W): drawn the same way with the
 *      dof of the layout above.
 *  The numbers depend only on (seed, subset, factor, t, position): batching a stage or
 *  splitting sweeps across calls does not change them.  bmf_generate_draws returns them.
 *
 * Memory and errors.  The context owns all device memory it allocates.  Host pointers passed
 * in are read during the call only; the caller keeps ownership.  Every call is synchronous
 * with respect to the host unless stated.  Calls return a bmf_status; nothing aborts or traps
 * on the device.  bmf_last_error() gives a message for the last failed call.  A context must
 * be used from one host thread at a time.
 */
#ifndef BMF_H
#define BMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmf_ctx bmf_ctx;

typedef enum {
    BMF_OK = 0,
    BMF_E_ARG = 1,       /* null pointer, index or size out of range, duplicate entry */
    BMF_E_SHAPE = 2,     /* inconsistent sizes (bounds, draw buffer length, K) */
    BMF_E_NOT_PD = 3,    /* a conditional precision or moment-matched covariance is not PD */
    BMF_E_NONFINITE = 4, /* NaN or Inf in an input value */
    BMF_E_TIMEOUT = 5,   /* a bounded device wait expired */
    BMF_E_OOM = 6,       /* device allocation failed */
    BMF_E_CUDA = 7,      /* CUDA runtime error */
    BMF_E_STATE = 8      /* call not valid now (e.g. stage 2 before stage 1) */
} bmf_status;

/* Precision of the gathered factor copies and of the Gram accumulation.  The conditional
 * assembly, Cholesky, solves, draws, hyperparameter step and moments are FP64 in all modes.
 * FP32 gathers at K > 16 reach the tensor cores as split TF32 (three products per tile, close to
 * FP32 products); BMF_TF32 keeps FP32 gathers but takes one TF32 product per tile (operands
 * rounded to 10-bit mantissas) at K > 16, and is BMF_FP32 at K <= 16. */
enum { BMF_FP64 = 0, BMF_FP32 = 1, BMF_BF16 = 2, BMF_TF32 = 3 };
enum { BMF_ORDER_NONE = 0, BMF_ORDER_DECREASING = 1 };
enum { BMF_FACTOR_X = 0, BMF_FACTOR_W = 1 };

#define BMF_MAX_K 64

typedef struct {
    int32_t K;         /* latent dimension, 1..BMF_MAX_K */
    int32_t precision; /* BMF_FP64 / BMF_FP32 / BMF_BF16 / BMF_TF32 */
    double tau;        /* noise precision (Eq. 3), > 0 */
    double beta0;      /* Normal-Wishart beta0 > 0 */
    double nu0;        /* Normal-Wishart nu0 > K - 1 */
    const double *mu0; /* host [K], or NULL for zeros */
    const double *W0;  /* host [K*K] symmetric positive definite, or NULL for the identity */
    int32_t order;     /* BMF_ORDER_NONE / BMF_ORDER_DECREASING */
    int32_t center;    /* 1: subtract the training mean from the values (added back in y_hat) */
    int32_t burnin;    /* sweeps discarded per chain before moments are accumulated */
    int32_t thin;      /* keep every thin-th sweep after burn-in (>= 1) */
    uint64_t seed;     /* device generator seed (used when draws == NULL) */
    double eps_rel;    /* Algorithm 2 epsilon scale (<= 0: 1e-6) */
    int32_t moments;   /* BMF_MOMENTS_AUTO: second moments (for moment matching) only when the
                          grid has more than one subset; BMF_MOMENTS_MEAN: sums of x only (enough
                          for posterior-mean prediction); BMF_MOMENTS_FULL: sums of x and x x^T */
    int32_t summary;   /* subset-posterior summary propagated between stages and aggregated
                          (Section 4.1): BMF_SUMMARY_MM moment matching (default),
                          BMF_SUMMARY_DM dominant mode, BMF_SUMMARY_GMM mixture of modes */
    int32_t components; /* GMM: largest clusters kept, 1..BMF_MAX_COMPONENTS (0: 3) */
    double lambda;     /* DM / GMM: lambda-means penalty on the squared distance (> 0) */
    int32_t max_samples; /* DM / GMM: retained samples kept per chain (a ring of max_samples x
                          K doubles per factor row); a call that would retain more fails with
                          BMF_E_STATE */
    int32_t independent; /* 1: no propagation -- every subset keeps the standard priors with its
                          own hyperparameter draws and its chain starts at the initial state
                          (the embarrassingly parallel MCMC baseline of Section 5.4, used by the
                          subset-posterior correlations of Section 5.6); 0: Algorithm 1 */
    int32_t noise;     /* noise precision (Section 2.1): BMF_NOISE_FIXED tau (default);
                          BMF_NOISE_GLOBAL one precision per chain, BMF_NOISE_COLUMN one per column
                          (tau_d), sampled after each sweep's W half from Gamma(a0, b0) priors
                          (shape, rate); every chain starts at tau */
    double noise_a0, noise_b0; /* the Gamma prior of a sampled precision (both > 0) */
} bmf_config;

enum { BMF_MOMENTS_AUTO = 0, BMF_MOMENTS_MEAN = 1, BMF_MOMENTS_FULL = 2 };
enum { BMF_SUMMARY_MM = 0, BMF_SUMMARY_DM = 1, BMF_SUMMARY_GMM = 2 };
enum { BMF_NOISE_FIXED = 0, BMF_NOISE_GLOBAL = 1, BMF_NOISE_COLUMN = 2 };
#define BMF_MAX_COMPONENTS 4

typedef struct {
    const double *ptr; /* draw buffer (layout above), FP64 */
    int64_t len;       /* number of doubles; must equal n_sweeps * bmf_draws_per_sweep() */
    int32_t on_device; /* 1: ptr is device memory of the context's GPU; 0: host memory */
} bmf_draws;

typedef struct {
    double rmse_sample; /* test RMSE of the last sweep's sample (NaN without a test set) */
    double rmse_mean;   /* test RMSE of the mean prediction over retained samples (NaN if none) */
    int64_t sweeps;     /* sweeps done by the batch's chains (of the first subset) */
    int64_t kept;       /* retained samples so far (of the first subset) */
} bmf_sweep_stats;

typedef struct {
    int32_t i, j, stage;
    int64_t row0, row1; /* row block [row0, row1) in the reordered row order */
    int64_t col0, col1;
    int64_t nnz;
} bmf_subset_info;

/* Create a context: validates the COO training data (indices in range, no duplicate (row,col),
 * finite values), reorders (cfg->order), splits it into the I x J grid (Section 3), builds the
 * per-subset CSR (rows) and CSC (columns) lists and uploads them, and initialises every
 * subset's chain from X0/W0init.
 *   row, col, val: host COO of the training entries, nnz each, 0-based original indices.
 *   row_bounds: host [I+1] increasing from 0 to N in the reordered order, or NULL for
 *     floor(i*N/I); col_bounds likewise with J and D.
 *   X0 [N*K], W0init [D*K]: host initial states in the ORIGINAL index order (row-major).
 *   test_row/test_col/test_val: host COO of held-out entries for the per-sweep RMSE
 *     (n_test may be 0 and the pointers NULL).
 *   stream: a cudaStream_t the context enqueues on (NULL: the legacy default stream).
 * On success *out owns the context; free it with bmf_destroy. */
bmf_status bmf_init(bmf_ctx **out, const bmf_config *cfg, int64_t N, int64_t D, int64_t nnz,
                    const int32_t *row, const int32_t *col, const double *val, int32_t I,
                    const int64_t *row_bounds, int32_t J, const int64_t *col_bounds,
                    const double *X0, const double *W0init, int64_t n_test,
                    const int32_t *test_row, const int32_t *test_col, const double *test_val,
                    void *stream);

/* Host-only preprocessing, exactly as bmf_init performs it, without a GPU or any device memory
 * (to check a data set and its grid before creating a context): validates the COO training data
 * (indices in range, no duplicate (row, col), finite values), orders rows and columns
 * (order = BMF_ORDER_NONE or BMF_ORDER_DECREASING, Section 5.2) and cuts the I x J grid
 * (row_bounds / col_bounds as for bmf_init, NULL for equal cuts).  Outputs, host, nullable:
 *   row_perm [N], col_perm [D]: original index at each reordered position;
 *   row_bounds_out [I+1], col_bounds_out [J+1]: the cuts in the reordered order;
 *   subset_nnz [I*J]: training entries of subset s = i*J + j.
 * Errors as bmf_init (BMF_E_ARG, BMF_E_SHAPE, BMF_E_NONFINITE), message via bmf_last_error(NULL). */
bmf_status bmf_plan(int64_t N, int64_t D, int64_t nnz, const int32_t *row, const int32_t *col,
                    const double *val, int32_t order, int32_t I, const int64_t *row_bounds,
                    int32_t J, const int64_t *col_bounds, int64_t *row_perm, int64_t *col_perm,
                    int64_t *row_bounds_out, int64_t *col_bounds_out, int64_t *subset_nnz);

/* Number of doubles of one sweep's draw buffer for a batch: the subsets of `stage` (1..3)
 * when subset < 0, else the single subset `subset`. */
int64_t bmf_draws_per_sweep(const bmf_ctx *ctx, int32_t stage, int32_t subset);

/* The device generator's draws (draws == NULL above) of sweeps t0 .. t0 + n_sweeps - 1 (t0 >= 1)
 * of a batch: the subsets of `stage` when subset < 0, else the single subset `subset`, in the
 * draw-buffer layout.  out: n_sweeps * bmf_draws_per_sweep() doubles, host memory
 * (out_on_device = 0) or device memory of the context's GPU (1).  The chains are unchanged. */
bmf_status bmf_generate_draws(bmf_ctx *ctx, int32_t stage, int32_t subset, int64_t t0,
                              int32_t n_sweeps, double *out, int32_t out_on_device);

/* Launch schedule of the sweeps (no counterpart in the paper; the sampled values do not depend
 * on it).  chunks_x / chunks_w (1..BMF_MAX_CHUNKS): the rows of the X (W) half of a batch are
 * split at conditional-block boundaries into this many chunks of about equal estimated cost
 * (observations + row_weight x rows); each chunk's Gram pass runs on the context stream, the
 * lightest rows first, and its conditional draw on a second stream as soon as that pass is
 * done, so that the FP64 conditional of one chunk overlaps the Gram pass of the next (1: one
 * Gram launch, then one conditional launch).  gram_blocks_per_sm (1..64): grid of a Gram
 * launch = SMs x this.  row_weight (>= 0): cost of a row in observations for the split; 0
 * selects a default from K and the precision.  Default {1, 1, 4, 0, 0, 0}. */
#define BMF_MAX_CHUNKS 8
typedef struct {
    int32_t chunks_x, chunks_w;
    int32_t gram_blocks_per_sm;
    double row_weight;
    int32_t graph;     /* 1: capture each call's launch sequence into one CUDA graph and launch it
                          once (kept and updated in place across calls of the same shape); 0: launch
                          directly.  Ignored while profiling is on, and for a call given host
                          draws: their copy then runs in groups of sweeps beside the sweeps,
                          each sweep waiting only for its own group. */
    int32_t cond_lanes; /* K >= 13: lanes that factor one row in the FP64 conditional draw (2, 4,
                          8, 16 or 32; every choice gives bit-identical values; 2, only for
                          K <= 16, keeps the row's matrix in registers; a team of 4 to 32 lanes
                          keeps it in shared memory, and bmf_set_schedule rejects a team whose
                          rows do not fit there, BMF_E_ARG); 0: a default from K (2 up to
                          K = 16, 16 up to 48, 32 above).  Ignored for K <= 12 (one thread per
                          row). */
} bmf_schedule;
bmf_status bmf_set_schedule(bmf_ctx *ctx, const bmf_schedule *sched);
bmf_status bmf_get_schedule(const bmf_ctx *ctx, bmf_schedule *sched);

/* Per-sweep test-RMSE monitor (no counterpart in the paper, whose PP evaluates the final
 * aggregated prediction only): with on = 1 (the default) every sweep predicts the held-out
 * entries of its batch with the current sample and with the running mean of the retained
 * samples, and bmf_sweep / bmf_stage report both RMSEs in bmf_sweep_stats; with on = 0 that pass
 * is skipped, the two RMSE fields are NaN, and the running mean stops accumulating (turn it off
 * for a whole run).  The sampled values do not depend on it; bmf_test_rmse and bmf_predict do
 * not use it. */
bmf_status bmf_set_monitor(bmf_ctx *ctx, int32_t on);

/* Schedule tuner: on the batch of `stage` (subset < 0) or of one subset, times candidate
 * schedules -- Gram grid 2/4/8 blocks per SM, then 1-4 row chunks for each half, then the split
 * weight, then (K >= 13) 2/4/8 (K <= 16) or 8/16/32 lanes per row of the conditional, those that
 * fit, then the CUDA-graph launch --
 * with one untimed and sweeps_per_trial timed sweeps each (device generator), and installs the
 * fastest.  Every trial starts from the same state and the
 * chains are restored afterwards (state, gathered copies, moment sums, hyperparameters, running
 * test predictions, sweep counters), so the call changes no sampled value.  The batch's stage
 * must be open.  best: host, nullable. */
bmf_status bmf_autotune(bmf_ctx *ctx, int32_t stage, int32_t subset, int32_t sweeps_per_trial,
                        bmf_schedule *best);

/* n_sweeps Gibbs sweeps of one subset's chain (the whole data for a 1 x 1 grid).  One sweep is
 * the BPMF Gibbs sampler of Section 5.1 (Salakhutdinov & Mnih's sampler, which the paper runs in
 * every subset of Algorithm 1): the Normal-Wishart hyperparameters of X and of W given the
 * current factors (centred scatter of the Section 5.1 footnote), then every row x_n given W
 * (Eqs. 2-4 with the rows' priors), then every row w_d given the new X, then, with a sampled
 * noise precision, tau given X and W (Section 2.1); the order and conventions are those at the
 * top of this header.  The subset's stage must be open (see bmf_stage).  draws: NULL for the
 * device generator, else the buffer for n_sweeps sweeps of this single-subset batch.  stats may
 * be NULL.  Errors: BMF_E_ARG for a bad subset or n_sweeps < 0, BMF_E_STATE when the stage is
 * not open or the context failed earlier,
 * BMF_E_SHAPE for a draw buffer of the wrong length, BMF_E_NOT_PD when a conditional precision
 * is not positive definite (the chain must then be reset with bmf_set_state or bmf_restart),
 * BMF_E_CUDA for a runtime error or a device-generator rejection run. */
bmf_status bmf_sweep(bmf_ctx *ctx, int32_t subset, int32_t n_sweeps, const bmf_draws *draws,
                     bmf_sweep_stats *stats);

/* n_sweeps Gibbs sweeps of every subset of `stage` (Algorithm 1), all subsets of the stage
 * batched into the same kernel launches.  The first call for stage 2 (3) finalises the moments
 * of stage 1 (2) and installs the propagated priors; stages are opened in order and a stage
 * may be called several times to continue its chains. */
bmf_status bmf_stage(bmf_ctx *ctx, int32_t stage, int32_t n_sweeps, const bmf_draws *draws,
                     bmf_sweep_stats *stats);

/* Posterior-mean predictions (Section 5.2) for n entries given by original indices (host
 * arrays).  Finalises the moments of the open stage and aggregates (Eq. 14, Algorithm 2).
 * yhat: host [n] or NULL; y: host [n] or NULL; rmse: RMSE against y (needs y) or NULL. */
bmf_status bmf_predict(bmf_ctx *ctx, int64_t n, const int32_t *row, const int32_t *col,
                       const double *y, double *yhat, double *rmse);

/* Test RMSE of the posterior-mean prediction (Section 5.2) of the held-out entries given to
 * bmf_init, computed on the device: finalises the moments of the open stage, aggregates (Eq. 14,
 * Algorithm 2; for a 1 x 1 grid the means of the retained samples) and predicts every held-out
 * entry; only the RMSE is read back.  NaN without held-out entries.  Needs every stage run
 * (BMF_E_STATE otherwise). */
bmf_status bmf_test_rmse(bmf_ctx *ctx, double *rmse);

/* Start a new run of Algorithm 1 on the same data and grid (no counterpart in the paper: a
 * context reuses its preprocessed observation lists across independent runs).  Every subset's
 * chain returns to the initial state: X0 [N*K] and W0init [D*K], host, ORIGINAL order, each
 * replacing the stored initial state, or NULL to reuse the stored one (the one given to bmf_init
 * or to the last bmf_restart).  Moment sums, running test predictions, hyperparameter draws,
 * propagated priors and sweep counters are cleared, stage 1 is open again, and the device
 * generator takes `seed`.  The launch schedule is kept.  Errors: BMF_E_NONFINITE (non-finite
 * initial state; nothing changed), BMF_E_CUDA. */
bmf_status bmf_restart(bmf_ctx *ctx, const double *X0, const double *W0init, uint64_t seed);

/* Aggregated posterior means (Eq. 14 / Algorithm 2) in the ORIGINAL order: Xm [N*K],
 * Wm [D*K] host; n_corrected (nullable) counts eigenvalue-corrected (row, submodel) pairs. */
bmf_status bmf_posterior_means(bmf_ctx *ctx, double *Xm, double *Wm, int64_t *n_corrected);

/* Chain state of one subset to / from host memory, in the subset's local (reordered) order:
 * X [n_rows*K], W [n_cols*K], hyper = mu_X[K], Lambda_X[K*K], mu_W[K], Lambda_W[K*K]
 * (the last hyperparameter draw).  Any pointer may be NULL to skip that part. */
bmf_status bmf_get_state(bmf_ctx *ctx, int32_t subset, double *X, double *W, double *hyper);
bmf_status bmf_set_state(bmf_ctx *ctx, int32_t subset, const double *X, const double *W);

/* Moment sums of one subset: S1 [n*K], S2 [n*K*K] for factor BMF_FACTOR_X / _W, and the
 * number of retained samples.  S2 needs second moments (BMF_E_STATE otherwise). */
bmf_status bmf_get_moments(bmf_ctx *ctx, int32_t subset, int32_t factor, double *S1, double *S2,
                           int64_t *kept);

/* Per-row summary of one subset's factor posterior (mu [n*K], Lambda [n*K*K]) as propagated to
 * the next stage and aggregated: moment matched (needs second moments; BMF_E_STATE otherwise),
 * the dominant mode (DM) or the mixture's pooled moments (GMM). */
bmf_status bmf_get_posterior(bmf_ctx *ctx, int32_t subset, int32_t factor, double *mu,
                             double *Lam);

/* Install a per-row Gaussian prior (mu [n*K], Lambda [n*K*K], host) on one subset's factor,
 * replacing its hyperparameter draws (as a propagated prior does). */
bmf_status bmf_set_prior(bmf_ctx *ctx, int32_t subset, int32_t factor, const double *mu,
                         const double *Lam);

/* Current noise precision of each column of one subset's chain, tau [n_cols] host (the fixed
 * tau when the noise is not sampled). */
bmf_status bmf_get_noise(bmf_ctx *ctx, int32_t subset, double *tau);

/* Grid geometry of one subset, and the reordering (new -> original index) of rows/columns. */
bmf_status bmf_get_subset_info(const bmf_ctx *ctx, int32_t subset, bmf_subset_info *info);
bmf_status bmf_get_perm(const bmf_ctx *ctx, int64_t *row_perm, int64_t *col_perm);

/* Adjoint of the masked log-joint of one subset (a project addition; the paper samples with
 * Gibbs only):
 *   l = -(a/2) sum_{Omega} (y - x_n^T w_d)^2 + (|Omega|/2) log a
 *       - 1/2 sum_n (x_n - mu_n)^T L_n (x_n - mu_n) - 1/2 sum_d (w_d - mu_d)^T L_d (w_d - mu_d),
 * a = exp(log_alpha), (mu, L) the rows' current priors in the subset (its last hyperparameter
 * draw, or the propagated per-row Gaussians); y are the centred training values.  The value is
 * returned up to an additive constant (the terms mu^T L mu are dropped).
 *   X: device [n_rows x ld], W: device [n_cols x ld], FP32, in the subset's local (reordered)
 *      order, 16-byte aligned, ld >= K and ld % 4 == 0 (padding is ignored);
 *   gX, gW: device, same layouts (padding written as 0); value, g_log_alpha: host, nullable.
 * FP32 arithmetic with FP64 scalar sums; deterministic.  1 <= K <= 64. */
bmf_status bmf_logjoint_grad(bmf_ctx *ctx, int32_t subset, const float *X, const float *W,
                             int64_t ld, double log_alpha, float *gX, float *gW,
                             double *g_log_alpha, double *value);

/* n_steps Langevin moves on caller-owned FP32 factors (layouts as in bmf_logjoint_grad), beside
 * the Gibbs sweep: theta' = theta + (eps/2) grad l(theta) + sqrt(eps) xi.  With uniforms == NULL
 * every proposal is taken (unadjusted Langevin); otherwise a Metropolis-Hastings test with the
 * host uniforms[n_steps] accepts or rejects each proposal (MALA).
 *   noise: device FP32 [n_steps][(n_rows + n_cols) * K] standard normals (X rows then W rows);
 *   accepted: host, nullable (number of accepted proposals); value: host, nullable (log-joint
 *   at the final state). */
bmf_status bmf_langevin(bmf_ctx *ctx, int32_t subset, int32_t n_steps, float *X, float *W,
                        int64_t ld, double log_alpha, double eps, const float *noise,
                        const double *uniforms, int32_t *accepted, double *value);

/* Tracing.  With profiling on, bmf_sweep / bmf_stage record a pair of CUDA events on the
 * context stream around every kernel launch and accumulate the elapsed time per kernel class
 * ("stats", "hyper", "gram_x", "cond_x", "gram_w", "cond_w", "rmse").  bmf_profile_read copies
 * up to `max` entries into `out`, returns how many classes there are and resets the totals.
 * bmf_launch_count returns the number of kernels this context has launched since bmf_init. */
typedef struct {
    char name[16];
    int64_t launches;
    double total_ms;
} bmf_kernel_time;
bmf_status bmf_profile_enable(bmf_ctx *ctx, int32_t on);
int32_t bmf_profile_read(bmf_ctx *ctx, bmf_kernel_time *out, int32_t max);
int64_t bmf_launch_count(const bmf_ctx *ctx);

void bmf_destroy(bmf_ctx *ctx);

/* Aggregation without allocating (no counterpart in the paper: a deployment addition).
 * Some callers cannot let a library call cudaMalloc: a runtime that owns all device memory
 * through its own pool allocator, or a service that must not grow its device footprint after
 * start-up.  This call combines, for R rows, the per-row Gaussians of J submodels by Eq. 14 with
 * the eigenvalue correction of Algorithm 2 (the same operation bmf_posterior_means applies to a
 * context's moment-matched subset posteriors) and allocates nothing: its per-row working
 * matrices live in a static device array of BMF_AGGREGATE_STATIC_MAX_DOUBLES doubles (32 MiB)
 * that every GPU loading this library holds until the process exits.
 *   mu:  device [J][R][K], Lam: device [J][R][K][K] (full symmetric precisions); submodel 0 is
 *        the one whose posterior was propagated to the others;
 *   mu_star: device [R][K] output; n_corrected: host, nullable (corrected (row, j) pairs);
 *   eps_rel as in bmf_config (<= 0: 1e-6); stream: cudaStream_t or NULL.
 * Limits: 1 <= K <= 16, J >= 1, R * K * K <= BMF_AGGREGATE_STATIC_MAX_DOUBLES (else
 * BMF_E_SHAPE; split the rows over several calls).  Returns BMF_E_NOT_PD if an aggregated
 * precision is not positive definite.  The call reads two counters back and waits for its
 * stream before returning.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it; calls after a cudaDeviceReset of that device are not
 * supported.  All calls share the array (each call clears its counters first); calls that
 * overlap on the GPU race on it.  Errors are reported by bmf_last_error(NULL). */
#define BMF_AGGREGATE_STATIC_MAX_DOUBLES 4194272
bmf_status bmf_aggregate_static(int32_t K, int64_t R, int32_t J, const double *mu,
                                const double *Lam, double eps_rel, double *mu_star,
                                int64_t *n_corrected, void *stream);

/* The summaries of the convention above for R rows of S samples each, without a context
 * (Section 4.1): samples device [S][R][K]; mode 0 one Gaussian over all samples, 1 dominant
 * mode, 2 mixture of the C largest modes (1 <= C <= BMF_MAX_COMPONENTS); lambda > 0 the
 * lambda-means penalty.  Outputs, device, indexed by row: pi [R][C] (0 for unused components),
 * mu [R][C][K], Lam [R][C][K][K], pooled_mu [R][K], pooled_Lam [R][K][K] (the mixture's
 * pooled mean and precision), assign [R][S] (cluster of each sample; nullable).  Limits:
 * 1 <= K <= 32, S >= 1, S * K <= 8192.  BMF_E_NOT_PD if a row's covariance is singular.  The
 * call waits for its stream; errors via bmf_last_error(NULL). */
bmf_status bmf_fit_summaries(int32_t K, int64_t R, int32_t S, const double *samples, int32_t mode,
                             int32_t C, double lambda, double *pi, double *mu, double *Lam,
                             double *pooled_mu, double *pooled_Lam, int32_t *assign, void *stream);

/* Message of the last failed call on ctx; with ctx NULL, of the last failed call of this thread
 * that takes no context (bmf_init, bmf_plan, bmf_aggregate_static, bmf_fit_summaries). */
const char *bmf_last_error(const bmf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BMF_H */
