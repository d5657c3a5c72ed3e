// kernels.h -- launchers of the library's CUDA kernels (internal).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "common.cuh"

namespace bmf {

// Template width of the latent dimension: K rounded up to an even number (the padded
// dimensions carry zeros in the gathered copies and an identity block in the conditional,
// which leaves the first K components bit-identical to an unpadded computation).
int padded_k(int K);
// Elements per row of a gathered factor copy (K padded, row = multiple of 16 bytes).
int gather_ld(int K, int prec);
// Gram entries per work item in the partial buffer.
int gram_part_ld(int K, int prec);

// Lanes per row of the Gram-gather pass for a row of `count` observations.
int gram_group(int64_t count);

struct GramParams {
    int K;                     // latent dimension (used by the K > 16 kernels)
    const GramTask *tasks;
    int64_t n_tasks;
    const GramItem *items;     // items of the launch: absolute item i at items[i - item0]
    int64_t n_items;
    const int32_t *idx;   // observation partner index (arena row of the partner factor)
    const void *val;      // observation values (double for FP64, float otherwise)
    const void *P;        // gathered partner copy [rows x ldP]
    int ldP;
    void *part;           // partial Gram per item [n_items x ld] (double for FP64, float else)
    int ld;
    // rows split over several items (see gram.cu)
    const int32_t *multi_idx;  // [R] slot of a multi-item row, else -1
    const int64_t *item_ptr;   // [R+1] absolute item index of each row
    int64_t item0;             // absolute index of items[0]
    int *counters;             // [slots x nparts], zero between launches
    int nparts;
    double *rowsum;            // [slots x ld_sum]
    int ld_sum;
    int nv;                    // entries per partial
};
void launch_gram(int K, int prec, const GramParams &a, int grid, cudaStream_t st);
int gram_parts(int K, int prec);

// A block of the conditional kernel: up to 64 consecutive arena rows of one subset.
struct CondBlock {
    int64_t row0;
    int32_t n;
    int32_t pad;
};

struct CondParams {
    int K;
    const CondBlock *blocks;     // this launch's blocks (one CUDA block each)
    int64_t blk0;                // absolute index of blocks[0] (stats partial slot)
    int64_t row0, row1;          // arena rows of this launch
    const int64_t *item_ptr;     // [R+1] first work item of each arena row
    int64_t item0;               // item index of part[0]
    const void *part;            // Gram partials (see GramParams)
    int ld;
    int part_rhs;                // offset of the right-hand side within a partial
    const int32_t *multi_idx;    // [R] slot in rowsum of a row with >= 2 items, else -1
    const double *rowsum;        // FP64 sums of multi-item rows [slots x ld_sum]
    int ld_sum;
    double tau;
    const double *tau_row;       // [R] per-row noise precision (sampled per column), or null
    const int32_t *row_hslot;    // [R] hyper slot of the row, or -1 for a per-row prior
    const double *hyper;         // [slots x hyper_slot_len(K)]
    const double *prior_L;       // per-row priors, SoA: [ntri(K)][R]
    const double *prior_b;       // [K][R] (Lambda mu)
    int64_t R;                   // arena rows (SoA stride)
    const double *z;             // standard normals of this launch's rows, [row1-row0][K]
    double *X;                   // FP64 state [R x K]
    void *Xg;                    // gathered copy [R x ldg]
    int ldg;
    int keep;                    // accumulate moments
    int full;                    // also second moments
    double *S1;                  // SoA [K][R]
    double *S2;                  // SoA [ntri(K)][R]
    double *stats;               // per-block sums of x and x x^T of the new state
                                 // [blocks x (K + ntri(K))], at slot blk0 + blockIdx.x
    DevError *err;
    // rows marked kFusedRow in multi_idx form their own Gram sums from their observations (in
    // list order), which the Gram pass skips: the row's list and the gathered partner copy
    const int64_t *obs_ptr;      // [R+1]
    const int32_t *obs_idx;      // partner arena rows
    const void *obs_val;         // values (double for FP64, float otherwise)
    const void *P;               // gathered partner copy [rows x ldP]
    int ldP;
};
void launch_cond(int prec, const CondParams &a, int n_blocks, cudaStream_t st);
// multi_idx of a row whose Gram sums the conditional draw forms itself: 13 <= K <= 16 (the
// two-lane and team conditionals) and 1 to kFuseMaxObs observations in one work item.  Such a
// row's partner rows are few and mostly cached, where its Gram partials would be a round trip
// through memory.  Measured on the 100k x 20k, K = 16 PP workload (FP32, 3 x 60 sweeps with
// resident draws): 237.1 ms without fusion, 225.6 / 215.2 / 209.7 / 204.9 / 205.4 / 226.3 ms
// with at most 8 / 16 / 32 / 64 / 128 / 512 observations fused.
constexpr int32_t kFusedRow = -2;
constexpr int kFuseMaxObs = 64;
constexpr int kCondBlock = 64;

// Per-chunk sums for the hyperparameter step: for each chunk, sum x and the packed lower
// sum x x^T over rows [r0, r1) of an FP64 arena.
struct StatChunk {
    int64_t r0, r1;
    int32_t out;      // output slot (chunk index)
    int32_t arena;    // 0 = X arena, 1 = W arena
};
void launch_stats(int K, const StatChunk *chunks, int n_chunks, const double *X, const double *W,
                  double *out, cudaStream_t st);

// Normal-Wishart posterior and draw for a list of (chunk range -> hyper slot) jobs.
struct HyperJob {
    int32_t chunk0, chunk1;  // stats chunks to sum
    int32_t slot;            // output hyper slot
    int32_t draw;            // offset of the draw block (doubles) in the sweep's draw buffer
    int64_t n;               // rows of the factor block
};
struct HyperParams {
    int K;
    const HyperJob *jobs;
    int n_jobs;
    const double *stats;     // [chunks x (K + ntri)]
    const double *mu0;       // [K]
    double beta0, nu0;
    const double *W0inv;     // [K*K]
    const double *draws;     // the sweep's draw buffer
    double *hyper;           // [slots x hyper_slot_len]
    DevError *err;
};
void launch_hyper(const HyperParams &a, cudaStream_t st);
// First level of the statistics sum: partials (j0 + j) * kStatParts + p of job j (see misc.cu).
constexpr int kStatParts = 64;
void launch_stats_reduce(int K, const HyperJob *jobs, int n_jobs, int j0, const double *stats,
                         double *out, cudaStream_t st);

// Test-set predictions of the current sample, running mean, squared errors.
struct RmseParams {
    int K, prec;
    int64_t t0, t1;          // test arena range
    const int32_t *trow, *tcol;
    const double *tval;
    const void *Xg, *Wg;
    int ldg;
    int keep;
    double *ysum;            // running sum of predictions over kept samples
    double inv_kept;         // 1 / (kept samples after this sweep), 0 when none (no mean)
    double *partial;         // [blocks x 2]
};
void launch_rmse(const RmseParams &a, int blocks, cudaStream_t st);
void launch_rmse_final(const double *partial, int blocks, double *out2, cudaStream_t st);

// Moment matching (Section 4.1) per arena row: mu = S1/S, Sigma = S2/S - mu mu^T,
// Lambda = Sigma^{-1}; writes mu [R x K] (AoS), Lambda packed SoA and b = Lambda mu SoA.
struct MMParams {
    int K;
    int64_t r0, r1, R;
    const double *S1, *S2;   // SoA
    double S;
    double *mu;              // [R x K]
    double *L;               // SoA [ntri][R]
    double *b;               // SoA [K][R]
    DevError *err;
};
void launch_mm(const MMParams &a, cudaStream_t st);

// Copy per-row propagated priors from a source arena range to a destination range and set the
// destination state to the propagated mean.
struct PropParams {
    int K;
    int64_t n, src0, dst0, R;
    const double *mu, *L, *b;     // source MM results (mu AoS [R x K], L/b SoA)
    double *pL, *pb;              // destination prior SoA
    double *X;                    // destination state [R x K]
    void *Xg;
    int ldg, prec;
};
void launch_propagate(const PropParams &a, cudaStream_t st);

// Algorithm 2 for one factor: for each global row n (reordered order), J submodel arena rows
// sub_row[j] + (n - block start); writes mu* [n_rows x K].
struct AggParams {
    int K;
    int64_t n_rows;           // rows of this block
    int J;
    const int64_t *sub_base;  // [J] arena row of the block's first row in submodel j
    const double *mu;         // MM means AoS [R x K]
    const double *L;          // MM precisions SoA [ntri][R]
    int64_t R;
    double eps_rel;
    double *out;              // [n_rows x K]
    double *corr;             // [(J - 1) x n_rows] eigenvalue correction of each (row, j >= 1)
    unsigned long long *n_corrected;
    DevError *err;
    int32_t *list;            // [(J - 1) x n_rows] scratch: pairs whose difference is not PD
    unsigned *list_n;         // their count (reset by the launcher)
};
void launch_aggregate(const AggParams &a, cudaStream_t st);

// A factor block with a single submodel: posterior mean = mean of the retained samples,
// out[r][k] = S1[k][base + r] * inv_kept.
void launch_mean_rows(int K, int64_t n, const double *S1, int64_t R, int64_t base,
                      double inv_kept, double *out, cudaStream_t st);

// Posterior-mean predictions y_hat = offset + Xm[row]^T Wm[col] of n entries; (row, col) are
// reordered indices when the rank maps are null, else original ones mapped through them.
// yhat (nullable) receives the predictions; with y non-null, partial[2 b] receives block b's
// sum of (y - y_hat)^2 and partial[2 b + 1] zero (sum them with launch_rmse_final).
struct PredictParams {
    int K;
    int64_t n;
    const int32_t *row, *col;
    const int64_t *row_rank, *col_rank;
    const double *Xm, *Wm;
    double offset;
    double *yhat;
    const double *y;
    double *partial;
};
void launch_predict_sq(const PredictParams &p, int blocks, cudaStream_t st);

// out[a][k] = in[src[a]][k] for the R rows of a factor arena (chain restart).
void launch_gather_rows(int K, int64_t R, const int64_t *src, const double *in, double *out,
                        cudaStream_t st);

// Summaries beyond moment matching (summary.cu; Section 4.1 PP DM / PP GMM): one warp per row
// clusters the row's retained samples by lambda-means and fits the dominant mode (mode 1), the
// C largest modes (mode 2) or all samples (mode 0), with the pooled moments of the mixture.
constexpr int kMaxComponents = 4;
struct SummaryParams {
    int K, S, C, mode;
    double lambda;
    const double *samples;     // sample s of arena row a at samples[s * sample_stride + a * K]
    int64_t sample_stride;
    int64_t row0, n_rows;      // rows [row0, row0 + n_rows), one block each
    // outputs indexed by row - row0 (nullable as a group): pi [n][C], mu [n][C][K],
    // Lam [n][C][K][K], pooled_mu [n][K], pooled_Lam [n][K][K]; assign [n][S] (nullable)
    double *pi, *mu, *Lam, *pooled_mu, *pooled_Lam;
    int32_t *assign;
    // library layout, indexed by arena row (nullable as a group): the summary that propagates
    // and aggregates (dominant component for mode 1, pooled moments otherwise) as mm_mu AoS
    // [R][K], mm_L SoA [ntri][R], mm_b SoA [K][R]; mix (nullable): the mixture store
    // [R][C][1 + 2K + ntri(K)] (score constant, mean, packed precision, precision x mean)
    double *mm_mu, *mm_L, *mm_b, *mix;
    int64_t R;
    DevError *err;
};
size_t summary_smem(int K, int S);
void launch_summary(const SummaryParams &p, cudaStream_t st);

// Component choice of a propagated mixture prior for arena rows [r0, r0 + n) that carry one
// (has_mix): the component with the largest responsibility at the current X becomes the row's
// prior (pL, pb).
struct MixChooseParams {
    int K, C;
    int64_t r0, n, R;
    const double *mix;
    const int8_t *has_mix;
    const double *X;
    double *pL, *pb;
    int32_t *chosen;           // [R] nullable
    DevError *err;
};
void launch_mix_choose(const MixChooseParams &p, cudaStream_t st);

// K > 16 (wide.cu): Gram on the tensor cores (BF16, split TF32) or FP64 lanes over entries;
// conditional draw with one warp per row.  Partials: packed lower of the exact K, then K rhs.
int wide_kt(int K);
int wide_part_ld(int K);
void launch_gram_wide(int K, int prec, const GramParams &a, int grid, cudaStream_t st,
                      bool tf32_single = false);
// Conditional draw with a team of `team` lanes (4, 8, 16 or 32) per row (wide.cu).
void launch_cond_team(int prec, const CondParams &a, int n_blocks, int team, cudaStream_t st);
int cond_team_size(int K);
// Whether the conditional can factor a row of dimension K with `lanes` lanes: two lanes (the
// register-resident kernel) for 13 <= K <= 16, else a team whose rows fit in shared memory.
bool cond_lanes_valid(int K, int lanes);
// The same draw for 13 <= K <= 16 with two lanes per row and the row's matrix in registers
// (cond_pair.cu; bit-identical to the team kernel).  False for other K (nothing launched).
bool launch_cond_pair(int prec, const CondParams &a, int n_blocks, cudaStream_t st);

// Adjoint of the masked log-joint (adjoint.cu).
int adjoint_kt(int K);          // template width (K rounded up to 4, 8, 12, 16, 32 or 64)
int adjoint_ld(int K);          // floats per item partial
int adjoint_row_blocks(int64_t n_rows);
struct AdjointParams {
    int K, kt, ldp;
    // pass 1: items items[0 .. n_items) (absolute index item_base + i)
    const GramItem *items;
    int64_t n_items, item_base;
    const int32_t *idx;         // partner arena rows
    const float *val;
    const float *self, *other;  // caller factors [rows x ld] FP32, 16-byte aligned, ld % 4 == 0
    int64_t ld;
    int64_t self0, other0;      // arena rows of local row 0
    float *part;                // [n_items x ldp]
    // pass 2
    int64_t n_rows;
    const int64_t *item_ptr;
    const int32_t *row_hslot;
    const double *hyper, *prior_L, *prior_b;
    int64_t R;
    float *grad;                // [n_rows x ld]
    double alpha;
    int count_r2;
    double *block_sums;         // [row blocks x 2]: sum r^2, sum prior quadratic
};
void launch_adjoint(const AdjointParams &a, int grid, cudaStream_t st);
void launch_langevin(float *theta, const float *grad, const float *xi, int64_t n_rows, int K,
                     int ld, float eps, cudaStream_t st);
void launch_to_float(const double *in, float *out, int64_t n, cudaStream_t st);
void launch_sqdiff(const float *a, const float *b, const float *g, double coef, int64_t n_rows,
                   int K, int64_t ld, double *block_sums, int blocks, cudaStream_t st);

// Device generator of the draws (counter-based, see rng.cu).  A segment is one stream of the
// draw buffer: kind 1 chi-square variates (one thread each, dof0 - k for variate k), kind 2/3
// normals (one thread per four).
struct GenSeg {
    int64_t unit0;   // first thread of the segment
    int64_t count;   // numbers in the segment
    int64_t out;     // offset in the sweep's draw buffer
    uint64_t tag;    // subset id * 256 + factor * 16 + kind
    double dof0;
    int32_t kind;    // 1 chi-square (dof0 - k), 2/3 normals, 4 chi-square (dof0 + entries)
    int64_t row0;    // kind 4: W arena row of variate 0 (dof0 + its entries), or -1 (dof0)
};
struct GenParams {
    const GenSeg *segs;
    int n_segs;
    int64_t n_units;
    uint64_t seed;
    int64_t t;       // 1-based sweep number of the batch's chains
    double *out;
    const int64_t *cnt_ptr;   // kind 4: W arena observation offsets (entries of a column)
    DevError *err;
};
struct GenSubset {
    int32_t sid;
    int64_t n, d;
    int64_t woff, nnz;   // W arena row of the subset's first column, its training entries
};
void launch_gen(const GenParams &p, cudaStream_t st);
// Segments of one sweep's buffer for the batch `subs` (id order); returns the thread count.
// noise: 0 none, 1 one precision per subset, 2 one per column (kind-4 chi-squares after the z's,
// dof 2 a0 + entries).
int64_t gen_segments(const std::vector<GenSubset> &subs, int K, double nu0, int noise, double a0,
                     std::vector<GenSeg> &segs);

// Sampled noise precision (Section 2.1).  noise_sse: per W arena row of [r0, r1), the sum of
// squared residuals over the column's entries (FP64, in order) into sse.  noise_tau: the new
// precisions from the chi-square variates (column mode: tau = c / (2 b0 + SSE) per row; global
// mode: per subset block [b0_k, b1_k) one value from the block's summed SSE).  noise_scale:
// the scaled copies the row-side Gram takes, Ws[r] = sqrt(tau[r]) W[r] for rows [r0, r1) and
// val[q] = val_orig[q] sqrt(tau[idx[q]]) for entries [q0, q1).
void launch_noise_sse(int K, int64_t r0, int64_t r1, const int64_t *ptr, const int32_t *idx,
                      const void *val, int prec, const double *X, const double *W, double *sse,
                      cudaStream_t st);
struct NoiseBlock {
    int64_t r0, r1;      // W arena rows of one subset
    int64_t draw;        // offset of its variates in the sweep's draw buffer
};
void launch_noise_tau(int mode, double b0, const NoiseBlock *blocks, int n_blocks,
                      const double *draws, const double *sse, double *tau, cudaStream_t st);
void launch_noise_scale(int K, int prec, int64_t r0, int64_t r1, const double *tau,
                        const double *W, void *Ws, int ldg, int64_t q0, int64_t q1,
                        const int32_t *idx, const void *val_orig, void *val, cudaStream_t st);

// Device helpers
void launch_fill_gather(int K, int prec, int64_t R, const double *X, void *Xg, int ldg,
                        cudaStream_t st);

}  // namespace bmf
