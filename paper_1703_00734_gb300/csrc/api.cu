// api.cu -- the C ABI of libbmf (include/bmf.h) and the runtime behind it: the context, its
// device arenas, the batched sweep of a stage (Algorithm 1), the stage transitions with
// propagated priors and the final aggregation (Eq. 14, Algorithm 2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bmf.h"
#include "common.cuh"
#include "kernels.h"
#include "plan.h"

using namespace bmf;

namespace {

thread_local std::string g_init_error;
thread_local const char *g_noctx_msg = nullptr;  // set by context-less calls that do not allocate

struct DevMem {
    std::vector<void *> ptrs;
    bool ok = true;
    template <typename T>
    T *alloc(size_t n)
    {
        if (n == 0) n = 1;
        void *p = nullptr;
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~DevMem()
    {
        for (void *p : ptrs) cudaFree(p);
    }
};

// One factor arena (all subsets' blocks of X, or of W, stacked in slot order) with the
// observation lists of its rows (partners in the other arena).
struct Side {
    int64_t R = 0;
    double *F = nullptr;         // FP64 state [R x K]
    void *G = nullptr;           // gathered copy [R x ldg]
    int64_t *ptr = nullptr;      // observation list offsets [R+1]
    int32_t *idx = nullptr;      // partner arena rows
    void *val = nullptr;         // values (double or float)
    GramItem *items = nullptr;   // Gram work items in arena-row order
    int64_t *item_ptr = nullptr; // [R+1]
    GramTask *tasks = nullptr;   // warp tasks, grouped per slot
    std::vector<int64_t> slot_task;  // [S+1] first task of each slot
    std::vector<int64_t> blk_task;   // [blocks+1] first task of each conditional block
    std::vector<int64_t> h_item_ptr;
    std::vector<int64_t> h_obs;      // [R+1] observation offsets (chunk costs)
    int32_t *hslot = nullptr;    // [R] hyper slot or -1
    std::vector<int32_t> h_hslot;
    // rows with more than one Gram work item, their FP64 sums
    std::vector<int32_t> h_multi;     // arena rows, increasing
    // conditional-kernel blocks: up to kCondBlock rows of one subset each, in slot order
    std::vector<CondBlock> h_blocks;
    std::vector<int64_t> slot_blk;    // [S+1] first block of each slot
    CondBlock *blocks = nullptr;
    StatChunk *chunks = nullptr;      // the same row ranges, for the standalone statistics pass
    int64_t stat0 = 0;                // first statistics slot of this arena
    int32_t *multi_idx = nullptr;     // [R] slot in rowsum or -1
    int *counters = nullptr;          // [slots x parts] completion counters (zero when idle)
    double *rowsum = nullptr;
    double *pL = nullptr, *pb = nullptr;            // per-row prior (SoA)
    double *S1 = nullptr, *S2 = nullptr;            // moment sums (SoA)
    double *mm_mu = nullptr, *mm_L = nullptr, *mm_b = nullptr;  // moment-matched posterior
};

struct SubState {
    int64_t t = 0, kept = 0;
    int prior[2] = {0, 0};  // 1: factor has a per-row (propagated or installed) prior
    int mix[2] = {0, 0};    // 1: that prior is a propagated mixture (GMM summary)
    bool finalized = false;
};

}  // namespace

constexpr int kMaxChunks = BMF_MAX_CHUNKS;
constexpr int kCopyGroups = 16;   // copy groups of a host draw buffer (events per call)

struct bmf_ctx {
    ~bmf_ctx()
    {
        for (cudaStream_t x : {st2, st3, st4, st5, cap})
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        for (cudaEvent_t e : {ev_fork, ev_fac[0], ev_fac[1], ev_hyp[0], ev_hyp[1], ev_cdone, ev_tail,
                              ev_tail2, ev_rmse, ev_gen[0], ev_gen[1]})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_copyq)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_chunk)
            if (e) cudaEventDestroy(e);
        for (auto &g : graphs)
            if (g.exec) cudaGraphExecDestroy(g.exec);
        if (rb) cudaFreeHost(rb);
    }
    int K = 0, prec = BMF_FP64;
    double tau = 1.0, beta0 = 2.0, nu0 = 1.0, eps_rel = 1e-6;
    int burnin = 0, thin = 1;
    uint64_t seed = 0;
    std::vector<double> mu0, W0inv;
    HostPlan P;
    cudaStream_t st = nullptr;
    cudaStream_t st2 = nullptr;      // side stream: factor statistics and hyperparameter draws
    cudaStream_t st3 = nullptr;      // conditional stream of the chunked schedule
    cudaStream_t st4 = nullptr;      // tail stream: test RMSE
    cudaStream_t st5 = nullptr;      // generator stream: the draws of the sweep after next
    cudaStream_t cap = nullptr;      // capture stream of the graph schedule (the context stream
                                     // may be the legacy default stream, which cannot capture)
    cudaEvent_t ev_fork = nullptr, ev_fac[2] = {nullptr, nullptr}, ev_hyp[2] = {nullptr, nullptr};
    cudaEvent_t ev_chunk[kMaxChunks] = {}, ev_cdone = nullptr;
    cudaEvent_t ev_tail = nullptr, ev_tail2 = nullptr, ev_rmse = nullptr, ev_gen[2] = {nullptr, nullptr};
    // a host draw buffer is copied on the generator stream in groups of sweeps, an event after
    // each group, so that sweep t waits only for its own group
    cudaEvent_t ev_copyq[kCopyGroups] = {};
    struct Readback {
        DevError err;
        double rmse[2];
    } *rb = nullptr;                 // pinned host block: the end-of-call readback
    bmf_schedule sched = {1, 1, 4, 0.0, 0, 0};
    // graph schedule: the last captured launch sequence of each batch (a stage or one subset),
    // updated in place by the next call of the same shape
    struct GraphEntry {
        int sl0, sl1;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    int device = 0, sms = 1;
    DevMem mem;
    Side X, W;
    int ldg = 0, ld_part = 0, part_rhs = 0;
    void *part = nullptr;
    int64_t part_cap = 0;            // items
    double *hyper = nullptr;         // [2 * S slots]
    double *stats = nullptr;
    int64_t stats_cap = 0;           // chunks
    HyperJob *d_jobs = nullptr;
    HyperJob *d_jobs2 = nullptr;     // the same jobs over the first-level partials
    std::vector<HyperJob> jobs_up;   // the job list last uploaded (skip identical uploads)
    std::vector<char> stats_ok;      // [S] per slot: c->stats hold the statistics of its state
    double *stats2 = nullptr;        // [2 S x kStatParts x (K + ntri(K))] first-level partials
    double *mu0_d = nullptr, *W0inv_d = nullptr;
    int32_t *trow = nullptr, *tcol = nullptr;
    double *tval = nullptr, *ysum = nullptr;
    double *rmse_part = nullptr, *rmse_out = nullptr;
    int rmse_blocks = 608;
    DevError *err_d = nullptr;
    double *draws_d = nullptr;
    int64_t draws_cap = 0;
    // device generator: two sweeps' draw buffers (ring) and the segment table
    double *gen_d = nullptr;
    int64_t gen_cap = 0;
    GenSeg *gen_segs_d = nullptr;
    int64_t gen_segs_cap = 0;
    double *aggX = nullptr, *aggW = nullptr;   // aggregated means, reordered order
    unsigned long long *ncorr_d = nullptr;
    int64_t *agg_base = nullptr;     // [(I + J) max(I, J)] submodel base rows of every launch
    double *agg_corr = nullptr;      // eigenvalue corrections of every (row, submodel) pair
    int32_t *agg_list = nullptr;     // pairs needing an eigenvalue (scratch of one launch)
    unsigned *agg_list_n = nullptr;
    // bmf_restart: the initial states in the original order and the original index of every
    // arena row (the chains restart by a gather on the device)
    double *X0o = nullptr, *W0o = nullptr;
    int64_t *xsrc = nullptr, *wsrc = nullptr;
    // held-out entries in the reordered index space (bmf_test_rmse) and original -> reordered
    // index maps (bmf_predict), so that predictions need no host round trip of the means
    int32_t *tg_row = nullptr, *tg_col = nullptr;
    int64_t *row_rank_d = nullptr, *col_rank_d = nullptr;
    double *pred_part = nullptr, *pred_out = nullptr;
    char *pred_buf = nullptr;        // prediction entries of bmf_predict (grown on use)
    int64_t pred_cap = 0;
    std::vector<SubState> ss;
    int stage_open = 0;
    bool failed = false;
    bool tf32 = false;               // BMF_TF32: one TF32 product per wide Gram tile
    std::string err;
    int chunk_obs = 1024;
    bool full_moments = false;
    bool monitor = true;             // per-sweep test RMSE (bmf_set_monitor)
    // DM / GMM summaries (Section 4.1): retained samples per arena ([max_samples][R][K]), the
    // mixture store of propagated mixture priors per arena and which rows carry one
    int summary = BMF_SUMMARY_MM, ncomp = 3, max_samples = 0;
    bool independent = false;        // no propagation between stages (cfg.independent)
    // sampled noise precision (cfg.noise): tau per W arena row, the row-side Gram's scaled copy
    // of W and scaled values (the originals kept), per-row SSE, the batch's subset blocks
    int noise = BMF_NOISE_FIXED;
    double noise_a0 = 1.0, noise_b0 = 1.0;
    double *tau_w = nullptr, *noise_sse = nullptr;
    void *Ws = nullptr, *xval_orig = nullptr;
    NoiseBlock *noise_blocks = nullptr;
    std::vector<NoiseBlock> h_noise_blocks;
    double lambda = 0.0;
    double *ring[2] = {nullptr, nullptr};
    double *mix[2] = {nullptr, nullptr};
    int8_t *has_mix[2] = {nullptr, nullptr};
    // adjoint / Langevin scratch (allocated on first use)
    float *adj_part = nullptr;
    int64_t adj_part_cap = 0;
    double *adj_sums = nullptr;
    int64_t adj_sums_cap = 0;
    float *fval[2] = {nullptr, nullptr};     // FP32 values for FP64 contexts
    float *lg_buf = nullptr;                 // Langevin proposals and gradients
    int64_t lg_cap = 0;
    // tracing
    int64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    size_t ev_used = 0;
    double prof_ms[9] = {0};
    int64_t prof_n[9] = {0};
};

namespace {

constexpr int kHyperJobsMax = 1 << 16;
constexpr int kNarrowMaxK = 16;   // CUDA-core Gram pass up to here, tensor cores beyond
constexpr int kTeamMinK = 13;     // conditional: one thread per row below, a team per row from here

enum { K_STATS = 0, K_HYPER, K_GRAM_X, K_COND_X, K_GRAM_W, K_COND_W, K_RMSE, K_ADJ, K_GEN, K_NCLASS };
const char *kClassName[K_NCLASS] = {"stats", "hyper", "gram_x", "cond_x", "gram_w", "cond_w", "rmse", "adjoint", "gen"};

cudaEvent_t pool_event(bmf_ctx *c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Run `launch` (which enqueues `n` kernels) and, with profiling on, bracket it with events.
template <typename F>
void traced(bmf_ctx *c, cudaStream_t st, int cls, int n, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        a = pool_event(c);
        b = pool_event(c);
        cudaEventRecord(a, st);
    }
    launch();
    c->launches += n;
    if (c->prof) {
        cudaEventRecord(b, st);
        c->ev_pending.push_back({cls, {a, b}});
    }
}

// After a synchronisation: fold the pending event pairs into the per-class totals.
void collect_profile(bmf_ctx *c)
{
    for (auto &p : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess) {
            c->prof_ms[p.first] += ms;
            c->prof_n[p.first] += 1;
        }
    }
    c->ev_pending.clear();
    c->ev_used = 0;
}

bmf_status fail(bmf_ctx *c, bmf_status s, const std::string &m)
{
    c->err = m;
    return s;
}

bmf_status cuda_fail(bmf_ctx *c, cudaError_t e, const char *where)
{
    c->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return BMF_E_CUDA;
}

bmf_status cuda_status(bmf_ctx *c, cudaError_t e, const char *where)
{
    return e == cudaSuccess ? BMF_OK : cuda_fail(c, e, where);
}

#define CUDA_TRY(c, call)                                         \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
    } while (0)

int64_t hyper_block_len(int K) { return K + (int64_t)K * (K - 1) / 2 + K; }

// Doubles per component in the mixture store: score constant, mean, packed precision, precision
// x mean.
int64_t mix_width(int K) { return 1 + 2 * (int64_t)K + (int64_t)K * (K + 1) / 2; }

// Host FP64 inverse of a small SPD matrix (Gauss-Jordan with partial pivoting).
bool host_inverse(int K, const std::vector<double> &A, std::vector<double> &Ainv)
{
    std::vector<double> a(A);
    Ainv.assign((size_t)K * K, 0.0);
    for (int i = 0; i < K; ++i) Ainv[i * K + i] = 1.0;
    for (int c = 0; c < K; ++c) {
        int p = c;
        for (int r = c + 1; r < K; ++r)
            if (std::fabs(a[r * K + c]) > std::fabs(a[p * K + c])) p = r;
        if (!(std::fabs(a[p * K + c]) > 0.0)) return false;
        if (p != c)
            for (int k = 0; k < K; ++k) {
                std::swap(a[p * K + k], a[c * K + k]);
                std::swap(Ainv[p * K + k], Ainv[c * K + k]);
            }
        double d = a[c * K + c];
        for (int k = 0; k < K; ++k) {
            a[c * K + k] /= d;
            Ainv[c * K + k] /= d;
        }
        for (int r = 0; r < K; ++r)
            if (r != c) {
                double f = a[r * K + c];
                if (f == 0.0) continue;
                for (int k = 0; k < K; ++k) {
                    a[r * K + k] -= f * a[c * K + k];
                    Ainv[r * K + k] -= f * Ainv[c * K + k];
                }
            }
    }
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (Ainv[i * K + j] + Ainv[j * K + i]);
            Ainv[i * K + j] = Ainv[j * K + i] = m;
        }
    return true;
}

const SubsetGeom &geom_of_slot(const bmf_ctx *c, int sl) { return c->P.subs[c->P.slot_sid[sl]]; }

// Gram partial layout: entries per item and the offset of the right-hand side.
int part_nv(int K) { return K > kNarrowMaxK ? ntri(K) + K : gram_nv(padded_k(K)); }
int part_rhs_of(int K) { return K > kNarrowMaxK ? ntri(K) : ntri(padded_k(K)); }
int part_ld_of(int K, int prec) { return K > kNarrowMaxK ? wide_part_ld(K) : gram_part_ld(K, prec); }
int part_parts(int K, int prec) { return K > kNarrowMaxK ? 1 : gram_parts(K, prec); }

// Slot range [sl0, sl1) of a stage (slots are sorted by stage).
bool stage_slots(const bmf_ctx *c, int stage, int &sl0, int &sl1)
{
    int S = (int)c->P.slot_sid.size();
    sl0 = sl1 = -1;
    for (int sl = 0; sl < S; ++sl)
        if (geom_of_slot(c, sl).stage == stage) {
            if (sl0 < 0) sl0 = sl;
            sl1 = sl + 1;
        }
    return sl0 >= 0;
}

int64_t per_sweep_draws(const bmf_ctx *c, int sl0, int sl1)
{
    int64_t n = 2 * (int64_t)(sl1 - sl0) * hyper_block_len(c->K);
    for (int sl = sl0; sl < sl1; ++sl) n += (geom_of_slot(c, sl).n() + geom_of_slot(c, sl).d()) * c->K;
    // sampled noise precisions: one chi-square per column of each subset, or one per subset
    for (int sl = sl0; sl < sl1 && c->noise; ++sl) n += c->noise == 2 ? geom_of_slot(c, sl).d() : 1;
    return n;
}

void refresh_hslots(bmf_ctx *c, int sl)
{
    const SubsetGeom &g = geom_of_slot(c, sl);
    SubState &s = c->ss[g.sid];
    for (int64_t r = 0; r < g.n(); ++r) c->X.h_hslot[g.xoff + r] = s.prior[0] ? -1 : 2 * sl + 0;
    for (int64_t r = 0; r < g.d(); ++r) c->W.h_hslot[g.woff + r] = s.prior[1] ? -1 : 2 * sl + 1;
}

bmf_status upload_hslots(bmf_ctx *c, int sl)
{
    const SubsetGeom &g = geom_of_slot(c, sl);
    if (g.n() > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->X.hslot + g.xoff, c->X.h_hslot.data() + g.xoff,
                                    g.n() * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    if (g.d() > 0)
        CUDA_TRY(c, cudaMemcpyAsync(c->W.hslot + g.woff, c->W.h_hslot.data() + g.woff,
                                    g.d() * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    return BMF_OK;
}

bmf_status dev_error_status(bmf_ctx *c, const DevError &h);

bmf_status check_dev_error(bmf_ctx *c)
{
    if (c->st2) CUDA_TRY(c, cudaStreamSynchronize(c->st2));
    if (c->st3) CUDA_TRY(c, cudaStreamSynchronize(c->st3));
    if (c->st4) CUDA_TRY(c, cudaStreamSynchronize(c->st4));
    if (c->st5) CUDA_TRY(c, cudaStreamSynchronize(c->st5));
    DevError h;
    CUDA_TRY(c, cudaMemcpyAsync(&h, c->err_d, sizeof(h), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return dev_error_status(c, h);
}

// Status of a device error word read back to the host (clears the word on the device).
bmf_status dev_error_status(bmf_ctx *c, const DevError &h)
{
    if (h.flags) {
        DevError z = {0u, INT32_MAX};
        cudaMemcpy(c->err_d, &z, sizeof(z), cudaMemcpyHostToDevice);
        c->failed = true;
        if (h.flags & ERR_NOT_PD)
            return fail(c, BMF_E_NOT_PD,
                        "matrix not positive definite (arena row " +
                            std::to_string(h.first_bad_row) + "); the context must be reset "
                            "with bmf_set_state before further sweeps");
        if (h.flags & ERR_RNG)
            return fail(c, BMF_E_CUDA, "device generator: 64 chi-square rejections in a row");
        return fail(c, BMF_E_CUDA, "device error flags " + std::to_string(h.flags));
    }
    return BMF_OK;
}

// One factor's observation lists -> device (values converted to the gather precision) and the
// Gram work items of every arena row (rows longer than chunk_obs are split).
bmf_status setup_side(bmf_ctx *c, Side &s, int64_t R, const std::vector<int64_t> &ptr,
                      const std::vector<int32_t> &idx, const std::vector<double> &val)
{
    s.R = R;
    const int64_t nnz = (int64_t)idx.size();
    s.ptr = c->mem.alloc<int64_t>(R + 1);
    s.idx = c->mem.alloc<int32_t>(nnz);
    if (c->prec == BMF_FP64)
        s.val = c->mem.alloc<double>(nnz);
    else
        s.val = c->mem.alloc<float>(nnz);
    if (!c->mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (observation lists)");
    CUDA_TRY(c, cudaMemcpy(s.ptr, ptr.data(), (R + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (nnz) {
        CUDA_TRY(c, cudaMemcpy(s.idx, idx.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
        if (c->prec == BMF_FP64) {
            CUDA_TRY(c, cudaMemcpy(s.val, val.data(), nnz * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(val.begin(), val.end());
            CUDA_TRY(c, cudaMemcpy(s.val, f.data(), nnz * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    std::vector<GramItem> items;
    s.h_obs = ptr;
    s.h_item_ptr.assign(R + 1, 0);
    for (int64_t r = 0; r < R; ++r) {
        s.h_item_ptr[r] = (int64_t)items.size();
        int64_t b = ptr[r], e = ptr[r + 1];
        for (int64_t q = b; q < e; q += c->chunk_obs) {
            GramItem it;
            it.begin = q;
            it.count = (int32_t)std::min<int64_t>(c->chunk_obs, e - q);
            it.row = (int32_t)r;
            items.push_back(it);
        }
    }
    s.h_item_ptr[R] = (int64_t)items.size();
    std::vector<int32_t> midx(R, -1);
    const bool fuse = c->K >= kTeamMinK && c->K <= kNarrowMaxK;
    for (int64_t r = 0; r < R; ++r) {
        const int64_t ni = s.h_item_ptr[r + 1] - s.h_item_ptr[r];
        if (ni > 1) {
            midx[r] = (int32_t)s.h_multi.size();
            s.h_multi.push_back((int32_t)r);
        } else if (fuse && ni == 1 && items[s.h_item_ptr[r]].count <= kFuseMaxObs) {
            midx[r] = kFusedRow;   // Gram sums formed by the conditional draw
        }
    }
    const size_t nctr = s.h_multi.size() * (size_t)part_parts(c->K, c->prec);
    s.counters = c->mem.alloc<int>(nctr);
    s.multi_idx = c->mem.alloc<int32_t>(R);
    s.rowsum = c->mem.alloc<double>(s.h_multi.size() * (size_t)part_nv(c->K));
    if (!c->mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (row sums)");
    CUDA_TRY(c, cudaMemset(s.counters, 0, std::max<size_t>(nctr, 1) * sizeof(int)));
    CUDA_TRY(c, cudaMemcpy(s.multi_idx, midx.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice));
    // warp tasks per slot: long rows / row chunks one per warp, short rows packed 32/G per warp
    {
        const int S = (int)c->P.slot_sid.size();
        const bool xs = &s == &c->X;
        std::vector<GramTask> tasks;
        s.slot_task.assign(S + 1, 0);
        for (int sl = 0; sl < S; ++sl) {
            s.slot_task[sl] = (int64_t)tasks.size();
            const SubsetGeom &g = geom_of_slot(c, sl);
            const int64_t r0 = xs ? g.xoff : g.woff, r1 = r0 + (xs ? g.n() : g.d());
            GramTask cur{0, 0, 0};
            for (int64_t r = r0; r < r1; ++r) {
                // tasks never cross a conditional block, so that any block range of the batch
                // is a task range (the chunked schedule of run_batch)
                if ((r - r0) % kCondBlock == 0) {
                    if (cur.n) tasks.push_back(cur), cur.n = 0;
                    s.blk_task.push_back((int64_t)tasks.size());
                }
                const int64_t i0 = s.h_item_ptr[r], i1 = s.h_item_ptr[r + 1];
                if (i1 == i0 || midx[r] == kFusedRow) continue;
                const int G = (i1 - i0 > 1) ? 32 : gram_group(items[i0].count);
                if (G == 32) {
                    if (cur.n) tasks.push_back(cur), cur.n = 0;
                    for (int64_t it = i0; it < i1; ++it) tasks.push_back(GramTask{it, 1, 32});
                    continue;
                }
                if (cur.n && (cur.G != G || cur.n == 32 / cur.G || cur.item0 + cur.n != i0))
                    tasks.push_back(cur), cur.n = 0;
                if (!cur.n) cur = GramTask{i0, 0, G};
                ++cur.n;
            }
            if (cur.n) tasks.push_back(cur);
        }
        s.slot_task[S] = (int64_t)tasks.size();
        s.blk_task.push_back((int64_t)tasks.size());
        s.tasks = c->mem.alloc<GramTask>(tasks.size());
        if (!c->mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (tasks)");
        if (!tasks.empty())
            CUDA_TRY(c, cudaMemcpy(s.tasks, tasks.data(), tasks.size() * sizeof(GramTask),
                                   cudaMemcpyHostToDevice));
    }
    s.items = c->mem.alloc<GramItem>(items.size());
    s.item_ptr = c->mem.alloc<int64_t>(R + 1);
    if (!c->mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (work items)");
    if (!items.empty())
        CUDA_TRY(c, cudaMemcpy(s.items, items.data(), items.size() * sizeof(GramItem),
                               cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(s.item_ptr, s.h_item_ptr.data(), (R + 1) * sizeof(int64_t),
                           cudaMemcpyHostToDevice));
    c->part_cap = std::max<int64_t>(c->part_cap, (int64_t)items.size());
    // state, copies, priors, moments
    const int K = c->K;
    const int NT = ntri(K);
    s.F = c->mem.alloc<double>(R * K);
    size_t gbytes = c->prec == BMF_FP64 ? 8 : (c->prec == BMF_FP32 ? 4 : 2);
    s.G = c->mem.alloc<char>(R * c->ldg * gbytes);
    s.hslot = c->mem.alloc<int32_t>(R);
    s.h_hslot.assign(R, -1);
    s.pL = c->mem.alloc<double>(R * NT);
    s.pb = c->mem.alloc<double>(R * K);
    s.S1 = c->mem.alloc<double>(R * K);
    s.S2 = c->mem.alloc<double>(R * NT);
    s.mm_mu = c->mem.alloc<double>(R * K);
    s.mm_L = c->mem.alloc<double>(R * NT);
    s.mm_b = c->mem.alloc<double>(R * K);
    if (!c->mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (factor arena)");
    CUDA_TRY(c, cudaMemset(s.S1, 0, R * K * sizeof(double)));
    CUDA_TRY(c, cudaMemset(s.S2, 0, R * NT * sizeof(double)));
    CUDA_TRY(c, cudaMemset(s.pL, 0, R * NT * sizeof(double)));
    CUDA_TRY(c, cudaMemset(s.pb, 0, R * K * sizeof(double)));
    return BMF_OK;
}

// Draw buffer of a call on the device.  A host buffer is copied on copy_st; with `groups`
// (offsets in doubles, ascending, from 0 to need) in pieces, event evs[q] recorded after piece q.
bmf_status stage_draws(bmf_ctx *c, const bmf_draws *d, int64_t need, const double **out,
                       cudaStream_t copy_st, const std::vector<int64_t> *groups = nullptr,
                       cudaEvent_t *evs = nullptr)
{
    if (!d) {
        *out = nullptr;   // the device generator fills the sweep buffers
        return BMF_OK;
    }
    if (!d->ptr || d->len != need)
        return fail(c, BMF_E_SHAPE, "draw buffer has " + std::to_string(d->len) +
                                        " doubles, expected " + std::to_string(need));
    if (d->on_device) {
        *out = d->ptr;
        return BMF_OK;
    }
    if (need > c->draws_cap) {
        if (c->draws_d) cudaFree(c->draws_d);
        c->draws_d = nullptr;
        c->draws_cap = 0;
        if (cudaMalloc(&c->draws_d, need * sizeof(double)) != cudaSuccess)
            return fail(c, BMF_E_OOM, "device allocation failed (draw buffer)");
        c->draws_cap = need;
    }
    if (groups && evs) {
        for (size_t q = 0; q + 1 < groups->size(); ++q) {
            const int64_t a = (*groups)[q], b = (*groups)[q + 1];
            if (b > a)
                CUDA_TRY(c, cudaMemcpyAsync(c->draws_d + a, d->ptr + a, (b - a) * sizeof(double),
                                            cudaMemcpyHostToDevice, copy_st));
            CUDA_TRY(c, cudaEventRecord(evs[q], copy_st));
        }
    } else {
        CUDA_TRY(c, cudaMemcpyAsync(c->draws_d, d->ptr, need * sizeof(double),
                                    cudaMemcpyHostToDevice, copy_st));
    }
    *out = c->draws_d;
    return BMF_OK;
}

// Device generator for the batch of slots [sl0, sl1): segment table to the device and room for
// `nbuf` sweep buffers of `per` doubles.  Returns the generator's thread count in *units.
bmf_status prepare_gen(bmf_ctx *c, int sl0, int sl1, int64_t per, int nbuf, int64_t *units,
                       int *n_segs)
{
    std::vector<GenSubset> subs;
    for (int sl = sl0; sl < sl1; ++sl) {
        const SubsetGeom &g = geom_of_slot(c, sl);
        subs.push_back(GenSubset{g.sid, g.n(), g.d(), g.woff,
                                 c->W.h_obs[g.woff + g.d()] - c->W.h_obs[g.woff]});
    }
    std::vector<GenSeg> segs;
    *units = gen_segments(subs, c->K, c->nu0, c->noise, c->noise_a0, segs);
    *n_segs = (int)segs.size();
    if ((int64_t)segs.size() > c->gen_segs_cap) {
        if (c->gen_segs_d) cudaFree(c->gen_segs_d);
    if (c->pred_buf) cudaFree(c->pred_buf);
        c->gen_segs_d = nullptr;
        c->gen_segs_cap = 0;
        if (cudaMalloc(&c->gen_segs_d, segs.size() * sizeof(GenSeg)) != cudaSuccess)
            return fail(c, BMF_E_OOM, "device allocation failed (generator segments)");
        c->gen_segs_cap = (int64_t)segs.size();
    }
    if (!segs.empty())
        CUDA_TRY(c, cudaMemcpyAsync(c->gen_segs_d, segs.data(), segs.size() * sizeof(GenSeg),
                                    cudaMemcpyHostToDevice, c->st));
    const int64_t need = (int64_t)nbuf * per;
    if (need > c->gen_cap) {
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
        if (c->gen_d) cudaFree(c->gen_d);
        c->gen_d = nullptr;
        c->gen_cap = 0;
        if (cudaMalloc(&c->gen_d, need * sizeof(double)) != cudaSuccess)
            return fail(c, BMF_E_OOM, "device allocation failed (generator buffers)");
        c->gen_cap = need;
    }
    return BMF_OK;
}

void enqueue_gen(bmf_ctx *c, int64_t units, int n_segs, int64_t t, double *out)
{
    GenParams gp{c->gen_segs_d, n_segs, units, c->seed, t, out, c->W.ptr, c->err_d};
    traced(c, c->st, K_GEN, 1, [&] { launch_gen(gp, c->st); });
}

bool keep_sample(const bmf_ctx *c, int64_t t)
{
    return t > c->burnin && (t - c->burnin - 1) % c->thin == 0;
}

// Row chunks of one sweep half for the chunked schedule: block boundaries b0 = B[0] < ... <
// B[n] = b1 at equal quantiles of an estimated cost (observations + row_weight x rows).
std::vector<int64_t> chunk_bounds(const bmf_ctx *c, const Side &sd, int64_t b0, int64_t b1,
                                  int n_chunks, int64_t r_end)
{
    std::vector<int64_t> B{b0};
    const int64_t nb = b1 - b0;
    const int n = (int)std::min<int64_t>(std::max(n_chunks, 1), std::max<int64_t>(nb, 1));
    if (n <= 1 || nb <= 1) {
        B.push_back(b1);
        return B;
    }
    const double w = c->sched.row_weight > 0.0
                         ? c->sched.row_weight
                         : (c->prec == BMF_FP64 ? 1.5 : 14.0) * c->K;
    auto row_of = [&](int64_t b) { return b == b1 ? r_end : sd.h_blocks[b].row0; };
    std::vector<double> cum(nb + 1, 0.0);
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t ra = row_of(b), rb = row_of(b + 1);
        cum[b - b0 + 1] = cum[b - b0] + (double)(sd.h_obs[rb] - sd.h_obs[ra]) + w * (double)(rb - ra);
    }
    int64_t q = 0;
    for (int k = 1; k < n; ++k) {
        const double target = cum[nb] * k / n;
        while (q < nb && cum[q] < target) ++q;
        if (q > B.back() - b0 && q < nb) B.push_back(b0 + q);
    }
    B.push_back(b1);
    return B;
}

// Graph schedule: while a call's launch sequence is captured, the context's main stream is the
// capture stream; the guard ends a capture left open by an early error return (discarding the
// graph) and gives the context its stream back.
struct CaptureGuard {
    bmf_ctx *c = nullptr;
    cudaStream_t user = nullptr;
    bool active = false;
    ~CaptureGuard()
    {
        if (!active) return;
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(c->st, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->st = user;
    }
};

// n sweeps of the subsets in slots [sl0, sl1) (a stage, or one subset), batched.
bmf_status run_batch(bmf_ctx *c, int sl0, int sl1, int n_sweeps, const bmf_draws *draws,
                     bmf_sweep_stats *stats)
{
    if (c->failed) return fail(c, BMF_E_STATE, "context is in a failed state; call bmf_set_state");
    if (n_sweeps < 0) return fail(c, BMF_E_ARG, "n_sweeps < 0");
    const int K = c->K;
    const SubsetGeom &g0 = geom_of_slot(c, sl0), &gl = geom_of_slot(c, sl1 - 1);
    const int64_t t_start = c->ss[g0.sid].t;
    for (int sl = sl0; sl < sl1; ++sl)
        if (c->ss[geom_of_slot(c, sl).sid].t != t_start)
            return fail(c, BMF_E_STATE, "subsets of the batch are at different sweep counts");
    const int64_t rx0 = g0.xoff, rx1 = gl.xoff + gl.n();
    const int64_t rw0 = g0.woff, rw1 = gl.woff + gl.d();
    const int64_t tt0 = g0.test_off, tt1 = gl.test_off + gl.n_test;
    // the per-sweep test-RMSE monitor (held-out entries of the batch, current sample and
    // running mean of the retained samples)
    const bool mon = c->monitor && tt1 > tt0;
    const int64_t per = per_sweep_draws(c, sl0, sl1);
    const double *dr = nullptr;
    // host draw buffers are copied on the generator stream (idle with host draws) in groups of
    // sweeps -- 1, 2, 4, ..., 32, then equal groups, at most kCopyGroups -- and each sweep's readers
    // wait only for their group, so the copy of later sweeps overlaps the sweeps; the graph
    // schedule (which would have to finish the copy before its launch) is not used then
    const bool host_draws = draws && !draws->on_device && n_sweeps > 0;
    const bool use_graph = c->sched.graph && !c->prof && n_sweeps > 0 && !host_draws;
    const bool copy_async = host_draws;
    std::vector<int64_t> gsweep;   // first sweep of each group, then n_sweeps
    if (copy_async) {
        gsweep.push_back(0);
        int64_t step = 1;
        while (gsweep.back() < n_sweeps) {
            const int left = kCopyGroups - 1 - (int)gsweep.size();   // one group for the first hyper blocks
            int64_t next = gsweep.back() + step;
            if (left <= 1 || next > n_sweeps) next = n_sweeps;
            gsweep.push_back(next);
            if (step < 32) step *= 2;
            else step = std::max<int64_t>(step, (n_sweeps - next + left - 2) / std::max(1, left - 1));
        }
    }
    // group boundaries in doubles: the first sweep's hyperparameter blocks alone (the call's
    // first hyperparameter draws read only them), then the groups of sweeps
    const int64_t first_hyper = 2 * (int64_t)(sl1 - sl0) * hyper_block_len(K);
    std::vector<int64_t> goff;
    if (copy_async) {
        goff.push_back(0);
        goff.push_back(first_hyper);
        for (size_t q = 1; q < gsweep.size(); ++q) goff.push_back(gsweep[q] * per);
    }
    bmf_status s = stage_draws(c, draws, per * n_sweeps, &dr, copy_async ? c->st5 : c->st,
                               copy_async ? &goff : nullptr, c->ev_copyq);
    if (s) return s;
    // a reader of the draws up to offset `need` (exclusive) on stream sx waits for the group
    // holding it (once per group and stream)
    cudaStream_t wst[3] = {nullptr, nullptr, nullptr};
    int wgot[3] = {-1, -1, -1};
    auto wait_upto = [&](cudaStream_t sx, int64_t need) -> bmf_status {
        if (!copy_async) return BMF_OK;
        int q = 0;
        while (goff[q + 1] < need) ++q;
        int k = 0;
        while (k < 3 && wst[k] && wst[k] != sx) ++k;
        if (k == 3) return fail(c, BMF_E_STATE, "internal: too many draw-reading streams");
        wst[k] = sx;
        if (q > wgot[k]) {
            CUDA_TRY(c, cudaStreamWaitEvent(sx, c->ev_copyq[q], 0));
            wgot[k] = q;
        }
        return BMF_OK;
    };
    // sweep it's hyperparameter blocks, and the whole sweep (its z's and noise variates)
    auto wait_hyper = [&](cudaStream_t sx, int64_t it) { return wait_upto(sx, it * per + first_hyper); };
    auto wait_draws = [&](cudaStream_t sx, int64_t it) { return wait_upto(sx, (it + 1) * per); };
    // the caller's host buffer is read until the copy completes: never return before that
    struct CopyWait {
        cudaStream_t st;
        bool on;
        ~CopyWait()
        {
            if (on) cudaStreamSynchronize(st);
        }
    } copy_wait{c->st5, copy_async};
    // with the device generator, sweep it's draws live in ring buffer it % 2: the main stream
    // fills sweep it + 2 after sweep it's conditionals, which are ordered after every reader
    // of that buffer (the side stream's hyperparameter draw of sweep it finishes before them)
    const bool gen = dr == nullptr;
    int64_t gen_units = 0;
    int gen_segs = 0;
    if (gen && n_sweeps > 0) {
        if ((s = prepare_gen(c, sl0, sl1, per, 2, &gen_units, &gen_segs))) return s;
        for (int it = 0; it < std::min(n_sweeps, 2); ++it)
            enqueue_gen(c, gen_units, gen_segs, t_start + it + 1, c->gen_d + (int64_t)it * per);
    }
    auto draws_of = [&](int it) -> const double * {
        return gen ? c->gen_d + (int64_t)(it & 1) * per : dr + (int64_t)it * per;
    };
    const std::vector<int64_t> bounds[2] = {
        chunk_bounds(c, c->X, c->X.slot_blk[sl0], c->X.slot_blk[sl1], c->sched.chunks_x, rx1),
        chunk_bounds(c, c->W, c->W.slot_blk[sl0], c->W.slot_blk[sl1], c->sched.chunks_w, rw1)};
    const size_t pbytes = c->prec == BMF_FP64 ? 8 : 4;
    const int gram_grid = c->sms * std::max(1, c->sched.gram_blocks_per_sm);
    // hyperparameter jobs: every factor block without a per-row prior (X jobs first).  A job
    // sums the statistics slots of its subset's conditional-kernel blocks, which the standalone
    // statistics pass fills before the first sweep and the conditional kernel refreshes after.
    std::vector<HyperJob> jobs;
    const int64_t HB = hyper_block_len(K);
    int nj[2] = {0, 0};
    for (int f = 0; f < 2; ++f) {
        const Side &sd = f == 0 ? c->X : c->W;
        const size_t j0 = jobs.size();
        for (int sl = sl0; sl < sl1; ++sl) {
            const SubsetGeom &g = geom_of_slot(c, sl);
            if (c->ss[g.sid].prior[f]) continue;
            HyperJob jb;
            jb.chunk0 = (int32_t)(sd.stat0 + sd.slot_blk[sl]);
            jb.chunk1 = (int32_t)(sd.stat0 + sd.slot_blk[sl + 1]);
            jb.slot = 2 * sl + f;
            jb.draw = (int32_t)((2 * (sl - sl0) + f) * HB);
            jb.n = f == 0 ? g.n() : g.d();
            jobs.push_back(jb);
        }
        nj[f] = (int)(jobs.size() - j0);
    }
    if ((int64_t)jobs.size() > kHyperJobsMax)
        return fail(c, BMF_E_ARG, "internal: too many hyperparameter jobs");
    const bool same_jobs = jobs.size() == c->jobs_up.size() &&
                           std::memcmp(jobs.data(), c->jobs_up.data(), jobs.size() * sizeof(HyperJob)) == 0;
    if (!jobs.empty() && !same_jobs) {
        CUDA_TRY(c, cudaMemcpyAsync(c->d_jobs, jobs.data(), jobs.size() * sizeof(HyperJob),
                                    cudaMemcpyHostToDevice, c->st));
        std::vector<HyperJob> jobs2(jobs);
        for (size_t q = 0; q < jobs2.size(); ++q) {
            jobs2[q].chunk0 = (int32_t)(q * kStatParts);
            jobs2[q].chunk1 = (int32_t)((q + 1) * kStatParts);
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->d_jobs2, jobs2.data(), jobs2.size() * sizeof(HyperJob),
                                    cudaMemcpyHostToDevice, c->st));
        c->jobs_up = jobs;
    }
    const int64_t hyper_len = 2 * (int64_t)(sl1 - sl0) * HB;
    const int64_t zx_len = (rx1 - rx0) * K;
    const int64_t zw_len = (rw1 - rw0) * K;
    if (c->noise && n_sweeps > 0) {
        // each subset's W rows and the offset of its noise variates in a sweep's draws
        c->h_noise_blocks.clear();
        int64_t off = hyper_len + zx_len + zw_len;
        for (int sl = sl0; sl < sl1; ++sl) {
            const SubsetGeom &g = geom_of_slot(c, sl);
            c->h_noise_blocks.push_back(NoiseBlock{g.woff, g.woff + g.d(), off});
            off += c->noise == BMF_NOISE_COLUMN ? g.d() : 1;
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->noise_blocks, c->h_noise_blocks.data(),
                                    c->h_noise_blocks.size() * sizeof(NoiseBlock),
                                    cudaMemcpyHostToDevice, c->st));
    }
    // the row-side Gram's copies scaled by the current noise precisions
    auto noise_scale = [&]() {
        launch_noise_scale(K, c->prec, rw0, rw1, c->tau_w, c->W.F, c->Ws, c->ldg, c->X.h_obs[rx0],
                           c->X.h_obs[rx1], c->X.idx, c->xval_orig, c->X.val, c->st);
    };
    int64_t kept = c->ss[g0.sid].kept;
    // the DM / GMM summaries keep every retained sample: the ring must hold this call's
    bool any_mix[2] = {false, false};
    for (int sl = sl0; sl < sl1; ++sl)
        for (int f = 0; f < 2; ++f) any_mix[f] = any_mix[f] || c->ss[geom_of_slot(c, sl).sid].mix[f];
    if (c->summary != BMF_SUMMARY_MM) {
        int64_t k2 = kept;
        for (int it = 0; it < n_sweeps; ++it) k2 += keep_sample(c, t_start + it + 1) ? 1 : 0;
        if (k2 > c->max_samples)
            return fail(c, BMF_E_STATE, "the call would retain " + std::to_string(k2) +
                                            " samples per chain; max_samples is " +
                                            std::to_string(c->max_samples));
    }
    // (mu, Lambda) | factor for sweep `it`, on the side stream.  The statistics of X for sweep
    // it+1 depend only on the X written by sweep it, so they run while the main stream does
    // W | X of sweep it and the Gram pass of sweep it+1 (and symmetrically for W).
    auto side_hyper = [&](int f, int it) -> bmf_status {
        const double *d = draws_of(it);
        if (bmf_status sw = wait_hyper(c->st2, it)) return sw;
        if (gen && it >= 2) CUDA_TRY(c, cudaStreamWaitEvent(c->st2, c->ev_gen[it & 1], 0));
        const int j0 = f == 0 ? 0 : nj[0];
        HyperParams hp{K, c->d_jobs2 + j0, nj[f], c->stats2, c->mu0_d, c->beta0, c->nu0,
                       c->W0inv_d, d, c->hyper, c->err_d};
        traced(c, c->st2, K_HYPER, 2, [&] {
            launch_stats_reduce(K, c->d_jobs + j0, nj[f], j0, c->stats, c->stats2, c->st2);
            launch_hyper(hp, c->st2);
        });
        CUDA_TRY(c, cudaEventRecord(c->ev_hyp[f], c->st2));
        return BMF_OK;
    };
    const bool hyp[2] = {nj[0] > 0, nj[1] > 0};
    bool used_tail = false, used_gen = false;
    // graph schedule: the whole launch sequence of the call (all streams) is captured into one
    // CUDA graph and launched once (the executable graph is kept and updated in place when the
    // next call has the same shape)
    CaptureGuard capture;
    if (use_graph) {
        capture.c = c;
        capture.user = c->st;
        const cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(c->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(c->cap, &g);
                if (g) cudaGraphDestroy(g);
            }
            return fail(c, BMF_E_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(e));
        }
        c->st = c->cap;
        capture.active = true;
    }
    if (n_sweeps > 0 && (hyp[0] || hyp[1])) {
        // statistics of the state at the start of the call, unless the last sweep of these
        // slots left them current (the conditional kernel keeps them current from then on)
        CUDA_TRY(c, cudaEventRecord(c->ev_fork, c->st));
        CUDA_TRY(c, cudaStreamWaitEvent(c->st2, c->ev_fork, 0));
        bool current = true;
        for (int sl = sl0; sl < sl1; ++sl) current = current && c->stats_ok[sl];
        for (int f = 0; f < 2; ++f) {
            if (!hyp[f] || current) continue;
            const Side &sd = f == 0 ? c->X : c->W;
            const int64_t b0 = sd.slot_blk[sl0], b1 = sd.slot_blk[sl1];
            traced(c, c->st2, K_STATS, 1, [&] {
                launch_stats(K, sd.chunks + b0, (int)(b1 - b0), c->X.F, c->W.F, c->stats, c->st2);
            });
        }
        for (int f = 0; f < 2; ++f)
            if (hyp[f] && (s = side_hyper(f, 0))) return s;
    }
    // from here the batch's statistics are in flux until the call completes
    for (int sl = sl0; sl < sl1 && n_sweeps > 0; ++sl) c->stats_ok[sl] = 0;
    if (c->noise && n_sweeps > 0) noise_scale();
    for (int it = 0; it < n_sweeps; ++it) {
        const double *d = draws_of(it);
        const int64_t t = t_start + it + 1;
        const bool keep = keep_sample(c, t);
        if (keep) ++kept;
        // X | W, then W | X
        for (int f = 0; f < 2; ++f) {
            Side &me = f == 0 ? c->X : c->W;
            Side &other = f == 0 ? c->W : c->X;
            const int64_t r0 = f == 0 ? rx0 : rw0, r1 = f == 0 ? rx1 : rw1;
            const int64_t i0 = me.h_item_ptr[r0], i1 = me.h_item_ptr[r1];
            GramParams gp;
            gp.K = K;
            gp.tasks = me.tasks + me.slot_task[sl0];
            gp.n_tasks = me.slot_task[sl1] - me.slot_task[sl0];
            gp.items = me.items + i0;
            gp.n_items = i1 - i0;
            gp.idx = me.idx;
            gp.val = me.val;
            gp.P = (c->noise && f == 0) ? c->Ws : other.G;
            gp.ldP = c->ldg;
            gp.part = c->part;
            gp.ld = c->ld_part;
            gp.multi_idx = me.multi_idx;
            gp.item_ptr = me.item_ptr;
            gp.item0 = i0;
            gp.counters = me.counters;
            gp.nparts = part_parts(K, c->prec);
            gp.rowsum = me.rowsum;
            gp.ld_sum = part_nv(K);
            gp.nv = part_nv(K);
            const int64_t b0 = me.slot_blk[sl0], b1 = me.slot_blk[sl1];
            // Gram pass over the rows of conditional blocks [ba, bb)
            auto gram_chunk = [&](int64_t ba, int64_t bb) {
                GramParams g = gp;
                if (K > kNarrowMaxK) {
                    const int64_t ia = ba == b1 ? i1 : me.h_item_ptr[me.h_blocks[ba].row0];
                    const int64_t ib = bb == b1 ? i1 : me.h_item_ptr[me.h_blocks[bb].row0];
                    g.items = me.items + ia;
                    g.n_items = ib - ia;
                    g.item0 = ia;
                    g.part = static_cast<char *>(c->part) + (ia - i0) * c->ld_part * pbytes;
                    if (g.n_items > 0)
                        traced(c, c->st, f == 0 ? K_GRAM_X : K_GRAM_W, 1,
                               [&] { launch_gram_wide(K, c->prec, g, gram_grid, c->st, c->tf32); });
                } else {
                    g.tasks = me.tasks + me.blk_task[ba];
                    g.n_tasks = me.blk_task[bb] - me.blk_task[ba];
                    if (g.n_tasks > 0)
                        traced(c, c->st, f == 0 ? K_GRAM_X : K_GRAM_W, 1,
                               [&] { launch_gram(K, c->prec, g, gram_grid, c->st); });
                }
            };
            const std::vector<int64_t> &B = bounds[f];
            const int nch = (int)B.size() - 1;
            cudaStream_t cs = nch == 1 ? c->st : c->st3;
            if (any_mix[f]) {
                // propagated mixture priors: each row's component from its current value,
                // installed as its prior before this half's draws
                MixChooseParams mp{K, c->ncomp, r0, r1 - r0, me.R, c->mix[f], c->has_mix[f], me.F,
                                   me.pL, me.pb, nullptr, c->err_d};
                traced(c, c->st, f == 0 ? K_COND_X : K_COND_W, 1, [&] { launch_mix_choose(mp, c->st); });
            }
            if (nch == 1) gram_chunk(b0, b1);
            if (f == 0) {
                // the previous sweep's RMSE pass reads the gathered copies this sweep rewrites;
                // the generator fills this sweep's draws on the tail stream
                if (it > 0 && mon) CUDA_TRY(c, cudaStreamWaitEvent(cs, c->ev_rmse, 0));
                if ((s = wait_draws(cs, it))) return s;
                if (gen && it >= 2) CUDA_TRY(c, cudaStreamWaitEvent(cs, c->ev_gen[it & 1], 0));
            }
            if (nch == 1) {
                if (hyp[f]) CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->ev_hyp[f], 0));
            } else {
                // chunked schedule: the Gram passes run in order on the main stream, lightest
                // rows first (rows are in decreasing degree order); each chunk's conditional
                // follows on the conditional stream as soon as its Gram pass is done, so the
                // FP64-bound conditional of one chunk overlaps the gather-bound Gram pass of the
                // next
                for (int q = nch - 1; q >= 0; --q) {
                    gram_chunk(B[q], B[q + 1]);
                    CUDA_TRY(c, cudaEventRecord(c->ev_chunk[q], c->st));
                }
                if (hyp[f]) CUDA_TRY(c, cudaStreamWaitEvent(c->st3, c->ev_hyp[f], 0));
            }
            CondParams cp;
            cp.K = K;
            cp.blocks = me.blocks + b0;
            cp.blk0 = me.stat0 + b0;
            cp.row0 = r0;
            cp.row1 = r1;
            cp.item_ptr = me.item_ptr;
            cp.item0 = i0;
            cp.part = c->part;
            cp.ld = c->ld_part;
            cp.part_rhs = part_rhs_of(K);
            cp.multi_idx = me.multi_idx;
            cp.rowsum = me.rowsum;
            cp.ld_sum = part_nv(K);
            // sampled noise: the row side has the precisions in its Gram sums (scaled copies),
            // the column side takes each column's own
            cp.tau = c->noise ? 1.0 : c->tau;
            cp.tau_row = (c->noise && f == 1) ? c->tau_w : nullptr;
            cp.row_hslot = me.hslot;
            cp.hyper = c->hyper;
            cp.prior_L = me.pL;
            cp.prior_b = me.pb;
            cp.R = me.R;
            cp.z = d + hyper_len + (f == 0 ? 0 : zx_len);
            cp.X = me.F;
            cp.Xg = me.G;
            cp.ldg = c->ldg;
            cp.keep = keep ? 1 : 0;
            cp.full = c->full_moments ? 1 : 0;
            cp.S1 = me.S1;
            cp.S2 = me.S2;
            cp.stats = c->stats;
            cp.err = c->err_d;
            cp.obs_ptr = me.ptr;
            cp.obs_idx = me.idx;
            cp.obs_val = me.val;
            cp.P = gp.P;
            cp.ldP = gp.ldP;
            // lanes per row of the conditional: one thread per row below K = 13, a team above
            const int team = K >= kTeamMinK
                                 ? (c->sched.cond_lanes > 0 ? c->sched.cond_lanes : cond_team_size(K))
                                 : 1;
            auto cond_chunk = [&](int64_t ba, int64_t bb, cudaStream_t sx) {
                if (bb <= ba) return;
                CondParams q = cp;
                q.blocks = me.blocks + ba;
                q.blk0 = me.stat0 + ba;
                traced(c, sx, f == 0 ? K_COND_X : K_COND_W, 1, [&] {
                    // two lanes per row: the register-resident kernel where it exists
                    if (team == 2 && launch_cond_pair(c->prec, q, (int)(bb - ba), sx)) return;
                    if (team > 1)
                        launch_cond_team(c->prec, q, (int)(bb - ba), team, sx);
                    else
                        launch_cond(c->prec, q, (int)(bb - ba), sx);
                });
            };
            if (nch == 1) {
                cond_chunk(b0, b1, c->st);
            } else {
                for (int q = nch - 1; q >= 0; --q) {
                    CUDA_TRY(c, cudaStreamWaitEvent(c->st3, c->ev_chunk[q], 0));
                    cond_chunk(B[q], B[q + 1], c->st3);
                }
                CUDA_TRY(c, cudaEventRecord(c->ev_cdone, c->st3));
                CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->ev_cdone, 0));
            }
            if (keep && c->summary != BMF_SUMMARY_MM && r1 > r0)
                CUDA_TRY(c, cudaMemcpyAsync(c->ring[f] + (kept - 1) * me.R * K + r0 * K, me.F + r0 * K,
                                            (size_t)(r1 - r0) * K * sizeof(double),
                                            cudaMemcpyDeviceToDevice, c->st));
            if (c->noise && f == 1) {
                // the noise precisions given the new X and W, then the scaled copies of the
                // next sweep's row-side Gram
                launch_noise_sse(K, rw0, rw1, c->W.ptr, c->W.idx, c->W.val, c->prec, c->X.F, c->W.F,
                                 c->noise_sse, c->st);
                launch_noise_tau(c->noise, c->noise_b0, c->noise_blocks, sl1 - sl0, d, c->noise_sse,
                                 c->tau_w, c->st);
                noise_scale();
                c->launches += 3;
            }
            if (hyp[f] && it + 1 < n_sweeps) {
                CUDA_TRY(c, cudaEventRecord(c->ev_fac[f], c->st));
                CUDA_TRY(c, cudaStreamWaitEvent(c->st2, c->ev_fac[f], 0));
                if ((s = side_hyper(f, it + 1))) return s;
            }
        }
        // tail of the sweep on two streams, overlapping the next sweep's Gram pass (which
        // leaves the FP64 pipes idle): the test RMSE of this sample, and the draws of sweep
        // t + 2 into this sweep's buffer (every reader of that buffer is ordered before here)
        const bool tail_gen = gen && it + 2 < n_sweeps;
        used_tail |= mon;
        used_gen |= tail_gen;
        if (mon || tail_gen) CUDA_TRY(c, cudaEventRecord(c->ev_tail, c->st));
        if (mon) CUDA_TRY(c, cudaStreamWaitEvent(c->st4, c->ev_tail, 0));
        if (tail_gen) CUDA_TRY(c, cudaStreamWaitEvent(c->st5, c->ev_tail, 0));
        if (mon) {
            RmseParams rp{K, c->prec, tt0, tt1, c->trow, c->tcol, c->tval, c->X.G, c->W.G, c->ldg,
                          keep ? 1 : 0, c->ysum, kept > 0 ? 1.0 / (double)kept : 0.0,
                          c->rmse_part};
            traced(c, c->st4, K_RMSE, 2, [&] {
                launch_rmse(rp, c->rmse_blocks, c->st4);
                launch_rmse_final(c->rmse_part, c->rmse_blocks, c->rmse_out, c->st4);
            });
            CUDA_TRY(c, cudaEventRecord(c->ev_rmse, c->st4));
        }
        if (tail_gen) {
            GenParams gp{c->gen_segs_d, gen_segs, gen_units, c->seed, t + 2,
                         c->gen_d + (int64_t)(it & 1) * per, c->W.ptr, c->err_d};
            traced(c, c->st5, K_GEN, 1, [&] { launch_gen(gp, c->st5); });
            CUDA_TRY(c, cudaEventRecord(c->ev_gen[it & 1], c->st5));
        }
    }
    // the context stream is complete when the call returns
    // (only streams this call used: under the graph schedule the others are not part of the
    // capture)
    if (used_tail) {
        CUDA_TRY(c, cudaEventRecord(c->ev_tail, c->st4));
        CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->ev_tail, 0));
    }
    if (used_gen) {
        CUDA_TRY(c, cudaEventRecord(c->ev_tail2, c->st5));
        CUDA_TRY(c, cudaStreamWaitEvent(c->st, c->ev_tail2, 0));
    }
    if (use_graph) {
        cudaGraph_t g = nullptr;
        capture.active = false;
        const cudaError_t ee = cudaStreamEndCapture(c->st, &g);
        c->st = capture.user;
        if (ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(c, BMF_E_CUDA, std::string("stream capture failed: ") + cudaGetErrorString(ee));
        }
        cudaGraphExec_t *ge = nullptr;
        for (auto &q : c->graphs)
            if (q.sl0 == sl0 && q.sl1 == sl1) ge = &q.exec;
        if (!ge) {
            c->graphs.push_back(bmf_ctx::GraphEntry{sl0, sl1, nullptr});
            ge = &c->graphs.back().exec;
        }
        bool updated = false;
        if (*ge) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(*ge, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(*ge);
                *ge = nullptr;
            }
        }
        cudaError_t e = updated ? cudaSuccess : cudaGraphInstantiate(ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            *ge = nullptr;
            return fail(c, BMF_E_CUDA, std::string("graph instantiation failed: ") + cudaGetErrorString(e));
        }
        CUDA_TRY(c, cudaGraphLaunch(*ge, c->st));
    }
    CUDA_TRY(c, cudaGetLastError());
    for (int sl = sl0; sl < sl1; ++sl) {
        SubState &su = c->ss[geom_of_slot(c, sl).sid];
        su.t = t_start + n_sweeps;
        su.kept = kept;
        su.finalized = false;
        if (n_sweeps > 0) c->stats_ok[sl] = 1;
    }
    // every stream of the call has joined the context stream: one readback, one synchronisation
    const bool want_rmse = stats && mon && n_sweeps > 0;
    CUDA_TRY(c, cudaMemcpyAsync(&c->rb->err, c->err_d, sizeof(DevError), cudaMemcpyDeviceToHost, c->st));
    if (want_rmse)
        CUDA_TRY(c, cudaMemcpyAsync(c->rb->rmse, c->rmse_out, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    s = dev_error_status(c, c->rb->err);
    if (s)
        for (int sl = sl0; sl < sl1; ++sl) c->stats_ok[sl] = 0;
    if (c->prof) collect_profile(c);
    if (s) return s;
    if (stats) {
        stats->sweeps = t_start + n_sweeps;
        stats->kept = kept;
        stats->rmse_sample = stats->rmse_mean = NAN;
        if (want_rmse) {
            const double n = (double)(tt1 - tt0);
            stats->rmse_sample = std::sqrt(c->rb->rmse[0] / n);
            if (kept > 0) stats->rmse_mean = std::sqrt(c->rb->rmse[1] / n);
        }
    }
    return BMF_OK;
}

// The summary of one subset's posterior that propagates and aggregates (Section 4.1): moment
// matching of the moment sums, or the dominant mode / mixture of the retained samples.
// Enqueued on the context stream; the caller checks the device error word.
bmf_status finalize_subset(bmf_ctx *c, int sid)
{
    const SubsetGeom &g = c->P.subs[sid];
    SubState &su = c->ss[sid];
    if (su.finalized) return BMF_OK;
    if (su.kept < 1)
        return fail(c, BMF_E_STATE, "subset " + std::to_string(g.sid) +
                                        " has no retained samples (burn-in not passed)");
    if (c->summary != BMF_SUMMARY_MM) {
        for (int f = 0; f < 2; ++f) {
            Side &sd = f == 0 ? c->X : c->W;
            SummaryParams sp{};
            sp.K = c->K;
            sp.S = (int)su.kept;
            sp.C = c->summary == BMF_SUMMARY_DM ? 1 : c->ncomp;
            sp.mode = c->summary;
            sp.lambda = c->lambda;
            sp.samples = c->ring[f];
            sp.sample_stride = sd.R * c->K;
            sp.row0 = f == 0 ? g.xoff : g.woff;
            sp.n_rows = f == 0 ? g.n() : g.d();
            sp.mm_mu = sd.mm_mu;
            sp.mm_L = sd.mm_L;
            sp.mm_b = sd.mm_b;
            sp.mix = c->summary == BMF_SUMMARY_GMM ? c->mix[f] : nullptr;
            sp.R = sd.R;
            sp.err = c->err_d;
            launch_summary(sp, c->st);
        }
        su.finalized = true;
        return BMF_OK;
    }
    if (!c->full_moments)
        return fail(c, BMF_E_STATE, "moment matching needs second moments (moments mode)");
    if (su.kept < c->K + 1)
        return fail(c, BMF_E_STATE, "subset " + std::to_string(g.sid) + " has " +
                                        std::to_string(su.kept) + " retained samples; moment "
                                        "matching needs at least K + 1 (a full-rank covariance)");
    for (int f = 0; f < 2; ++f) {
        Side &sd = f == 0 ? c->X : c->W;
        MMParams mp{c->K, f == 0 ? g.xoff : g.woff, f == 0 ? g.xoff + g.n() : g.woff + g.d(),
                    sd.R, sd.S1, sd.S2, (double)su.kept, sd.mm_mu, sd.mm_L, sd.mm_b, c->err_d};
        launch_mm(mp, c->st);
    }
    su.finalized = true;
    return BMF_OK;
}

// The summaries of every subset of a stage.
bmf_status finalize_stage(bmf_ctx *c, int stage)
{
    int sl0, sl1;
    if (!stage_slots(c, stage, sl0, sl1)) return BMF_OK;
    // moment matching of a whole stage in one launch per factor when its subsets are alike (the
    // stage's rows are contiguous in each arena; a launch per subset leaves most SMs idle on
    // small subsets)
    bool batch = c->summary == BMF_SUMMARY_MM && c->full_moments && sl1 - sl0 > 1;
    const int64_t kept0 = c->ss[geom_of_slot(c, sl0).sid].kept;
    for (int sl = sl0; sl < sl1 && batch; ++sl) {
        const SubState &su = c->ss[geom_of_slot(c, sl).sid];
        batch = !su.finalized && su.kept == kept0 && kept0 >= c->K + 1;
    }
    if (batch) {
        const SubsetGeom &ga = geom_of_slot(c, sl0), &gb = geom_of_slot(c, sl1 - 1);
        for (int f = 0; f < 2; ++f) {
            Side &sd = f == 0 ? c->X : c->W;
            MMParams mp{c->K, f == 0 ? ga.xoff : ga.woff, f == 0 ? gb.xoff + gb.n() : gb.woff + gb.d(),
                        sd.R, sd.S1, sd.S2, (double)kept0, sd.mm_mu, sd.mm_L, sd.mm_b, c->err_d};
            launch_mm(mp, c->st);
        }
        for (int sl = sl0; sl < sl1; ++sl) c->ss[geom_of_slot(c, sl).sid].finalized = true;
    }
    for (int sl = sl0; sl < sl1 && !batch; ++sl) {
        bmf_status s = finalize_subset(c, geom_of_slot(c, sl).sid);
        if (s) return s;
    }
    CUDA_TRY(c, cudaGetLastError());
    return check_dev_error(c);
}

bmf_status install_prior_from(bmf_ctx *c, int dst_sid, int f, int src_sid)
{
    const SubsetGeom &gd = c->P.subs[dst_sid], &gs = c->P.subs[src_sid];
    Side &sd = f == 0 ? c->X : c->W;
    const int64_t n = f == 0 ? gd.n() : gd.d();
    PropParams pp{c->K, n, f == 0 ? gs.xoff : gs.woff, f == 0 ? gd.xoff : gd.woff, sd.R,
                  sd.mm_mu, sd.mm_L, sd.mm_b, sd.pL, sd.pb, sd.F, sd.G, c->ldg, c->prec};
    launch_propagate(pp, c->st);
    c->ss[dst_sid].prior[f] = 1;
    if (c->summary == BMF_SUMMARY_GMM && n > 0) {
        // the source rows' mixture becomes the destination rows' prior; each draw picks its
        // component (the chain starts at the pooled mean set above)
        const int64_t W = mix_width(c->K), src0 = f == 0 ? gs.xoff : gs.woff,
                      dst0 = f == 0 ? gd.xoff : gd.woff;
        CUDA_TRY(c, cudaMemcpyAsync(c->mix[f] + dst0 * c->ncomp * W, c->mix[f] + src0 * c->ncomp * W,
                                    (size_t)n * c->ncomp * W * sizeof(double), cudaMemcpyDeviceToDevice,
                                    c->st));
        CUDA_TRY(c, cudaMemsetAsync(c->has_mix[f] + dst0, 1, (size_t)n, c->st));
        c->ss[dst_sid].mix[f] = 1;
    }
    c->stats_ok[gd.slot] = 0;    // the propagated factor starts at the propagated mean
    refresh_hslots(c, gd.slot);
    return upload_hslots(c, gd.slot);
}

// Open `stage` (Algorithm 1): finalise the previous stage and install the propagated priors.
bmf_status open_stage(bmf_ctx *c, int stage)
{
    if (stage == c->stage_open) return BMF_OK;
    if (stage != c->stage_open + 1)
        return fail(c, BMF_E_STATE, "stages must be opened in order (open: " +
                                        std::to_string(c->stage_open) + ", requested: " +
                                        std::to_string(stage) + ")");
    int sl0, sl1;
    if (!stage_slots(c, stage, sl0, sl1))
        return fail(c, BMF_E_STATE, "stage " + std::to_string(stage) + " has no subsets");
    if (stage > 1 && !c->independent) {
        bmf_status s = finalize_stage(c, stage - 1);
        if (s) return s;
        const int J = c->P.J;
        for (int sl = sl0; sl < sl1; ++sl) {
            const SubsetGeom &g = geom_of_slot(c, sl);
            if (stage == 2) {
                if (g.j == 0)
                    s = install_prior_from(c, g.sid, 1, 0);      // W^(0) from (0,0)
                else
                    s = install_prior_from(c, g.sid, 0, 0);      // X^(0) from (0,0)
            } else {
                s = install_prior_from(c, g.sid, 0, g.i * J);    // X^(i) from (i,0)
                if (!s) s = install_prior_from(c, g.sid, 1, g.j);  // W^(j) from (0,j)
            }
            if (s) return s;
        }
        CUDA_TRY(c, cudaGetLastError());
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    c->stage_open = stage;
    return BMF_OK;
}

int last_stage(const bmf_ctx *c)
{
    int m = 0;
    for (const auto &g : c->P.subs) m = std::max(m, g.stage);
    return m;
}

// Aggregated means (reordered order) into c->aggX / c->aggW: Eq. 14 with Algorithm 2 for every
// row block of X (submodels (i, 0..J-1)) and column block of W (submodels (0..I-1, j)); a block
// with a single submodel takes the mean of its retained samples.  All launches are enqueued on
// the context stream, then one synchronisation reads the device error word.
bmf_status aggregate_all(bmf_ctx *c, int64_t *n_corrected)
{
    if (c->stage_open != last_stage(c))
        return fail(c, BMF_E_STATE, "every stage must be run before prediction");
    bmf_status s = BMF_OK;
    const int I = c->P.I, J = c->P.J, K = c->K;
    bool single = (I == 1 && J == 1);
    if (!single) {
        // with propagation the earlier stages were summarised when the next one opened
        for (int st = c->independent ? 1 : c->stage_open; st <= c->stage_open; ++st) {
            s = finalize_stage(c, st);
            if (s) return s;
        }
    }
    CUDA_TRY(c, cudaMemsetAsync(c->ncorr_d, 0, sizeof(unsigned long long), c->st));
    int64_t nb_done = 0;   // launches so far (their bases are at agg_base + nb_done * max(I, J))
    const int MB = std::max(I, J);
    for (int f = 0; f < 2; ++f) {
        Side &sd = f == 0 ? c->X : c->W;
        const int nb = f == 0 ? I : J, ns = f == 0 ? J : I;
        for (int b = 0; b < nb; ++b, ++nb_done) {
            const SubsetGeom &g0 = f == 0 ? c->P.subs[b * J] : c->P.subs[b];
            const int64_t n = f == 0 ? g0.n() : g0.d();
            const int64_t out0 = f == 0 ? g0.r0 : g0.c0;
            double *out = (f == 0 ? c->aggX : c->aggW) + out0 * K;
            if (ns == 1) {
                // one submodel: the posterior mean is the mean of the retained samples
                const SubState &su = c->ss[g0.sid];
                if (su.kept < 1) return fail(c, BMF_E_STATE, "no retained samples");
                launch_mean_rows(K, n, sd.S1, sd.R, f == 0 ? g0.xoff : g0.woff,
                                 1.0 / (double)su.kept, out, c->st);
                continue;
            }
            if (n * (int64_t)(ns - 1) > (int64_t)INT32_MAX)
                return fail(c, BMF_E_SHAPE, "too many (row, submodel) pairs in one aggregation block");
            AggParams ap{K, n, ns, c->agg_base + nb_done * MB, sd.mm_mu, sd.mm_L, sd.R,
                         c->eps_rel, out, c->agg_corr, c->ncorr_d, c->err_d, c->agg_list,
                         c->agg_list_n};
            launch_aggregate(ap, c->st);
        }
    }
    CUDA_TRY(c, cudaGetLastError());
    s = check_dev_error(c);
    if (s) return s;
    if (n_corrected) {
        unsigned long long h = 0;
        CUDA_TRY(c, cudaMemcpy(&h, c->ncorr_d, sizeof(h), cudaMemcpyDeviceToHost));
        *n_corrected = (int64_t)h;
    }
    return BMF_OK;
}

// Aggregated means in the ORIGINAL order on the host.
bmf_status means_original(bmf_ctx *c, std::vector<double> &Xm, std::vector<double> &Wm,
                          int64_t *n_corrected)
{
    bmf_status s = aggregate_all(c, n_corrected);
    if (s) return s;
    const int K = c->K;
    std::vector<double> xr((size_t)c->P.N * K), wr((size_t)c->P.D * K);
    CUDA_TRY(c, cudaMemcpy(xr.data(), c->aggX, xr.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(wr.data(), c->aggW, wr.size() * sizeof(double), cudaMemcpyDeviceToHost));
    Xm.assign(xr.size(), 0.0);
    Wm.assign(wr.size(), 0.0);
    for (int64_t k = 0; k < c->P.N; ++k)
        std::memcpy(&Xm[(size_t)c->P.row_perm[k] * K], &xr[(size_t)k * K], K * sizeof(double));
    for (int64_t k = 0; k < c->P.D; ++k)
        std::memcpy(&Wm[(size_t)c->P.col_perm[k] * K], &wr[(size_t)k * K], K * sizeof(double));
    return BMF_OK;
}

// Every chain back to the stored initial state (the X0o / W0o copies): states and gathered
// copies, moment sums, running test predictions, hyperparameter slots, counters, priors and
// the open stage.  Enqueued on the context stream and synchronised.
bmf_status restart_chains(bmf_ctx *c)
{
    const int K = c->K, NT = ntri(K);
    const int S = (int)c->P.subs.size();
    launch_gather_rows(K, c->X.R, c->xsrc, c->X0o, c->X.F, c->st);
    launch_gather_rows(K, c->W.R, c->wsrc, c->W0o, c->W.F, c->st);
    launch_fill_gather(K, c->prec, c->X.R, c->X.F, c->X.G, c->ldg, c->st);
    launch_fill_gather(K, c->prec, c->W.R, c->W.F, c->W.G, c->ldg, c->st);
    for (Side *sd : {&c->X, &c->W}) {
        if (!sd->R) continue;
        CUDA_TRY(c, cudaMemsetAsync(sd->S1, 0, sd->R * K * sizeof(double), c->st));
        CUDA_TRY(c, cudaMemsetAsync(sd->S2, 0, sd->R * NT * sizeof(double), c->st));
        CUDA_TRY(c, cudaMemsetAsync(sd->pL, 0, sd->R * NT * sizeof(double), c->st));
        CUDA_TRY(c, cudaMemsetAsync(sd->pb, 0, sd->R * K * sizeof(double), c->st));
    }
    const int64_t nt = (int64_t)c->P.trow.size();
    if (nt) CUDA_TRY(c, cudaMemsetAsync(c->ysum, 0, nt * sizeof(double), c->st));
    CUDA_TRY(c, cudaMemsetAsync(c->hyper, 0, (size_t)2 * S * hyper_slot_len(K) * sizeof(double), c->st));
    for (int f = 0; f < 2; ++f)
        if (c->has_mix[f])
            CUDA_TRY(c, cudaMemsetAsync(c->has_mix[f], 0, (size_t)(f == 0 ? c->X.R : c->W.R), c->st));
    if (c->tau_w && c->W.R) {
        // every chain's noise precisions start at the configured tau
        const std::vector<double> t0((size_t)c->W.R, c->tau);
        CUDA_TRY(c, cudaMemcpyAsync(c->tau_w, t0.data(), t0.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, c->st));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
    }
    c->ss.assign(S, SubState());
    c->stats_ok.assign(S, 0);
    for (int sl = 0; sl < S; ++sl) {
        refresh_hslots(c, sl);
        bmf_status s = upload_hslots(c, sl);
        if (s) return s;
    }
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    c->failed = false;
    c->stage_open = 1;
    return BMF_OK;
}

// Room for n prediction entries (row, col int32; y and y_hat FP64) in c->pred_buf.
bmf_status pred_room(bmf_ctx *c, int64_t n)
{
    const int64_t need = n * (int64_t)(2 * sizeof(int32_t) + 2 * sizeof(double));
    if (need <= c->pred_cap) return BMF_OK;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (c->pred_buf) cudaFree(c->pred_buf);
    c->pred_buf = nullptr;
    c->pred_cap = 0;
    if (cudaMalloc(&c->pred_buf, need) != cudaSuccess)
        return fail(c, BMF_E_OOM, "device allocation failed (prediction entries)");
    c->pred_cap = need;
    return BMF_OK;
}

bool valid_subset(const bmf_ctx *c, int32_t s) { return s >= 0 && s < (int32_t)c->P.subs.size(); }

}  // namespace

namespace bmf {
void set_noctx_error(const char *m) { g_noctx_msg = m; }
}

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

bmf_status bmf_init(bmf_ctx **out, const bmf_config *cfg, int64_t N, int64_t D, int64_t nnz,
                    const int32_t *row, const int32_t *col, const double *val, int32_t I,
                    const int64_t *row_bounds, int32_t J, const int64_t *col_bounds,
                    const double *X0, const double *W0init, int64_t n_test,
                    const int32_t *test_row, const int32_t *test_col, const double *test_val,
                    void *stream)
{
    g_init_error.clear();
    g_noctx_msg = nullptr;
    if (!out || !cfg || !X0 || !W0init) {
        g_init_error = "null argument";
        return BMF_E_ARG;
    }
    *out = nullptr;
    const int K = cfg->K;
    if (K < 1 || K > BMF_MAX_K) {
        g_init_error = "K must be in 1..64";
        return BMF_E_ARG;
    }
    if (cfg->precision < BMF_FP64 || cfg->precision > BMF_TF32) {
        g_init_error = "unknown precision";
        return BMF_E_ARG;
    }
    if (!(cfg->tau > 0) || !(cfg->beta0 > 0) || cfg->thin < 1 || cfg->burnin < 0) {
        g_init_error = "need tau > 0, beta0 > 0, thin >= 1, burnin >= 0";
        return BMF_E_ARG;
    }
    double nu0 = cfg->nu0 > 0 ? cfg->nu0 : (double)K;
    if (!(nu0 > K - 1)) {
        g_init_error = "need nu0 > K - 1";
        return BMF_E_ARG;
    }
    bmf_ctx *c = new bmf_ctx();
    c->K = K;
    // single-pass TF32 is the FP32 storage and kernels with one product per wide Gram tile
    c->prec = cfg->precision == BMF_TF32 ? BMF_FP32 : cfg->precision;
    c->tf32 = cfg->precision == BMF_TF32;
    c->tau = cfg->tau;
    c->beta0 = cfg->beta0;
    c->nu0 = nu0;
    c->eps_rel = cfg->eps_rel > 0 ? cfg->eps_rel : 1e-6;
    c->burnin = cfg->burnin;
    c->thin = cfg->thin;
    c->seed = cfg->seed;
    c->st = static_cast<cudaStream_t>(stream);
    if (cfg->moments < BMF_MOMENTS_AUTO || cfg->moments > BMF_MOMENTS_FULL) {
        g_init_error = "unknown moments mode";
        delete c;
        return BMF_E_ARG;
    }
    c->full_moments = cfg->moments == BMF_MOMENTS_FULL || (cfg->moments == BMF_MOMENTS_AUTO && I * J > 1);
    if (cfg->summary < BMF_SUMMARY_MM || cfg->summary > BMF_SUMMARY_GMM) {
        g_init_error = "unknown summary";
        delete c;
        return BMF_E_ARG;
    }
    c->summary = cfg->summary;
    c->independent = cfg->independent != 0;
    if (cfg->noise < BMF_NOISE_FIXED || cfg->noise > BMF_NOISE_COLUMN ||
        (cfg->noise != BMF_NOISE_FIXED && (!(cfg->noise_a0 > 0.0) || !(cfg->noise_b0 > 0.0) ||
                                           !std::isfinite(cfg->noise_a0) || !std::isfinite(cfg->noise_b0)))) {
        g_init_error = "noise must be FIXED, GLOBAL or COLUMN, with a0 > 0 and b0 > 0 when sampled";
        delete c;
        return BMF_E_ARG;
    }
    c->noise = cfg->noise;
    c->noise_a0 = cfg->noise_a0;
    c->noise_b0 = cfg->noise_b0;
    if (c->summary != BMF_SUMMARY_MM) {
        c->ncomp = c->summary == BMF_SUMMARY_DM ? 1 : (cfg->components > 0 ? cfg->components : 3);
        c->lambda = cfg->lambda;
        c->max_samples = cfg->max_samples;
        std::string e;
        if (!(c->lambda > 0.0) || !std::isfinite(c->lambda)) e = "the DM / GMM summaries need lambda > 0";
        else if (c->ncomp < 1 || c->ncomp > BMF_MAX_COMPONENTS) e = "components must be in 1..4";
        else if (c->max_samples < 1) e = "the DM / GMM summaries need max_samples >= 1";
        else if (K > 32 || (int64_t)c->max_samples * K > 8192)
            e = "the DM / GMM summaries need K <= 32 and max_samples * K <= 8192";
        if (!e.empty()) {
            g_init_error = e;
            delete c;
            return BMF_E_ARG;
        }
    }
    c->mu0.assign(K, 0.0);
    if (cfg->mu0) std::memcpy(c->mu0.data(), cfg->mu0, K * sizeof(double));
    std::vector<double> W0((size_t)K * K, 0.0);
    if (cfg->W0)
        std::memcpy(W0.data(), cfg->W0, W0.size() * sizeof(double));
    else
        for (int k = 0; k < K; ++k) W0[k * K + k] = 1.0;
    if (!host_inverse(K, W0, c->W0inv)) {
        g_init_error = "W0 is singular";
        delete c;
        return BMF_E_ARG;
    }
    auto bail = [&](bmf_status s, const std::string &m) {
        g_init_error = m.empty() ? c->err : m;
        delete c;
        return s;
    };
    std::string err;
    int st = build_plan(N, D, nnz, row, col, val, cfg->order, cfg->center, I, row_bounds, J,
                        col_bounds, n_test, test_row, test_col, test_val, c->P, err);
    if (st) return bail((bmf_status)st, err);
    for (int64_t e = 0; e < N * K; ++e)
        if (!std::isfinite(X0[e])) return bail(BMF_E_NONFINITE, "non-finite X0");
    for (int64_t e = 0; e < D * K; ++e)
        if (!std::isfinite(W0init[e])) return bail(BMF_E_NONFINITE, "non-finite W0init");
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(BMF_E_CUDA, "no CUDA device");
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        bool ok = cudaStreamCreateWithPriority(&c->st2, cudaStreamNonBlocking, hi) == cudaSuccess;
        ok = ok && cudaStreamCreateWithPriority(&c->st3, cudaStreamNonBlocking, hi) == cudaSuccess;
        ok = ok && cudaStreamCreateWithPriority(&c->st4, cudaStreamNonBlocking, hi) == cudaSuccess;
        ok = ok && cudaStreamCreateWithPriority(&c->st5, cudaStreamNonBlocking, hi) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t *e : {&c->ev_fork, &c->ev_fac[0], &c->ev_fac[1], &c->ev_hyp[0], &c->ev_hyp[1],
                               &c->ev_cdone, &c->ev_tail, &c->ev_tail2, &c->ev_rmse, &c->ev_gen[0],
                               &c->ev_gen[1]})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        for (cudaEvent_t &e : c->ev_copyq)
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        for (cudaEvent_t &e : c->ev_chunk)
            ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaMallocHost(&c->rb, sizeof(*c->rb)) == cudaSuccess;
        if (!ok) return bail(BMF_E_CUDA, "stream/event creation failed");
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    c->ldg = gather_ld(K, c->prec);
    c->ld_part = part_ld_of(K, c->prec);
    bmf_status s = setup_side(c, c->X, c->P.RX, c->P.rptr, c->P.ridx, c->P.rval);
    if (!s) s = setup_side(c, c->W, c->P.RW, c->P.cptr, c->P.cidx, c->P.cval);
    if (s) return bail(s, "");
    // free the host copies of the lists
    std::vector<int64_t>().swap(c->P.rptr);
    std::vector<int32_t>().swap(c->P.ridx);
    std::vector<double>().swap(c->P.rval);
    std::vector<int64_t>().swap(c->P.cptr);
    std::vector<int32_t>().swap(c->P.cidx);
    std::vector<double>().swap(c->P.cval);
    const int S = I * J;
    const size_t pbytes = c->prec == BMF_FP64 ? 8 : 4;
    c->part = c->mem.alloc<char>(std::max<int64_t>(c->part_cap, 1) * c->ld_part * pbytes);
    c->hyper = c->mem.alloc<double>((size_t)2 * S * hyper_slot_len(K));
    // block tables (subset-aligned) and the statistics slots they fill
    for (int f = 0; f < 2; ++f) {
        Side &sd = f == 0 ? c->X : c->W;
        sd.slot_blk.assign(S + 1, 0);
        for (int sl = 0; sl < S; ++sl) {
            const SubsetGeom &g = geom_of_slot(c, sl);
            sd.slot_blk[sl] = (int64_t)sd.h_blocks.size();
            const int64_t base = f == 0 ? g.xoff : g.woff, n = f == 0 ? g.n() : g.d();
            for (int64_t q = 0; q < n; q += kCondBlock) {
                CondBlock b;
                b.row0 = base + q;
                b.n = (int32_t)std::min<int64_t>(kCondBlock, n - q);
                b.pad = 0;
                sd.h_blocks.push_back(b);
            }
        }
        sd.slot_blk[S] = (int64_t)sd.h_blocks.size();
    }
    c->W.stat0 = (int64_t)c->X.h_blocks.size();
    c->stats_cap = (int64_t)(c->X.h_blocks.size() + c->W.h_blocks.size());
    c->stats = c->mem.alloc<double>(c->stats_cap * (K + ntri(K)));
    c->d_jobs = c->mem.alloc<HyperJob>(kHyperJobsMax);
    c->d_jobs2 = c->mem.alloc<HyperJob>(kHyperJobsMax);
    c->stats2 = c->mem.alloc<double>((size_t)2 * S * kStatParts * (K + ntri(K)));
    for (int f = 0; f < 2; ++f) {
        Side &sd = f == 0 ? c->X : c->W;
        std::vector<StatChunk> ch(sd.h_blocks.size());
        for (size_t b = 0; b < ch.size(); ++b) {
            ch[b].r0 = sd.h_blocks[b].row0;
            ch[b].r1 = sd.h_blocks[b].row0 + sd.h_blocks[b].n;
            ch[b].out = (int32_t)(sd.stat0 + (int64_t)b);
            ch[b].arena = f;
        }
        sd.blocks = c->mem.alloc<CondBlock>(sd.h_blocks.size());
        sd.chunks = c->mem.alloc<StatChunk>(ch.size());
        if (!c->mem.ok) return bail(BMF_E_OOM, "device allocation failed (block tables)");
        if (!ch.empty()) {
            cudaMemcpy(sd.blocks, sd.h_blocks.data(), ch.size() * sizeof(CondBlock), cudaMemcpyHostToDevice);
            cudaMemcpy(sd.chunks, ch.data(), ch.size() * sizeof(StatChunk), cudaMemcpyHostToDevice);
        }
    }
    c->mu0_d = c->mem.alloc<double>(K);
    c->W0inv_d = c->mem.alloc<double>((size_t)K * K);
    const int64_t nt = (int64_t)c->P.trow.size();
    c->trow = c->mem.alloc<int32_t>(nt);
    c->tcol = c->mem.alloc<int32_t>(nt);
    c->tval = c->mem.alloc<double>(nt);
    c->ysum = c->mem.alloc<double>(nt);
    c->rmse_part = c->mem.alloc<double>(2 * c->rmse_blocks);
    c->rmse_out = c->mem.alloc<double>(2);
    c->err_d = c->mem.alloc<DevError>(1);
    c->aggX = c->mem.alloc<double>(N * K);
    c->aggW = c->mem.alloc<double>(D * K);
    c->ncorr_d = c->mem.alloc<unsigned long long>(1);
    const int MB = std::max(I, J);
    c->agg_base = c->mem.alloc<int64_t>((size_t)(I + J) * MB);
    // eigenvalue corrections of one aggregation launch (at most N (J - 1) or D (I - 1) pairs;
    // the launches run in order on the context stream and reuse the buffer)
    c->agg_corr = c->mem.alloc<double>((size_t)N * std::max(J - 1, 0) + (size_t)D * std::max(I - 1, 0));
    c->agg_list = c->mem.alloc<int32_t>((size_t)N * std::max(J - 1, 0) + (size_t)D * std::max(I - 1, 0));
    c->agg_list_n = c->mem.alloc<unsigned>(1);
    c->X0o = c->mem.alloc<double>(N * K);
    c->W0o = c->mem.alloc<double>(D * K);
    c->xsrc = c->mem.alloc<int64_t>(c->P.RX);
    c->wsrc = c->mem.alloc<int64_t>(c->P.RW);
    c->tg_row = c->mem.alloc<int32_t>(nt);
    c->tg_col = c->mem.alloc<int32_t>(nt);
    c->row_rank_d = c->mem.alloc<int64_t>(N);
    c->col_rank_d = c->mem.alloc<int64_t>(D);
    c->pred_part = c->mem.alloc<double>(2 * c->rmse_blocks);
    c->pred_out = c->mem.alloc<double>(2);
    if (c->noise != BMF_NOISE_FIXED) {
        const size_t gb = c->prec == BMF_FP64 ? 8 : (c->prec == BMF_FP32 ? 4 : 2);
        const size_t vb = c->prec == BMF_FP64 ? 8 : 4;
        const int64_t nx = c->X.h_obs[c->P.RX];
        c->tau_w = c->mem.alloc<double>(c->P.RW);
        c->noise_sse = c->mem.alloc<double>(c->P.RW);
        c->Ws = c->mem.alloc<char>((size_t)c->P.RW * c->ldg * gb);
        c->xval_orig = c->mem.alloc<char>((size_t)nx * vb);
        c->noise_blocks = c->mem.alloc<NoiseBlock>(S);
        if (c->mem.ok && nx)
            cudaMemcpy(c->xval_orig, c->X.val, (size_t)nx * vb, cudaMemcpyDeviceToDevice);
    }
    if (c->summary != BMF_SUMMARY_MM)
        for (int f = 0; f < 2; ++f) {
            const int64_t R = f == 0 ? c->P.RX : c->P.RW;
            c->ring[f] = c->mem.alloc<double>((size_t)c->max_samples * R * K);
            c->has_mix[f] = c->mem.alloc<int8_t>(R);
            if (c->summary == BMF_SUMMARY_GMM)
                c->mix[f] = c->mem.alloc<double>((size_t)R * c->ncomp * mix_width(K));
        }
    if (!c->mem.ok) return bail(BMF_E_OOM, "device allocation failed");
    cudaMemcpy(c->mu0_d, c->mu0.data(), K * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->W0inv_d, c->W0inv.data(), (size_t)K * K * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(c->hyper, 0, (size_t)2 * S * hyper_slot_len(K) * sizeof(double));
    if (nt) {
        cudaMemcpy(c->trow, c->P.trow.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->tcol, c->P.tcol.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->tval, c->P.tval.data(), nt * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemset(c->ysum, 0, nt * sizeof(double));
    }
    DevError z = {0u, INT32_MAX};
    cudaMemcpy(c->err_d, &z, sizeof(z), cudaMemcpyHostToDevice);
    // aggregation bases: X block i over submodels (i, j), then W block j over (i, j)
    {
        std::vector<int64_t> base((size_t)(I + J) * MB, 0);
        for (int i = 0; i < I; ++i)
            for (int j = 0; j < J; ++j) base[(size_t)i * MB + j] = c->P.subs[i * J + j].xoff;
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < I; ++i) base[(size_t)(I + j) * MB + i] = c->P.subs[i * J + j].woff;
        cudaMemcpy(c->agg_base, base.data(), base.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    }
    // held-out entries in the reordered index space; original -> reordered maps
    if (nt) {
        std::vector<int32_t> gr(nt), gc(nt);
        for (const auto &g : c->P.subs)
            for (int64_t k = g.test_off; k < g.test_off + g.n_test; ++k) {
                gr[k] = (int32_t)(g.r0 + (c->P.trow[k] - g.xoff));
                gc[k] = (int32_t)(g.c0 + (c->P.tcol[k] - g.woff));
            }
        cudaMemcpy(c->tg_row, gr.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice);
        cudaMemcpy(c->tg_col, gc.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (N) cudaMemcpy(c->row_rank_d, c->P.row_rank.data(), N * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (D) cudaMemcpy(c->col_rank_d, c->P.col_rank.data(), D * sizeof(int64_t), cudaMemcpyHostToDevice);
    // initial states: kept in the original order; every subset's blocks gathered from them
    {
        std::vector<int64_t> xs(c->P.RX), ws(c->P.RW);
        for (const auto &g : c->P.subs) {
            for (int64_t r = 0; r < g.n(); ++r) xs[g.xoff + r] = c->P.row_perm[g.r0 + r];
            for (int64_t r = 0; r < g.d(); ++r) ws[g.woff + r] = c->P.col_perm[g.c0 + r];
        }
        if (c->P.RX) cudaMemcpy(c->xsrc, xs.data(), xs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (c->P.RW) cudaMemcpy(c->wsrc, ws.data(), ws.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    }
    if (N) cudaMemcpy(c->X0o, X0, N * K * sizeof(double), cudaMemcpyHostToDevice);
    if (D) cudaMemcpy(c->W0o, W0init, D * K * sizeof(double), cudaMemcpyHostToDevice);
    c->ss.assign(S, SubState());
    c->stats_ok.assign(S, 0);
    s = restart_chains(c);
    if (s) return bail(s, "");
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(BMF_E_CUDA, std::string("CUDA: ") + cudaGetErrorString(e));
    c->stage_open = 1;
    *out = c;
    return BMF_OK;
}

int64_t bmf_draws_per_sweep(const bmf_ctx *c, int32_t stage, int32_t subset)
{
    if (!c) return -1;
    if (subset >= 0) {
        if (!valid_subset(c, subset)) return -1;
        int sl = c->P.subs[subset].slot;
        return per_sweep_draws(c, sl, sl + 1);
    }
    int sl0, sl1;
    if (!stage_slots(c, stage, sl0, sl1)) return -1;
    return per_sweep_draws(c, sl0, sl1);
}

bmf_status bmf_set_schedule(bmf_ctx *c, const bmf_schedule *s)
{
    if (!c || !s) return BMF_E_ARG;
    if (s->chunks_x < 1 || s->chunks_x > kMaxChunks || s->chunks_w < 1 || s->chunks_w > kMaxChunks)
        return fail(c, BMF_E_ARG, "chunks must be in 1.." + std::to_string(kMaxChunks));
    if (s->gram_blocks_per_sm < 1 || s->gram_blocks_per_sm > 64)
        return fail(c, BMF_E_ARG, "gram_blocks_per_sm must be in 1..64");
    if (!(s->row_weight >= 0.0) || !std::isfinite(s->row_weight))
        return fail(c, BMF_E_ARG, "row_weight must be finite and >= 0");
    if (s->graph != 0 && s->graph != 1) return fail(c, BMF_E_ARG, "graph must be 0 or 1");
    if (s->cond_lanes != 0 && s->cond_lanes != 2 && s->cond_lanes != 4 && s->cond_lanes != 8 &&
        s->cond_lanes != 16 && s->cond_lanes != 32)
        return fail(c, BMF_E_ARG, "cond_lanes must be 0, 2, 4, 8, 16 or 32");
    if (s->cond_lanes != 0 && c->K >= kTeamMinK && !cond_lanes_valid(c->K, s->cond_lanes))
        return fail(c, BMF_E_ARG, "cond_lanes " + std::to_string(s->cond_lanes) +
                                      " cannot factor rows of K = " + std::to_string(c->K) +
                                      " (two lanes: 13 <= K <= 16; teams must fit in shared memory)");
    c->sched = *s;
    return BMF_OK;
}

bmf_status bmf_set_monitor(bmf_ctx *c, int32_t on)
{
    if (!c) return BMF_E_ARG;
    if (on != 0 && on != 1) return fail(c, BMF_E_ARG, "monitor must be 0 or 1");
    c->monitor = on != 0;
    return BMF_OK;
}

bmf_status bmf_get_schedule(const bmf_ctx *c, bmf_schedule *s)
{
    if (!c || !s) return BMF_E_ARG;
    *s = c->sched;
    return BMF_OK;
}

// Everything a batch of sweeps changes, for the schedule tuner: FP64 state, gathered copies,
// moment sums (SoA) of the batch's rows, its hyperparameter slots, the running test predictions
// and the per-subset counters.
struct BatchSnapshot {
    DevMem mem;
    struct Part {
        void *dst;
        const void *src;
        size_t width, height, spitch;
    };
    std::vector<Part> parts;
    std::vector<SubState> ss;
    bool ok = true;
    void add(bmf_ctx *c, void *live, size_t width, size_t height = 1, size_t pitch = 0)
    {
        if (!width || !height) return;
        char *b = mem.alloc<char>(width * height);
        if (!b) {
            ok = false;
            return;
        }
        parts.push_back(Part{b, live, width, height, pitch ? pitch : width});
    }
    bmf_status take(bmf_ctx *c)
    {
        for (const Part &q : parts)
            CUDA_TRY(c, cudaMemcpy2DAsync(q.dst, q.width, q.src, q.spitch, q.width, q.height,
                                          cudaMemcpyDeviceToDevice, c->st));
        return BMF_OK;
    }
    bmf_status restore(bmf_ctx *c)
    {
        for (const Part &q : parts)
            CUDA_TRY(c, cudaMemcpy2DAsync(const_cast<void *>(q.src), q.spitch, q.dst, q.width,
                                          q.width, q.height, cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(c, cudaStreamSynchronize(c->st));
        return BMF_OK;
    }
};

bmf_status bmf_autotune(bmf_ctx *c, int32_t stage, int32_t subset, int32_t sweeps_per_trial,
                        bmf_schedule *best_out)
{
    if (!c) return BMF_E_ARG;
    if (sweeps_per_trial < 1) return fail(c, BMF_E_ARG, "sweeps_per_trial must be >= 1");
    int sl0, sl1;
    if (subset >= 0) {
        if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
        sl0 = c->P.subs[subset].slot;
        sl1 = sl0 + 1;
    } else if (!stage_slots(c, stage, sl0, sl1)) {
        return fail(c, BMF_E_ARG, "stage has no subsets");
    }
    if (geom_of_slot(c, sl0).stage != c->stage_open)
        return fail(c, BMF_E_STATE, "the batch's stage is not the open stage");
    const int K = c->K;
    const size_t gb = c->prec == BMF_FP64 ? 8 : (c->prec == BMF_FP32 ? 4 : 2);
    const SubsetGeom &g0 = geom_of_slot(c, sl0), &gl = geom_of_slot(c, sl1 - 1);
    BatchSnapshot snap;
    for (int f = 0; f < 2; ++f) {
        Side &sd = f == 0 ? c->X : c->W;
        const int64_t r0 = f == 0 ? g0.xoff : g0.woff;
        const int64_t r1 = f == 0 ? gl.xoff + gl.n() : gl.woff + gl.d();
        const size_t n = (size_t)(r1 - r0);
        snap.add(c, sd.F + r0 * K, n * K * sizeof(double));
        snap.add(c, static_cast<char *>(sd.G) + r0 * c->ldg * gb, n * c->ldg * gb);
        snap.add(c, sd.S1 + r0, n * sizeof(double), K, sd.R * sizeof(double));
        snap.add(c, sd.S2 + r0, n * sizeof(double), ntri(K), sd.R * sizeof(double));
    }
    snap.add(c, c->hyper + (int64_t)2 * sl0 * hyper_slot_len(K),
             (size_t)2 * (sl1 - sl0) * hyper_slot_len(K) * sizeof(double));
    if (c->tau_w) snap.add(c, c->tau_w + g0.woff, (size_t)(gl.woff + gl.d() - g0.woff) * sizeof(double));
    const int64_t tt0 = g0.test_off, tt1 = gl.test_off + gl.n_test;
    snap.add(c, c->ysum + tt0, (size_t)(tt1 - tt0) * sizeof(double));
    if (!snap.ok || !snap.mem.ok) return fail(c, BMF_E_OOM, "device allocation failed (tuner)");
    bmf_status s = snap.take(c);
    if (s) return s;
    snap.ss = c->ss;
    const bmf_schedule keep = c->sched;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto trial = [&](const bmf_schedule &sc, float *ms) -> bmf_status {
        c->sched = sc;
        bmf_status st = run_batch(c, sl0, sl1, 1, nullptr, nullptr);
        if (!st) {
            cudaEventRecord(e0, c->st);
            st = run_batch(c, sl0, sl1, sweeps_per_trial, nullptr, nullptr);
            cudaEventRecord(e1, c->st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(ms, e0, e1);
        }
        c->ss = snap.ss;
        bmf_status rs = snap.restore(c);
        for (int sl = sl0; sl < sl1; ++sl) c->stats_ok[sl] = 0;   // statistics of a trial
        return st ? st : rs;
    };
    bmf_schedule best = keep;
    float best_ms = 0.f;
    std::vector<bmf_schedule> cands;
    // coordinate search: Gram grid, then row chunks of each half, then the split weight
    auto run_all = [&](const std::vector<bmf_schedule> &cs) -> bmf_status {
        for (const bmf_schedule &sc : cs) {
            float ms = 0.f;
            bmf_status st = trial(sc, &ms);
            if (st) return st;
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best = sc;
            }
        }
        return BMF_OK;
    };
    bmf_schedule b0{1, 1, 4, 0.0, 0, 0};
    cands = {b0};
    for (int g : {2, 8}) cands.push_back(bmf_schedule{1, 1, g, 0.0, 0, 0});
    s = run_all(cands);
    for (int f = 0; f < 2 && !s; ++f) {
        cands.clear();
        for (int ch : {2, 3, 4}) {
            bmf_schedule sc = best;
            (f == 0 ? sc.chunks_x : sc.chunks_w) = ch;
            cands.push_back(sc);
        }
        s = run_all(cands);
    }
    if (!s && (best.chunks_x > 1 || best.chunks_w > 1)) {
        const double w0 = (c->prec == BMF_FP64 ? 1.5 : 14.0) * K;
        cands.clear();
        for (double m : {0.3, 3.0}) {
            bmf_schedule sc = best;
            sc.row_weight = w0 * m;
            cands.push_back(sc);
        }
        s = run_all(cands);
    }
    if (!s && K >= kTeamMinK) {
        // lanes per row of the conditional (every choice gives bit-identical values)
        cands.clear();
        const std::vector<int> tries = K <= 16 ? std::vector<int>{2, 4, 8} : std::vector<int>{8, 16, 32};
        for (int lanes : tries)
            if (cond_lanes_valid(K, lanes) &&
                lanes != (best.cond_lanes > 0 ? best.cond_lanes : cond_team_size(K))) {
                bmf_schedule sc = best;
                sc.cond_lanes = lanes;
                cands.push_back(sc);
            }
        s = run_all(cands);
    }
    if (!s) {
        bmf_schedule sc = best;
        sc.graph = 1;
        s = run_all({sc});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sched = s ? keep : best;
    if (s) return s;
    if (best_out) *best_out = best;
    return BMF_OK;
}

bmf_status bmf_generate_draws(bmf_ctx *c, int32_t stage, int32_t subset, int64_t t0,
                              int32_t n_sweeps, double *out, int32_t out_on_device)
{
    if (!c) return BMF_E_ARG;
    int sl0, sl1;
    if (subset >= 0) {
        if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
        sl0 = c->P.subs[subset].slot;
        sl1 = sl0 + 1;
    } else if (!stage_slots(c, stage, sl0, sl1)) {
        return fail(c, BMF_E_ARG, "stage has no subsets");
    }
    if (t0 < 1 || n_sweeps < 0) return fail(c, BMF_E_ARG, "need t0 >= 1 and n_sweeps >= 0");
    if (n_sweeps > 0 && !out) return fail(c, BMF_E_ARG, "out is NULL");
    const int64_t per = per_sweep_draws(c, sl0, sl1);
    int64_t units = 0;
    int n_segs = 0;
    bmf_status s = prepare_gen(c, sl0, sl1, per, out_on_device ? 0 : 1, &units, &n_segs);
    if (s) return s;
    for (int i = 0; i < n_sweeps; ++i) {
        double *dst = out_on_device ? out + (int64_t)i * per : c->gen_d;
        enqueue_gen(c, units, n_segs, t0 + i, dst);
        if (!out_on_device)
            CUDA_TRY(c, cudaMemcpyAsync(out + (int64_t)i * per, c->gen_d, per * sizeof(double),
                                        cudaMemcpyDeviceToHost, c->st));
    }
    CUDA_TRY(c, cudaGetLastError());
    s = check_dev_error(c);
    if (c->prof) collect_profile(c);
    return s;
}

bmf_status bmf_sweep(bmf_ctx *c, int32_t subset, int32_t n_sweeps, const bmf_draws *draws,
                     bmf_sweep_stats *stats)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    const SubsetGeom &g = c->P.subs[subset];
    if (g.stage != c->stage_open)
        return fail(c, BMF_E_STATE, "the subset's stage is not the open stage");
    return run_batch(c, g.slot, g.slot + 1, n_sweeps, draws, stats);
}

bmf_status bmf_stage(bmf_ctx *c, int32_t stage, int32_t n_sweeps, const bmf_draws *draws,
                     bmf_sweep_stats *stats)
{
    if (!c) return BMF_E_ARG;
    if (stage < 1 || stage > 3) return fail(c, BMF_E_ARG, "stage must be 1, 2 or 3");
    bmf_status s = open_stage(c, stage);
    if (s) return s;
    int sl0, sl1;
    stage_slots(c, stage, sl0, sl1);
    return run_batch(c, sl0, sl1, n_sweeps, draws, stats);
}

bmf_status bmf_posterior_means(bmf_ctx *c, double *Xm, double *Wm, int64_t *n_corrected)
{
    if (!c) return BMF_E_ARG;
    std::vector<double> x, w;
    bmf_status s = means_original(c, x, w, n_corrected);
    if (s) return s;
    if (Xm) std::memcpy(Xm, x.data(), x.size() * sizeof(double));
    if (Wm) std::memcpy(Wm, w.data(), w.size() * sizeof(double));
    return BMF_OK;
}

bmf_status bmf_predict(bmf_ctx *c, int64_t n, const int32_t *row, const int32_t *col,
                       const double *y, double *yhat, double *rmse)
{
    if (!c) return BMF_E_ARG;
    if (n < 0 || (n > 0 && (!row || !col))) return fail(c, BMF_E_ARG, "bad prediction entries");
    if (rmse && !y) return fail(c, BMF_E_ARG, "rmse needs y");
    for (int64_t e = 0; e < n; ++e)
        if (row[e] < 0 || row[e] >= c->P.N || col[e] < 0 || col[e] >= c->P.D)
            return fail(c, BMF_E_ARG, "prediction index out of range");
    bmf_status s = aggregate_all(c, nullptr);
    if (s) return s;
    if (n == 0) {
        if (rmse) *rmse = NAN;
        return BMF_OK;
    }
    // entries to the device, predictions there with the aggregated means (reordered order,
    // reached through the original -> reordered maps), squared errors summed there
    if ((s = pred_room(c, n))) return s;
    int32_t *rd = reinterpret_cast<int32_t *>(c->pred_buf), *cd = rd + n;
    double *yd = reinterpret_cast<double *>(c->pred_buf + n * 2 * sizeof(int32_t)), *hd = yd + n;
    CUDA_TRY(c, cudaMemcpyAsync(rd, row, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    CUDA_TRY(c, cudaMemcpyAsync(cd, col, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
    if (rmse) CUDA_TRY(c, cudaMemcpyAsync(yd, y, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    PredictParams pp{c->K, n, rd, cd, c->row_rank_d, c->col_rank_d, c->aggX, c->aggW,
                     c->P.offset, hd, rmse ? yd : nullptr, rmse ? c->pred_part : nullptr};
    launch_predict_sq(pp, c->rmse_blocks, c->st);
    if (rmse) {
        launch_rmse_final(c->pred_part, c->rmse_blocks, c->pred_out, c->st);
        CUDA_TRY(c, cudaMemcpyAsync(c->rb->rmse, c->pred_out, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->st));
    }
    if (yhat) CUDA_TRY(c, cudaMemcpyAsync(yhat, hd, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (rmse) *rmse = std::sqrt(c->rb->rmse[0] / (double)n);
    return BMF_OK;
}

bmf_status bmf_test_rmse(bmf_ctx *c, double *rmse)
{
    if (!c || !rmse) return BMF_E_ARG;
    bmf_status s = aggregate_all(c, nullptr);
    if (s) return s;
    const int64_t nt = (int64_t)c->P.trow.size();
    if (nt == 0) {
        *rmse = NAN;
        return BMF_OK;
    }
    // held-out values are stored centred: the prediction of the centred value has no offset
    PredictParams pp{c->K, nt, c->tg_row, c->tg_col, nullptr, nullptr, c->aggX, c->aggW, 0.0,
                     nullptr, c->tval, c->pred_part};
    launch_predict_sq(pp, c->rmse_blocks, c->st);
    launch_rmse_final(c->pred_part, c->rmse_blocks, c->pred_out, c->st);
    CUDA_TRY(c, cudaMemcpyAsync(c->rb->rmse, c->pred_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->st));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    *rmse = std::sqrt(c->rb->rmse[0] / (double)nt);
    return BMF_OK;
}

bmf_status bmf_restart(bmf_ctx *c, const double *X0, const double *W0init, uint64_t seed)
{
    if (!c) return BMF_E_ARG;
    const int K = c->K;
    if (X0)
        for (int64_t e = 0; e < c->P.N * K; ++e)
            if (!std::isfinite(X0[e])) return fail(c, BMF_E_NONFINITE, "non-finite X0");
    if (W0init)
        for (int64_t e = 0; e < c->P.D * K; ++e)
            if (!std::isfinite(W0init[e])) return fail(c, BMF_E_NONFINITE, "non-finite W0init");
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (X0 && c->P.N)
        CUDA_TRY(c, cudaMemcpyAsync(c->X0o, X0, c->P.N * K * sizeof(double), cudaMemcpyHostToDevice,
                                    c->st));
    if (W0init && c->P.D)
        CUDA_TRY(c, cudaMemcpyAsync(c->W0o, W0init, c->P.D * K * sizeof(double),
                                    cudaMemcpyHostToDevice, c->st));
    c->seed = seed;
    return restart_chains(c);
}

bmf_status bmf_get_state(bmf_ctx *c, int32_t subset, double *X, double *W, double *hyper)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    const SubsetGeom &g = c->P.subs[subset];
    const int K = c->K;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (X && g.n())
        CUDA_TRY(c, cudaMemcpy(X, c->X.F + g.xoff * K, g.n() * K * sizeof(double), cudaMemcpyDeviceToHost));
    if (W && g.d())
        CUDA_TRY(c, cudaMemcpy(W, c->W.F + g.woff * K, g.d() * K * sizeof(double), cudaMemcpyDeviceToHost));
    if (hyper) {
        const int HS = hyper_slot_len(K);
        std::vector<double> h(2 * HS);
        CUDA_TRY(c, cudaMemcpy(h.data(), c->hyper + (int64_t)2 * g.slot * HS, 2 * HS * sizeof(double),
                               cudaMemcpyDeviceToHost));
        for (int f = 0; f < 2; ++f) {
            const double *sl = h.data() + f * HS;
            double *o = hyper + f * (K + K * K);
            for (int i = 0; i < K; ++i) o[i] = sl[i];
            for (int i = 0; i < K; ++i)
                for (int j = 0; j <= i; ++j) o[K + i * K + j] = o[K + j * K + i] = sl[K + tri(i, j)];
        }
    }
    return BMF_OK;
}

bmf_status bmf_set_state(bmf_ctx *c, int32_t subset, const double *X, const double *W)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    const SubsetGeom &g = c->P.subs[subset];
    const int K = c->K;
    if (X) {
        for (int64_t e = 0; e < g.n() * K; ++e)
            if (!std::isfinite(X[e])) return fail(c, BMF_E_NONFINITE, "non-finite X");
        if (g.n())
            CUDA_TRY(c, cudaMemcpy(c->X.F + g.xoff * K, X, g.n() * K * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (W) {
        for (int64_t e = 0; e < g.d() * K; ++e)
            if (!std::isfinite(W[e])) return fail(c, BMF_E_NONFINITE, "non-finite W");
        if (g.d())
            CUDA_TRY(c, cudaMemcpy(c->W.F + g.woff * K, W, g.d() * K * sizeof(double), cudaMemcpyHostToDevice));
    }
    // refresh the gathered copies of the whole arenas (cheap, keeps the call simple)
    launch_fill_gather(K, c->prec, c->X.R, c->X.F, c->X.G, c->ldg, c->st);
    launch_fill_gather(K, c->prec, c->W.R, c->W.F, c->W.G, c->ldg, c->st);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    c->failed = false;
    c->stats_ok[g.slot] = 0;
    return BMF_OK;
}

bmf_status bmf_get_moments(bmf_ctx *c, int32_t subset, int32_t factor, double *S1, double *S2,
                           int64_t *kept)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset) || (factor != 0 && factor != 1))
        return fail(c, BMF_E_ARG, "bad subset or factor");
    const SubsetGeom &g = c->P.subs[subset];
    const Side &sd = factor == 0 ? c->X : c->W;
    const int64_t n = factor == 0 ? g.n() : g.d(), base = factor == 0 ? g.xoff : g.woff;
    const int K = c->K, NT = ntri(K);
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    std::vector<double> col(n);
    if (S1)
        for (int i = 0; i < K && n; ++i) {
            CUDA_TRY(c, cudaMemcpy(col.data(), sd.S1 + (int64_t)i * sd.R + base, n * sizeof(double),
                                   cudaMemcpyDeviceToHost));
            for (int64_t r = 0; r < n; ++r) S1[r * K + i] = col[r];
        }
    if (S2 && !c->full_moments)
        return fail(c, BMF_E_STATE, "second moments are not accumulated (moments mode)");
    if (S2)
        for (int e = 0; e < NT && n; ++e) {
            CUDA_TRY(c, cudaMemcpy(col.data(), sd.S2 + (int64_t)e * sd.R + base, n * sizeof(double),
                                   cudaMemcpyDeviceToHost));
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            int j = e - i * (i + 1) / 2;
            for (int64_t r = 0; r < n; ++r) S2[(r * K + i) * K + j] = S2[(r * K + j) * K + i] = col[r];
        }
    if (kept) *kept = c->ss[subset].kept;
    return BMF_OK;
}

bmf_status bmf_get_posterior(bmf_ctx *c, int32_t subset, int32_t factor, double *mu, double *Lam)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset) || (factor != 0 && factor != 1))
        return fail(c, BMF_E_ARG, "bad subset or factor");
    if (!c->ss[subset].finalized) {
        // finalise on demand (does not change the chain)
        bmf_status s = finalize_subset(c, subset);
        if (!s) s = cuda_status(c, cudaGetLastError(), "summary launch");
        if (!s) s = check_dev_error(c);
        if (s) {
            c->ss[subset].finalized = false;
            return s;
        }
    }
    const SubsetGeom &g = c->P.subs[subset];
    const Side &sd = factor == 0 ? c->X : c->W;
    const int64_t n = factor == 0 ? g.n() : g.d(), base = factor == 0 ? g.xoff : g.woff;
    const int K = c->K, NT = ntri(K);
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (mu && n)
        CUDA_TRY(c, cudaMemcpy(mu, sd.mm_mu + base * K, n * K * sizeof(double), cudaMemcpyDeviceToHost));
    if (Lam) {
        std::vector<double> col(n);
        for (int e = 0; e < NT && n; ++e) {
            CUDA_TRY(c, cudaMemcpy(col.data(), sd.mm_L + (int64_t)e * sd.R + base, n * sizeof(double),
                                   cudaMemcpyDeviceToHost));
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            int j = e - i * (i + 1) / 2;
            for (int64_t r = 0; r < n; ++r) Lam[(r * K + i) * K + j] = Lam[(r * K + j) * K + i] = col[r];
        }
    }
    return BMF_OK;
}

bmf_status bmf_set_prior(bmf_ctx *c, int32_t subset, int32_t factor, const double *mu,
                         const double *Lam)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset) || (factor != 0 && factor != 1) || !mu || !Lam)
        return fail(c, BMF_E_ARG, "bad subset, factor or null prior");
    const SubsetGeom &g = c->P.subs[subset];
    Side &sd = factor == 0 ? c->X : c->W;
    const int64_t n = factor == 0 ? g.n() : g.d(), base = factor == 0 ? g.xoff : g.woff;
    const int K = c->K, NT = ntri(K);
    std::vector<double> L((size_t)NT * n), b((size_t)K * n);
    for (int64_t r = 0; r < n; ++r) {
        const double *Lr = Lam + r * K * K, *mr = mu + r * K;
        for (int i = 0; i < K; ++i) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += Lr[i * K + k] * mr[k];
            b[(size_t)i * n + r] = acc;
            for (int j = 0; j <= i; ++j) L[(size_t)tri(i, j) * n + r] = Lr[i * K + j];
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    for (int e = 0; e < NT && n; ++e)
        CUDA_TRY(c, cudaMemcpy(sd.pL + (int64_t)e * sd.R + base, &L[(size_t)e * n], n * sizeof(double),
                               cudaMemcpyHostToDevice));
    for (int i = 0; i < K && n; ++i)
        CUDA_TRY(c, cudaMemcpy(sd.pb + (int64_t)i * sd.R + base, &b[(size_t)i * n], n * sizeof(double),
                               cudaMemcpyHostToDevice));
    c->ss[subset].prior[factor] = 1;
    if (c->ss[subset].mix[factor]) {     // an installed Gaussian replaces a mixture prior
        c->ss[subset].mix[factor] = 0;
        if (n) CUDA_TRY(c, cudaMemset(c->has_mix[factor] + base, 0, (size_t)n));
    }
    refresh_hslots(c, g.slot);
    bmf_status s = upload_hslots(c, g.slot);
    if (s) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    return BMF_OK;
}

bmf_status bmf_get_noise(bmf_ctx *c, int32_t subset, double *tau)
{
    if (!c || !tau) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    const SubsetGeom &g = c->P.subs[subset];
    if (!c->tau_w) {
        for (int64_t k = 0; k < g.d(); ++k) tau[k] = c->tau;
        return BMF_OK;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (g.d())
        CUDA_TRY(c, cudaMemcpy(tau, c->tau_w + g.woff, g.d() * sizeof(double), cudaMemcpyDeviceToHost));
    return BMF_OK;
}

bmf_status bmf_get_subset_info(const bmf_ctx *c, int32_t subset, bmf_subset_info *info)
{
    if (!c || !info || !valid_subset(c, subset)) return BMF_E_ARG;
    const SubsetGeom &g = c->P.subs[subset];
    info->i = g.i;
    info->j = g.j;
    info->stage = g.stage;
    info->row0 = g.r0;
    info->row1 = g.r1;
    info->col0 = g.c0;
    info->col1 = g.c1;
    info->nnz = g.nnz;
    return BMF_OK;
}

bmf_status bmf_get_perm(const bmf_ctx *c, int64_t *row_perm, int64_t *col_perm)
{
    if (!c) return BMF_E_ARG;
    if (row_perm) std::memcpy(row_perm, c->P.row_perm.data(), c->P.N * sizeof(int64_t));
    if (col_perm) std::memcpy(col_perm, c->P.col_perm.data(), c->P.D * sizeof(int64_t));
    return BMF_OK;
}

bmf_status bmf_profile_enable(bmf_ctx *c, int32_t on)
{
    if (!c) return BMF_E_ARG;
    c->prof = on != 0;
    return BMF_OK;
}

int32_t bmf_profile_read(bmf_ctx *c, bmf_kernel_time *out, int32_t max)
{
    if (!c) return -1;
    for (int k = 0; k < K_NCLASS && k < max && out; ++k) {
        std::memset(out[k].name, 0, sizeof(out[k].name));
        std::strncpy(out[k].name, kClassName[k], sizeof(out[k].name) - 1);
        out[k].launches = c->prof_n[k];
        out[k].total_ms = c->prof_ms[k];
    }
    for (int k = 0; k < K_NCLASS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return K_NCLASS;
}

int64_t bmf_launch_count(const bmf_ctx *c) { return c ? c->launches : -1; }

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Adjoint of the masked log-joint and Langevin moves
// ------------------------------------------------------------------------------------------
namespace {

template <typename T>
bmf_status grow(bmf_ctx *c, T *&p, int64_t &cap, int64_t need)
{
    if (need <= cap) return BMF_OK;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, std::max<int64_t>(need, 1) * sizeof(T)) != cudaSuccess)
        return fail(c, BMF_E_OOM, "device allocation failed (adjoint scratch)");
    cap = need;
    return BMF_OK;
}

struct LogJoint {
    double r2 = 0.0, quad = 0.0, value = 0.0, g_log_alpha = 0.0;
};

// Gradient of the subset's log-joint at (X, W) into (gX, gW); scalar parts on the host.
bmf_status logjoint(bmf_ctx *c, int32_t subset, const float *X, const float *W, int64_t ld,
                    double log_alpha, float *gX, float *gW, LogJoint &out)
{
    const SubsetGeom &g = c->P.subs[subset];
    const int K = c->K, kt = adjoint_kt(K), ldp = adjoint_ld(K);
    const double alpha = std::exp(log_alpha);
    int64_t need_part = 0, nb[2];
    for (int f = 0; f < 2; ++f) {
        const Side &me = f == 0 ? c->X : c->W;
        const int64_t r0 = f == 0 ? g.xoff : g.woff, r1 = r0 + (f == 0 ? g.n() : g.d());
        need_part = std::max(need_part, (me.h_item_ptr[r1] - me.h_item_ptr[r0]) * ldp);
        nb[f] = adjoint_row_blocks(r1 - r0);
    }
    bmf_status s = grow(c, c->adj_part, c->adj_part_cap, need_part);
    if (!s) s = grow(c, c->adj_sums, c->adj_sums_cap, 2 * (nb[0] + nb[1]));
    if (s) return s;
    for (int f = 0; f < 2 && c->prec == BMF_FP64; ++f)
        if (!c->fval[f]) {
            const int64_t nnz = c->P.nnz;
            if (cudaMalloc(&c->fval[f], std::max<int64_t>(nnz, 1) * sizeof(float)) != cudaSuccess)
                return fail(c, BMF_E_OOM, "device allocation failed (FP32 values)");
            launch_to_float(static_cast<const double *>((f == 0 ? c->X : c->W).val), c->fval[f], nnz, c->st);
        }
    for (int f = 0; f < 2; ++f) {
        const Side &me = f == 0 ? c->X : c->W;
        const int64_t r0 = f == 0 ? g.xoff : g.woff, r1 = r0 + (f == 0 ? g.n() : g.d());
        const int64_t i0 = me.h_item_ptr[r0], i1 = me.h_item_ptr[r1];
        AdjointParams ap;
        ap.K = K;
        ap.kt = kt;
        ap.ldp = ldp;
        ap.items = me.items + i0;
        ap.n_items = i1 - i0;
        ap.item_base = i0;
        ap.idx = me.idx;
        ap.val = c->prec == BMF_FP64 ? c->fval[f] : static_cast<const float *>(me.val);
        ap.self = f == 0 ? X : W;
        ap.other = f == 0 ? W : X;
        ap.ld = ld;
        ap.self0 = r0;
        ap.other0 = f == 0 ? g.woff : g.xoff;
        ap.part = c->adj_part;
        ap.n_rows = r1 - r0;
        ap.item_ptr = me.item_ptr;
        ap.row_hslot = me.hslot;
        ap.hyper = c->hyper;
        ap.prior_L = me.pL;
        ap.prior_b = me.pb;
        ap.R = me.R;
        ap.grad = f == 0 ? gX : gW;
        ap.alpha = alpha;
        ap.count_r2 = f == 0 ? 1 : 0;
        ap.block_sums = c->adj_sums + (f == 0 ? 0 : 2 * nb[0]);
        traced(c, c->st, K_ADJ, 2, [&] { launch_adjoint(ap, c->sms * 8, c->st); });
    }
    CUDA_TRY(c, cudaGetLastError());
    std::vector<double> h(2 * (nb[0] + nb[1]));
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->adj_sums, h.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    out.r2 = out.quad = 0.0;
    for (int64_t b = 0; b < nb[0] + nb[1]; ++b) {
        out.r2 += h[2 * b];
        out.quad += h[2 * b + 1];
    }
    const double M = (double)g.nnz;
    out.value = -0.5 * alpha * out.r2 + 0.5 * M * log_alpha - 0.5 * out.quad;
    out.g_log_alpha = 0.5 * M - 0.5 * alpha * out.r2;
    return BMF_OK;
}

double sqdiff(bmf_ctx *c, const float *a, const float *b, const float *g, double coef, int64_t n,
              int64_t ld, bmf_status &st)
{
    const int blocks = 256;
    st = grow(c, c->adj_sums, c->adj_sums_cap, (int64_t)blocks);
    if (st) return 0.0;
    launch_sqdiff(a, b, g, coef, n, c->K, ld, c->adj_sums, blocks, c->st);
    std::vector<double> h(blocks);
    if (cudaMemcpyAsync(h.data(), c->adj_sums, blocks * sizeof(double), cudaMemcpyDeviceToHost,
                        c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
        st = fail(c, BMF_E_CUDA, "CUDA error in the Langevin test");
        return 0.0;
    }
    double s = 0.0;
    for (double v : h) s += v;
    return s;
}

bool check_factor_layout(const void *p, int64_t ld, int K)
{
    return p && ld >= K && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(p) % 16) == 0;
}

}  // namespace

extern "C" {

bmf_status bmf_logjoint_grad(bmf_ctx *c, int32_t subset, const float *X, const float *W,
                             int64_t ld, double log_alpha, float *gX, float *gW,
                             double *g_log_alpha, double *value)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    if (c->K > 64) return fail(c, BMF_E_ARG, "the adjoint needs K <= 64");
    if (!check_factor_layout(X, ld, c->K) || !check_factor_layout(W, ld, c->K) ||
        !check_factor_layout(gX, ld, c->K) || !check_factor_layout(gW, ld, c->K))
        return fail(c, BMF_E_ARG, "factors must be 16-byte aligned with ld >= K and ld % 4 == 0");
    if (!std::isfinite(log_alpha)) return fail(c, BMF_E_NONFINITE, "non-finite log_alpha");
    LogJoint lj;
    bmf_status s = logjoint(c, subset, X, W, ld, log_alpha, gX, gW, lj);
    if (s) return s;
    if (c->prof) collect_profile(c);
    if (value) *value = lj.value;
    if (g_log_alpha) *g_log_alpha = lj.g_log_alpha;
    return BMF_OK;
}

bmf_status bmf_langevin(bmf_ctx *c, int32_t subset, int32_t n_steps, float *X, float *W,
                        int64_t ld, double log_alpha, double eps, const float *noise,
                        const double *uniforms, int32_t *accepted, double *value)
{
    if (!c) return BMF_E_ARG;
    if (!valid_subset(c, subset)) return fail(c, BMF_E_ARG, "subset out of range");
    if (n_steps < 0 || !(eps > 0) || !noise) return fail(c, BMF_E_ARG, "need n_steps >= 0, eps > 0, noise");
    if (c->K > 64) return fail(c, BMF_E_ARG, "Langevin moves need K <= 64");
    if (!check_factor_layout(X, ld, c->K) || !check_factor_layout(W, ld, c->K))
        return fail(c, BMF_E_ARG, "factors must be 16-byte aligned with ld >= K and ld % 4 == 0");
    const SubsetGeom &g = c->P.subs[subset];
    const int64_t n = g.n(), d = g.d(), K = c->K;
    const int64_t sx = n * ld, sw = d * ld;
    // buffers: gradient at the current state (gX, gW), proposal (pX, pW), its gradient (qX, qW)
    bmf_status s = grow(c, c->lg_buf, c->lg_cap, 3 * (sx + sw) + 8);
    if (s) return s;
    float *gX = c->lg_buf, *gW = gX + sx, *pX = gW + sw, *pW = pX + sx, *qX = pW + sw, *qW = qX + sx;
    LogJoint cur, prop;
    s = logjoint(c, subset, X, W, ld, log_alpha, gX, gW, cur);
    if (s) return s;
    int32_t acc = 0;
    for (int32_t it = 0; it < n_steps; ++it) {
        const float *xi = noise + (int64_t)it * (n + d) * K;
        CUDA_TRY(c, cudaMemcpyAsync(pX, X, sx * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
        CUDA_TRY(c, cudaMemcpyAsync(pW, W, sw * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
        traced(c, c->st, K_ADJ, 2, [&] {
            launch_langevin(pX, gX, xi, n, (int)K, (int)ld, (float)eps, c->st);
            launch_langevin(pW, gW, xi + n * K, d, (int)K, (int)ld, (float)eps, c->st);
        });
        s = logjoint(c, subset, pX, pW, ld, log_alpha, qX, qW, prop);
        if (s) return s;
        bool take = true;
        if (uniforms) {
            // log A = l' - l + log q(theta | theta') - log q(theta' | theta),
            // log q(a | b) = -|a - b - (eps/2) grad l(b)|^2 / (2 eps)
            bmf_status e1, e2, e3, e4;
            const double back = sqdiff(c, X, pX, qX, 0.5 * eps, n, ld, e1) +
                                sqdiff(c, W, pW, qW, 0.5 * eps, d, ld, e2);
            const double fwd = sqdiff(c, pX, X, gX, 0.5 * eps, n, ld, e3) +
                               sqdiff(c, pW, W, gW, 0.5 * eps, d, ld, e4);
            if (e1 || e2 || e3 || e4) return BMF_E_CUDA;
            const double logA = prop.value - cur.value - back / (2 * eps) + fwd / (2 * eps);
            take = std::log(uniforms[it]) < logA;
        }
        if (take) {
            CUDA_TRY(c, cudaMemcpyAsync(X, pX, sx * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
            CUDA_TRY(c, cudaMemcpyAsync(W, pW, sw * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
            CUDA_TRY(c, cudaMemcpyAsync(gX, qX, sx * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
            CUDA_TRY(c, cudaMemcpyAsync(gW, qW, sw * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
            cur = prop;
            ++acc;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    if (c->prof) collect_profile(c);
    if (accepted) *accepted = acc;
    if (value) *value = cur.value;
    return BMF_OK;
}

void bmf_destroy(bmf_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->draws_d) cudaFree(c->draws_d);
    if (c->gen_d) cudaFree(c->gen_d);
    if (c->gen_segs_d) cudaFree(c->gen_segs_d);
    if (c->pred_buf) cudaFree(c->pred_buf);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (void *p : {(void *)c->adj_part, (void *)c->adj_sums, (void *)c->fval[0], (void *)c->fval[1],
                    (void *)c->lg_buf})
        if (p) cudaFree(p);
    delete c;
}

bmf_status bmf_plan(int64_t N, int64_t D, int64_t nnz, const int32_t *row, const int32_t *col,
                    const double *val, int32_t order, int32_t I, const int64_t *row_bounds,
                    int32_t J, const int64_t *col_bounds, int64_t *row_perm, int64_t *col_perm,
                    int64_t *row_bounds_out, int64_t *col_bounds_out, int64_t *subset_nnz)
{
    g_init_error.clear();
    g_noctx_msg = nullptr;
    if (order != BMF_ORDER_NONE && order != BMF_ORDER_DECREASING) {
        g_init_error = "unknown order";
        return BMF_E_ARG;
    }
    HostPlan P;
    std::string err;
    const int st = build_plan(N, D, nnz, row, col, val, order, 0, I, row_bounds, J, col_bounds, 0,
                              nullptr, nullptr, nullptr, P, err);
    if (st) {
        g_init_error = err;
        return (bmf_status)st;
    }
    if (row_perm) std::copy(P.row_perm.begin(), P.row_perm.end(), row_perm);
    if (col_perm) std::copy(P.col_perm.begin(), P.col_perm.end(), col_perm);
    if (row_bounds_out) std::copy(P.row_bounds.begin(), P.row_bounds.end(), row_bounds_out);
    if (col_bounds_out) std::copy(P.col_bounds.begin(), P.col_bounds.end(), col_bounds_out);
    if (subset_nnz)
        for (int s = 0; s < I * J; ++s) subset_nnz[s] = P.subs[s].nnz;
    return BMF_OK;
}

bmf_status bmf_fit_summaries(int32_t K, int64_t R, int32_t S, const double *samples, int32_t mode,
                             int32_t C, double lambda, double *pi, double *mu, double *Lam,
                             double *pooled_mu, double *pooled_Lam, int32_t *assign, void *stream)
{
    g_init_error.clear();
    g_noctx_msg = nullptr;
    if (K < 1 || K > 32 || S < 1 || (int64_t)S * K > 8192 || R < 0) {
        g_init_error = "bmf_fit_summaries: need 1 <= K <= 32, S >= 1, S * K <= 8192, R >= 0";
        return BMF_E_SHAPE;
    }
    if (mode < 0 || mode > 2 || C < 1 || C > BMF_MAX_COMPONENTS || (mode != 2 && C != 1) ||
        !(lambda > 0.0) || !std::isfinite(lambda)) {
        g_init_error = "bmf_fit_summaries: need mode 0..2, 1 <= C <= 4 (C = 1 unless mode 2), lambda > 0";
        return BMF_E_ARG;
    }
    if (R > 0 && (!samples || !pi || !mu || !Lam || !pooled_mu || !pooled_Lam)) {
        g_init_error = "bmf_fit_summaries: null pointer";
        return BMF_E_ARG;
    }
    if (R == 0) return BMF_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevError *err = nullptr;
    if (cudaMalloc(&err, sizeof(DevError)) != cudaSuccess) {
        g_init_error = "bmf_fit_summaries: device allocation failed";
        return BMF_E_OOM;
    }
    DevError z = {0u, INT32_MAX}, h = z;
    cudaError_t e = cudaMemcpyAsync(err, &z, sizeof z, cudaMemcpyHostToDevice, st);
    SummaryParams sp{};
    sp.K = K;
    sp.S = S;
    sp.C = C;
    sp.mode = mode;
    sp.lambda = lambda;
    sp.samples = samples;
    sp.sample_stride = R * K;
    sp.row0 = 0;
    sp.n_rows = R;
    sp.pi = pi;
    sp.mu = mu;
    sp.Lam = Lam;
    sp.pooled_mu = pooled_mu;
    sp.pooled_Lam = pooled_Lam;
    sp.assign = assign;
    sp.R = R;
    sp.err = err;
    if (e == cudaSuccess) {
        launch_summary(sp, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) {
        g_init_error = std::string("bmf_fit_summaries: CUDA error: ") + cudaGetErrorString(e);
        return BMF_E_CUDA;
    }
    if (h.flags) {
        g_init_error = "bmf_fit_summaries: a covariance is singular (row " +
                       std::to_string(h.first_bad_row) + ")";
        return BMF_E_NOT_PD;
    }
    return BMF_OK;
}

const char *bmf_last_error(const bmf_ctx *c)
{
    if (!c) return g_noctx_msg ? g_noctx_msg : g_init_error.c_str();
    return c->err.c_str();
}

}  // extern "C"
