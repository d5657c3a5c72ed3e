// aggregate_static.cu -- bmf_aggregate_static: the aggregation of per-row Gaussian submodels
// (Eq. 14 with the eigenvalue correction of Algorithm 2) for callers that cannot allocate GPU
// memory, e.g. a runtime that owns all device memory through its own allocator and forbids
// libraries from calling cudaMalloc, or a service whose device footprint is fixed at start-up.
//
// The per-row working matrices live in one file-scope static device array of fixed size
// (kStaticBytes).  Every GPU that loads this library holds that array until the process exits.
// All calls share it: the array keeps the previous call's contents, the call clears the part
// that must start at zero, and two calls whose work overlaps on the GPU (different streams or
// different host threads) race on it.  The call reads its counters back and synchronises its
// stream before returning.
#include <cstdint>
#include <mutex>

#include "bmf.h"
#include "common.cuh"

namespace bmf {
void set_noctx_error(const char *m);  // message for bmf_last_error(NULL); no allocation
}

namespace {

constexpr size_t kStaticBytes = size_t(32) << 20;                // 32 MiB
constexpr size_t kHeaderDoubles = 32;                             // 256 bytes: counters, flags
constexpr size_t kStaticDoubles = kStaticBytes / sizeof(double);
static_assert(kStaticDoubles - kHeaderDoubles == BMF_AGGREGATE_STATIC_MAX_DOUBLES,
              "public limit and static array disagree");
constexpr int kThreads = 32;
constexpr int kMaxDevices = 64;

// [0]: number of corrected (row, submodel) pairs (as unsigned long long bits)
// [1]: error flags (bit 0: an aggregated precision is not positive definite)
// [kHeaderDoubles ...]: K x K working matrix of every row of the call
static __device__ __align__(256) double g_scratch[kStaticDoubles];

#define RS(base, e) (base)[(e) * kThreads]

__device__ double min_eig_jacobi(double *a, int K)
{
    double fro = 0.0;
    for (int e = 0; e < K * K; ++e) fro += a[e] * a[e];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) off += a[p * K + q] * a[p * K + q];
        if (off <= 1e-30 * fro || off == 0.0) break;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                const double apq = a[p * K + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * K + q] - a[p * K + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < K; ++k) {
                    const double akp = a[k * K + p], akq = a[k * K + q];
                    a[k * K + p] = c * akp - s * akq;
                    a[k * K + q] = s * akp + c * akq;
                }
                for (int k = 0; k < K; ++k) {
                    const double apk = a[p * K + k], aqk = a[q * K + k];
                    a[p * K + k] = c * apk - s * aqk;
                    a[q * K + k] = s * apk + c * aqk;
                }
            }
    }
    double m = a[0];
    for (int i = 1; i < K; ++i) m = fmin(m, a[i * K + i]);
    return m;
}

// In-place packed lower Cholesky of one thread's interleaved matrix.
__device__ bool chol_packed(double *P, int K)
{
    for (int j = 0; j < K; ++j) {
        const int jj = bmf::tri(j, 0);
        double d = RS(P, jj + j);
        for (int k = 0; k < j; ++k) d = fma(-RS(P, jj + k), RS(P, jj + k), d);
        if (!(d > 0.0)) return false;
        const double sd = sqrt(d);
        RS(P, jj + j) = sd;
        for (int i = j + 1; i < K; ++i) {
            const int ii = bmf::tri(i, 0);
            double s = RS(P, ii + j);
            for (int k = 0; k < j; ++k) s = fma(-RS(P, ii + k), RS(P, jj + k), s);
            RS(P, ii + j) = s / sd;
        }
    }
    return true;
}

__device__ void solve_packed(const double *P, double *v, int K)
{
    for (int i = 0; i < K; ++i) {
        const int ii = bmf::tri(i, 0);
        double s = RS(v, i);
        for (int k = 0; k < i; ++k) s = fma(-RS(P, ii + k), RS(v, k), s);
        RS(v, i) = s / RS(P, ii + i);
    }
    for (int i = K - 1; i >= 0; --i) {
        double s = RS(v, i);
        for (int k = i + 1; k < K; ++k) s = fma(-RS(P, bmf::tri(k, i)), RS(v, k), s);
        RS(v, i) = s / RS(P, bmf::tri(i, i));
    }
}

// One thread per row; submodel 0 is the one whose posterior was propagated to the others.
// mu: [J][R][K], Lam: [J][R][K][K] (full symmetric), out: [R][K].
__global__ void __launch_bounds__(kThreads)
aggregate_static_kernel(int K, int64_t R, int J, const double *__restrict__ mu,
                        const double *__restrict__ Lam, double eps_rel, double *__restrict__ out,
                        double *scratch)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x;
    const int64_t n = (int64_t)blockIdx.x * kThreads + t;
    if (n >= R) return;
    const int KK = K * K, NT = bmf::ntri(K);
    unsigned long long *ncorr = reinterpret_cast<unsigned long long *>(scratch);
    unsigned long long *flags = reinterpret_cast<unsigned long long *>(scratch + 1);
    double *F = scratch + kHeaderDoubles + n * (int64_t)KK;
    double *Ls = sm + t, *Dm = Ls + NT * kThreads, *h = Dm + NT * kThreads;
    const double *L1 = Lam + n * (int64_t)KK, *m1 = mu + n * K;
    const double c0 = 2.0 - (double)J;
    double mean_diag = 0.0;
    for (int i = 0; i < K; ++i) mean_diag += L1[i * K + i];
    mean_diag /= (double)K;
    const double eps = eps_rel * (mean_diag > 1.0 ? mean_diag : 1.0);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j <= i; ++j) RS(Ls, bmf::tri(i, j)) = c0 * L1[i * K + j];
    for (int i = 0; i < K; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s = fma(L1[i * K + k], m1[k], s);
        RS(h, i) = c0 * s;
    }
    unsigned long long nc = 0;
    for (int j = 1; j < J; ++j) {
        const double *Lj = Lam + ((int64_t)j * R + n) * KK, *mj = mu + ((int64_t)j * R + n) * K;
        for (int i = 0; i < K; ++i)
            for (int k = 0; k <= i; ++k) RS(Dm, bmf::tri(i, k)) = Lj[i * K + k] - L1[i * K + k];
        // positive definiteness of the difference: FP64 Cholesky of a copy in F
        bool pd = true;
        for (int e = 0; e < NT; ++e) F[e] = RS(Dm, e);
        for (int jj = 0; jj < K && pd; ++jj) {
            const int b = bmf::tri(jj, 0);
            double d = F[b + jj];
            for (int k = 0; k < jj; ++k) d = fma(-F[b + k], F[b + k], d);
            if (!(d > 0.0)) {
                pd = false;
                break;
            }
            const double sd = sqrt(d);
            F[b + jj] = sd;
            for (int i = jj + 1; i < K; ++i) {
                const int ib = bmf::tri(i, 0);
                double s = F[ib + jj];
                for (int k = 0; k < jj; ++k) s = fma(-F[ib + k], F[b + k], s);
                F[ib + jj] = s / sd;
            }
        }
        if (!pd) {
            for (int i = 0; i < K; ++i)
                for (int k = 0; k < K; ++k)
                    F[i * K + k] = RS(Dm, i >= k ? bmf::tri(i, k) : bmf::tri(k, i));
            const double lmin = min_eig_jacobi(F, K);
            for (int i = 0; i < K; ++i) RS(Dm, bmf::tri(i, i)) += fabs(lmin) + eps;
            for (int i = 0; i < K; ++i)
                for (int k = 0; k <= i; ++k) RS(Dm, bmf::tri(i, k)) += L1[i * K + k];
            ++nc;
        } else {
            for (int i = 0; i < K; ++i)
                for (int k = 0; k <= i; ++k) RS(Dm, bmf::tri(i, k)) = Lj[i * K + k];
        }
        for (int e = 0; e < NT; ++e) RS(Ls, e) += RS(Dm, e);
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int k = 0; k < K; ++k)
                s = fma(RS(Dm, i >= k ? bmf::tri(i, k) : bmf::tri(k, i)), mj[k], s);
            RS(h, i) += s;
        }
    }
    if (!chol_packed(Ls, K)) {
        atomicOr(flags, 1ull);
        return;
    }
    solve_packed(Ls, h, K);
    for (int i = 0; i < K; ++i) out[n * K + i] = RS(h, i);
    if (nc) atomicAdd(ncorr, nc);
}

// Device address of the static array, looked up once per device with that device current and
// kept for the life of the process (a cudaDeviceReset of that device is not supported after it).
std::mutex g_mutex;
double *g_addr[kMaxDevices] = {nullptr};

bool scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return false;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return true;
}

bmf_status fail(bmf_status s, const char *m)
{
    bmf::set_noctx_error(m);
    return s;
}

}  // namespace

extern "C" bmf_status bmf_aggregate_static(int32_t K, int64_t R, int32_t J, const double *mu,
                                           const double *Lam, double eps_rel, double *mu_star,
                                           int64_t *n_corrected, void *stream)
{
    bmf::set_noctx_error("");
    if (K < 1 || K > 16 || J < 1 || R < 0)
        return fail(BMF_E_ARG, "bmf_aggregate_static: need 1 <= K <= 16, J >= 1, R >= 0");
    if ((uint64_t)R * (uint64_t)K * (uint64_t)K > kStaticDoubles - kHeaderDoubles)
        return fail(BMF_E_SHAPE, "bmf_aggregate_static: R * K * K exceeds the static scratch "
                                 "(BMF_AGGREGATE_STATIC_MAX_DOUBLES); split the rows over calls");
    if (R > 0 && (!mu || !Lam || !mu_star)) return fail(BMF_E_ARG, "bmf_aggregate_static: null pointer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(BMF_E_CUDA, "bmf_aggregate_static: no current CUDA device");
    double *scr = nullptr;
    if (!scratch_address(dev, &scr))
        return fail(BMF_E_CUDA, "bmf_aggregate_static: cudaGetSymbolAddress failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(scr, 0, kHeaderDoubles * sizeof(double), st) != cudaSuccess)
        return fail(BMF_E_CUDA, "bmf_aggregate_static: clearing the counters failed");
    if (R > 0) {
        const size_t smem = (size_t)(2 * bmf::ntri(K) + K) * kThreads * sizeof(double);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(aggregate_static_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return fail(BMF_E_CUDA, "bmf_aggregate_static: shared-memory attribute failed");
        const int grid = (int)((R + kThreads - 1) / kThreads);
        aggregate_static_kernel<<<grid, kThreads, smem, st>>>(K, R, J, mu, Lam,
                                                              eps_rel > 0 ? eps_rel : 1e-6,
                                                              mu_star, scr);
        if (cudaGetLastError() != cudaSuccess)
            return fail(BMF_E_CUDA, "bmf_aggregate_static: kernel launch failed");
    }
    unsigned long long head[2] = {0, 0};
    if (cudaMemcpyAsync(head, scr, sizeof(head), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(BMF_E_CUDA, "bmf_aggregate_static: CUDA error");
    if (n_corrected) *n_corrected = (int64_t)head[0];
    if (head[1] & 1ull)
        return fail(BMF_E_NOT_PD, "bmf_aggregate_static: an aggregated precision is not positive definite");
    return BMF_OK;
}
