// misc.cu -- the smaller kernels of the sweep and of posterior propagation:
//   * per-chunk factor statistics and the Normal-Wishart hyperparameter draw (Section 5.1 and
//     its footnote),
//   * the predictive RMSE pass (Section 5.2),
//   * moment matching of the retained samples (Section 4.1),
//   * installation of propagated priors (Algorithm 1),
//   * the eigenvalue-corrected aggregation of Algorithm 2 / Eq. 14 (Section 4.2),
//   * posterior-mean prediction.
// All FP64 except the test-set dot products of the reduced-precision modes.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

__device__ __forceinline__ void decode_tri(int e, int &i, int &j)
{
    int r = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    i = r;
    j = e - r * (r + 1) / 2;
}

// ------------------------------------------------------------------------------------------
// Factor statistics: per chunk of rows, sum_x [K] then packed lower sum_x x^T [ntri(K)], each
// entry summed over the chunk's rows in row order -- the order of the conditional kernels'
// statistics epilogue, so that a call's first hyperparameter draw (statistics from this kernel)
// equals the draw the previous call's last sweep would have made (statistics from the epilogue).
// ------------------------------------------------------------------------------------------
constexpr int kStatThreads = 256, kStatTile = 32, kStatMaxPer = 9;

__global__ void __launch_bounds__(kStatThreads)
stats_kernel(int K, const StatChunk *__restrict__ chunks, const double *__restrict__ X,
             const double *__restrict__ W, double *__restrict__ out)
{
    extern __shared__ double tile[];  // [kStatTile][K]
    const StatChunk c = chunks[blockIdx.x];
    const double *A = c.arena ? W : X;
    const int NS = K + ntri(K);
    const int t = threadIdx.x;
    double acc[kStatMaxPer];
    int ei[kStatMaxPer], ej[kStatMaxPer];
#pragma unroll
    for (int q = 0; q < kStatMaxPer; ++q) {
        acc[q] = 0.0;
        const int e = t + q * kStatThreads;
        if (e < K) {
            ei[q] = e;
            ej[q] = -1;
        } else if (e < NS) {
            decode_tri(e - K, ei[q], ej[q]);
        } else {
            ei[q] = -1;
            ej[q] = -1;
        }
    }
    for (int64_t r0 = c.r0; r0 < c.r1; r0 += kStatTile) {
        const int rows = (int)min((int64_t)kStatTile, c.r1 - r0);
        __syncthreads();
        for (int q = t; q < rows * K; q += kStatThreads) tile[q] = A[r0 * K + q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kStatMaxPer; ++q) {
            if (ei[q] < 0) continue;
            const int i = ei[q], j = ej[q];
            double s = acc[q];
            if (j < 0)
                for (int rr = 0; rr < rows; ++rr) s += tile[rr * K + i];
            else
                for (int rr = 0; rr < rows; ++rr) s = fma(tile[rr * K + i], tile[rr * K + j], s);
            acc[q] = s;
        }
    }
#pragma unroll
    for (int q = 0; q < kStatMaxPer; ++q) {
        const int e = t + q * kStatThreads;
        if (e < NS) out[(int64_t)c.out * NS + e] = acc[q];
    }
}

void launch_stats(int K, const StatChunk *chunks, int n_chunks, const double *X, const double *W,
                  double *out, cudaStream_t st)
{
    if (n_chunks <= 0) return;
    stats_kernel<<<n_chunks, kStatThreads, kStatTile * K * sizeof(double), st>>>(K, chunks, X, W,
                                                                                 out);
}

// ------------------------------------------------------------------------------------------
// Block-level dense FP64 linear algebra on K x K row-major matrices in shared memory.
// ------------------------------------------------------------------------------------------

// In-place lower Cholesky (right-looking); rinv[k] = 1 / L_kk.  Returns false (uniformly) if a
// pivot is not > 0.  Two barriers per column: the trailing update of column k uses the unscaled
// column times 1 / d_k, and column k is scaled during the next pivot step.
__device__ bool block_chol(double *A, int K, double *rinv, int *flag)
{
    const int t = threadIdx.x, T = blockDim.x;
    for (int k = 0; k < K; ++k) {
        if (t == 0) {
            const double d = A[k * K + k];
            if (!(d > 0.0)) {
                *flag = 1;
            } else {
                const double r = rsqrt(d);
                A[k * K + k] = d * r;
                rinv[k] = r;
            }
        } else if (k > 0) {
            const double r = rinv[k - 1];
            for (int i = k + t - 1; i < K; i += T - 1) A[i * K + k - 1] *= r;
        }
        __syncthreads();
        if (*flag) return false;
        const double r2 = rinv[k] * rinv[k];
        const int m = K - k - 1;
        for (int e = t; e < m * m; e += T) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * K + j] = fma(-A[i * K + k] * A[j * K + k], r2, A[i * K + j]);
        }
        __syncthreads();
    }
    // zero the strict upper triangle (column K - 1 has nothing below its pivot to scale)
    for (int e = t; e < K * K; e += T)
        if (e % K > e / K) A[e] = 0.0;
    __syncthreads();
    return true;
}

// ------------------------------------------------------------------------------------------
// First level of the statistics sum of the hyperparameter step: block (p, j) sums, entry by
// entry in chunk order, the p-th of kStatParts equal runs of job j's chunks into partial
// (j0 + j) * kStatParts + p (zero for an empty run).  The hyperparameter kernel then sums the
// kStatParts partials of its job in order.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) stats_reduce_kernel(int K, const HyperJob *__restrict__ jobs,
                                                           int j0, const double *__restrict__ stats,
                                                           double *__restrict__ out)
{
    const int NS = K + ntri(K);
    const HyperJob jb = jobs[blockIdx.y];
    const int n = jb.chunk1 - jb.chunk0;
    const int len = (n + kStatParts - 1) / kStatParts;
    const int c0 = jb.chunk0 + min(n, (int)blockIdx.x * len), c1 = jb.chunk0 + min(n, ((int)blockIdx.x + 1) * len);
    double *dst = out + ((int64_t)(j0 + blockIdx.y) * kStatParts + blockIdx.x) * NS;
    for (int e = threadIdx.x; e < NS; e += blockDim.x) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int c = c0;
        for (; c + 3 < c1; c += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += stats[(int64_t)(c + u) * NS + e];
        }
        for (; c < c1; ++c) acc[0] += stats[(int64_t)c * NS + e];
        dst[e] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
}

void launch_stats_reduce(int K, const HyperJob *jobs, int n_jobs, int j0, const double *stats,
                         double *out, cudaStream_t st)
{
    if (n_jobs <= 0) return;
    stats_reduce_kernel<<<dim3(kStatParts, n_jobs), 256, 0, st>>>(K, jobs, j0, stats, out);
}

// ------------------------------------------------------------------------------------------
// Normal-Wishart hyperparameter draw: one block per (subset, factor) job.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) hyper_kernel(HyperParams a)
{
    const HyperJob jb = a.jobs[blockIdx.x];
    const int K = a.K, KK = K * K, NS = K + ntri(K);
    const int t = threadIdx.x, T = blockDim.x;
    extern __shared__ double s[];
    double *M = s, *C = M + KK, *L = C + KK, *B = L + KK;
    double *s1 = B + KK, *xbar = s1 + K, *mus = xbar + K, *v = mus + K, *mu = v + K;
    double *rinv = mu + K;  // [K] reciprocal pivots
    double *red = rinv + K;  // [T] stripe partial sums
    __shared__ int flag;
    if (t == 0) flag = 0;
    // 1. sum the chunk statistics: each entry is split over `ns` stripes of chunks, each
    //    stripe summed with eight independent accumulators, then the stripes in order (a fixed
    //    order for a given block size, so the result is deterministic)
    const int ns = NS < T ? T / NS : 1;
    for (int q = t; q < ns * NS; q += T) {
        const int e = q % NS, sidx = q / NS;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int c = jb.chunk0 + sidx;
        for (; c + 7 * ns < jb.chunk1; c += 8 * ns) {
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += a.stats[(int64_t)(c + u * ns) * NS + e];
        }
        for (; c < jb.chunk1; c += ns) acc[0] += a.stats[(int64_t)c * NS + e];
        const double part = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
        if (ns > 1)
            red[q] = part;
        else if (e < K)
            s1[e] = part;
        else {
            int i, j;
            decode_tri(e - K, i, j);
            M[i * K + j] = part;
            M[j * K + i] = part;
        }
    }
    __syncthreads();
    if (ns > 1) {
        for (int e = t; e < NS; e += T) {
            double acc = 0.0;
            for (int sidx = 0; sidx < ns; ++sidx) acc += red[sidx * NS + e];
            if (e < K) {
                s1[e] = acc;
            } else {
                int i, j;
                decode_tri(e - K, i, j);
                M[i * K + j] = acc;
                M[j * K + i] = acc;
            }
        }
        __syncthreads();
    }
    const double N = (double)jb.n;
    const double bstar = a.beta0 + N;
    for (int e = t; e < K; e += T) {
        xbar[e] = N > 0 ? s1[e] / N : 0.0;
        mus[e] = (a.beta0 * a.mu0[e] + N * (N > 0 ? s1[e] / N : 0.0)) / bstar;
    }
    __syncthreads();
    // 2. [W*]^{-1} = W0^{-1} + N Sbar + (beta0 N / beta*) (mu0 - xbar)(mu0 - xbar)^T with the
    //    centred Sbar = (1/N) sum x x^T - xbar xbar^T
    const double cw = a.beta0 * N / bstar;
    for (int e = t; e < KK; e += T) {
        const int i = e / K, j = e % K;
        const double Sb = N > 0 ? M[e] / N - xbar[i] * xbar[j] : 0.0;
        C[e] = a.W0inv[e] + N * Sb + cw * (a.mu0[i] - xbar[i]) * (a.mu0[j] - xbar[j]);
    }
    __syncthreads();
    // 3. the lower Cholesky factor of W* = ([W*]^{-1})^{-1} without forming W*: with P the
    //    order reversal, P [W*]^{-1} P = R R^T (R lower) gives W* = (P R^{-T} P)(P R^{-T} P)^T,
    //    and P R^{-T} P is lower with a positive diagonal, so it is that factor
    for (int e = t; e < KK; e += T) L[e] = C[(KK - 1) - e];
    __syncthreads();
    if (!block_chol(L, K, rinv, &flag)) goto fail;
    for (int c = t; c < K; c += T) {           // R^{-1} (lower) into M, a column per thread
        for (int i = 0; i < c; ++i) M[i * K + c] = 0.0;
        for (int i = c; i < K; ++i) {
            double acc = i == c ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) acc = fma(-L[i * K + k], M[k * K + c], acc);
            M[i * K + c] = acc * rinv[i];
        }
    }
    __syncthreads();
    // 4. L = P R^{-T} P: L_ij = (R^{-1})_{K-1-j, K-1-i}
    for (int e = t; e < KK; e += T) {
        const int i = e / K, j = e % K;
        L[e] = j <= i ? M[(K - 1 - j) * K + (K - 1 - i)] : 0.0;
    }
    __syncthreads();
    // 5. Bartlett factor A (lower) in B
    {
        const double *dr = a.draws + jb.draw;
        const int nlow = K * (K - 1) / 2;
        for (int e = t; e < KK; e += T) {
            const int i = e / K, j = e % K;
            double val = 0.0;
            if (i == j)
                val = sqrt(dr[i]);
            else if (j < i)
                val = dr[K + i * (i - 1) / 2 + j];
            B[e] = val;
        }
        if (t < K) v[t] = dr[K + nlow + t];   // z_mu
    }
    __syncthreads();
    // 6. C = L A (lower), Lambda = C C^T in M
    for (int e = t; e < KK; e += T) {
        const int i = e / K, j = e % K;
        double acc = 0.0;
        if (j <= i)
            for (int k = j; k <= i; ++k) acc = fma(L[i * K + k], B[k * K + j], acc);
        C[e] = acc;
    }
    __syncthreads();
    for (int e = t; e < KK; e += T) {
        const int i = e / K, j = e % K;
        double acc = 0.0;
        const int kmax = min(i, j);
        for (int k = 0; k <= kmax; ++k) acc = fma(C[i * K + k], C[j * K + k], acc);
        M[e] = acc;
    }
    __syncthreads();
    // 7. mu = mu* + chol(beta* Lambda)^{-T} z_mu, where chol(beta* Lambda) = sqrt(beta*) L A
    //    (L A is lower with a positive diagonal and (L A)(L A)^T = Lambda)
    for (int i = t; i < K; i += T) {
        const double d = C[i * K + i];
        if (!(d > 0.0)) flag = 1;
        rinv[i] = 1.0 / d;
    }
    __syncthreads();
    if (flag) goto fail;
    if (t == 0) {
        const double sb = rsqrt(bstar);
        for (int i = K - 1; i >= 0; --i) {
            double acc = v[i];
            for (int k = i + 1; k < K; ++k) acc = fma(-C[k * K + i], v[k], acc);
            v[i] = acc * rinv[i];
        }
        for (int i = 0; i < K; ++i) mu[i] = fma(v[i], sb, mus[i]);
    }
    __syncthreads();
    // 8. write the slot: mu, Lambda (packed lower), b = Lambda mu
    {
        double *slot = a.hyper + (int64_t)jb.slot * hyper_slot_len(K);
        for (int e = t; e < K; e += T) slot[e] = mu[e];
        for (int e = t; e < ntri(K); e += T) {
            int i, j;
            decode_tri(e, i, j);
            slot[K + e] = M[i * K + j];
        }
        for (int i = t; i < K; i += T) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc = fma(M[i * K + k], mu[k], acc);
            slot[K + ntri(K) + i] = acc;
        }
    }
    return;
fail:
    if (t == 0) atomicOr(&a.err->flags, ERR_NOT_PD);
}

void launch_hyper(const HyperParams &a, cudaStream_t st)
{
    if (a.n_jobs <= 0) return;
    const size_t smem = (size_t)(4 * a.K * a.K + 6 * a.K + 256) * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(hyper_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    hyper_kernel<<<a.n_jobs, 256, smem, st>>>(a);
}

// ------------------------------------------------------------------------------------------
// Predictive RMSE of the current sample and of the running mean (Section 5.2).
// ------------------------------------------------------------------------------------------
// Dot product of two gathered rows (ldg elements, zero padded) with 16-byte vector loads.
__device__ __forceinline__ float dot_rows(const float *x, const float *w, int ldg)
{
    const float4 *a = reinterpret_cast<const float4 *>(x), *b = reinterpret_cast<const float4 *>(w);
    float s = 0.f;
    for (int v = 0; v < ldg / 4; ++v) {
        const float4 p = __ldg(a + v), q = __ldg(b + v);
        s = fmaf(p.x, q.x, s);
        s = fmaf(p.y, q.y, s);
        s = fmaf(p.z, q.z, s);
        s = fmaf(p.w, q.w, s);
    }
    return s;
}
__device__ __forceinline__ double dot_rows(const double *x, const double *w, int ldg)
{
    const double2 *a = reinterpret_cast<const double2 *>(x), *b = reinterpret_cast<const double2 *>(w);
    double s = 0.0;
    for (int v = 0; v < ldg / 2; ++v) {
        const double2 p = __ldg(a + v), q = __ldg(b + v);
        s = fma(p.x, q.x, s);
        s = fma(p.y, q.y, s);
    }
    return s;
}
__device__ __forceinline__ float dot_rows(const __nv_bfloat16 *x, const __nv_bfloat16 *w, int ldg)
{
    const uint4 *a = reinterpret_cast<const uint4 *>(x), *b = reinterpret_cast<const uint4 *>(w);
    float s = 0.f;
    for (int v = 0; v < ldg / 8; ++v) {
        uint4 p = __ldg(a + v), q = __ldg(b + v);
        const __nv_bfloat162 *pp = reinterpret_cast<const __nv_bfloat162 *>(&p);
        const __nv_bfloat162 *qq = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 u = __bfloat1622float2(pp[h]), t = __bfloat1622float2(qq[h]);
            s = fmaf(u.x, t.x, s);
            s = fmaf(u.y, t.y, s);
        }
    }
    return s;
}

template <typename GT>
__global__ void __launch_bounds__(256) rmse_kernel(RmseParams a)
{
    const GT *Xg = static_cast<const GT *>(a.Xg), *Wg = static_cast<const GT *>(a.Wg);
    // the dot product in the gather precision, widened on the integer pipe; five FP64
    // operations per entry (this pass shares the FP64 pipe with the conditional draws)
    double s0 = 0.0, s1 = 0.0;
    const bool mean = a.inv_kept > 0.0;
    for (int64_t e = a.t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.t1;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double yh = widen(dot_rows(Xg + (int64_t)a.trow[e] * a.ldg,
                                         Wg + (int64_t)a.tcol[e] * a.ldg, a.ldg));
        const double y = a.tval[e];
        const double d0 = y - yh;
        s0 = fma(d0, d0, s0);
        if (a.keep) {
            const double ys = a.ysum[e] + yh;
            a.ysum[e] = ys;
            const double d1 = fma(-ys, a.inv_kept, y);
            s1 = fma(d1, d1, s1);
        } else if (mean) {
            const double d1 = fma(-a.ysum[e], a.inv_kept, y);
            s1 = fma(d1, d1, s1);
        }
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.partial[2 * blockIdx.x] = red[0][0];
        a.partial[2 * blockIdx.x + 1] = red[1][0];
    }
}

// Deterministic final sum: each thread sums a fixed strided subset, then a fixed tree.
__global__ void __launch_bounds__(256) rmse_final_kernel(const double *partial, int blocks,
                                                         double *out2)
{
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < blocks; k += 256) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            red[0][threadIdx.x] += red[0][threadIdx.x + o];
            red[1][threadIdx.x] += red[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = red[0][0];
        out2[1] = red[1][0];
    }
}

void launch_rmse(const RmseParams &a, int blocks, cudaStream_t st)
{
    if (a.prec == BMF_FP64)
        rmse_kernel<double><<<blocks, 256, 0, st>>>(a);
    else if (a.prec == BMF_FP32)
        rmse_kernel<float><<<blocks, 256, 0, st>>>(a);
    else
        rmse_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(a);
}

void launch_rmse_final(const double *partial, int blocks, double *out2, cudaStream_t st)
{
    rmse_final_kernel<<<1, 256, 0, st>>>(partial, blocks, out2);
}

// ------------------------------------------------------------------------------------------
// Thread-per-row FP64 helpers on packed lower matrices in interleaved shared memory: entry e of
// a thread's matrix at base[e * rb], rb = threads per block (32, fewer when K is large enough
// that 32 rows' matrices would not fit in shared memory).
// ------------------------------------------------------------------------------------------
constexpr int kRowBlock = 32;
constexpr size_t kRowSmemCap = 200 * 1024;
#define RS(base, e) (base)[(e) * rb]

// Threads per block of a thread-per-row kernel holding `per_row` doubles per row.
static int row_block(size_t per_row)
{
    const size_t fit = kRowSmemCap / (per_row * sizeof(double));
    return (int)(fit >= (size_t)kRowBlock ? kRowBlock : (fit < 1 ? 1 : fit));
}

// In-place packed lower Cholesky (Crout order) with one reciprocal square root per pivot and no
// division: L_jj in P, 1 / L_jj in ri.  Returns false if a pivot is not > 0.
__device__ bool row_chol(double *P, double *ri, int K, int rb)
{
    for (int j = 0; j < K; ++j) {
        const int jj = tri(j, 0);
        double d = RS(P, jj + j);
        for (int k = 0; k < j; ++k) d = fma(-RS(P, jj + k), RS(P, jj + k), d);
        if (!(d > 0.0)) return false;
        const double rs = rsqrt(d);
        RS(ri, j) = rs;
        RS(P, jj + j) = d * rs;
        for (int i = j + 1; i < K; ++i) {
            const int ii = tri(i, 0);
            double s = RS(P, ii + j);
            for (int k = 0; k < j; ++k) s = fma(-RS(P, ii + k), RS(P, jj + k), s);
            RS(P, ii + j) = s * rs;
        }
    }
    return true;
}

// Solve (L L^T) x = b in place in vector v (interleaved), L packed in P, 1 / L_ii in ri.
__device__ void row_solve(const double *P, const double *ri, double *v, int K, int rb)
{
    for (int i = 0; i < K; ++i) {
        const int ii = tri(i, 0);
        double s = RS(v, i);
        for (int k = 0; k < i; ++k) s = fma(-RS(P, ii + k), RS(v, k), s);
        RS(v, i) = s * RS(ri, i);
    }
    for (int i = K - 1; i >= 0; --i) {
        double s = RS(v, i);
        for (int k = i + 1; k < K; ++k) s = fma(-RS(P, tri(k, i)), RS(v, k), s);
        RS(v, i) = s * RS(ri, i);
    }
}

// ------------------------------------------------------------------------------------------
// Moment matching: mu = S1/S, Sigma = S2/S - mu mu^T, Lambda = Sigma^{-1}, b = Lambda mu.
// Sigma = L L^T in place, then W = L^{-1} in place (columns left to right; W_ij =
// -(1/L_ii) sum_{k=j}^{i-1} L_ik W_kj reads only entries of L right of column j and entries of W
// already written), then Lambda = W^T W in place (rows top to bottom through a K-vector: row i
// of Lambda needs only rows k >= i of W), then b.  K^3/2 multiply-adds and no division.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kRowBlock) mm_kernel(MMParams a)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x, rb = blockDim.x;
    const int64_t r = a.r0 + (int64_t)blockIdx.x * rb + t;
    if (r >= a.r1) return;
    const int K = a.K, NT = ntri(K);
    const int64_t R = a.R;
    double *A = sm + t, *mu = A + NT * rb, *v = mu + K * rb;
    const double inv = 1.0 / a.S;
    for (int i = 0; i < K; ++i) RS(mu, i) = a.S1[(int64_t)i * R + r] * inv;
    for (int i = 0; i < K; ++i) {
        const double mi = RS(mu, i);
        for (int j = 0; j <= i; ++j)
            RS(A, tri(i, j)) = fma(-mi, RS(mu, j), a.S2[(int64_t)tri(i, j) * R + r] * inv);
    }
    if (!row_chol(A, v, K, rb)) {
        atomicOr(&a.err->flags, ERR_NOT_PD);
        atomicMin(&a.err->first_bad_row, (int)r);
        return;
    }
    for (int j = 0; j < K; ++j) {
        RS(A, tri(j, j)) = RS(v, j);
        for (int i = j + 1; i < K; ++i) {
            const int ii = tri(i, 0);
            double s = 0.0;
            for (int k = j; k < i; ++k) s = fma(RS(A, ii + k), RS(A, tri(k, j)), s);
            RS(A, ii + j) = -s * RS(v, i);
        }
    }
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = 0.0;
            for (int k = i; k < K; ++k) s = fma(RS(A, tri(k, i)), RS(A, tri(k, j)), s);
            RS(v, j) = s;
        }
        for (int j = 0; j <= i; ++j) RS(A, tri(i, j)) = RS(v, j);
    }
    for (int i = 0; i < K; ++i) a.mu[r * K + i] = RS(mu, i);
    for (int e = 0; e < NT; ++e) a.L[(int64_t)e * R + r] = RS(A, e);
    for (int i = 0; i < K; ++i) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k)
            acc = fma(RS(A, i >= k ? tri(i, k) : tri(k, i)), RS(mu, k), acc);
        a.b[(int64_t)i * R + r] = acc;
    }
}

void launch_mm(const MMParams &a, cudaStream_t st)
{
    const int64_t n = a.r1 - a.r0;
    if (n <= 0) return;
    const size_t per_row = (size_t)(ntri(a.K) + 2 * a.K);
    const int rb = row_block(per_row);
    const size_t smem = per_row * rb * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(mm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mm_kernel<<<(int)((n + rb - 1) / rb), rb, smem, st>>>(a);
}

// ------------------------------------------------------------------------------------------
// Propagated priors: destination rows get the source rows' moment-matched Gaussian as prior
// and start their chain at its mean.
// ------------------------------------------------------------------------------------------
template <typename GT>
__global__ void propagate_kernel(PropParams a)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.n) return;
    const int64_t s = a.src0 + q, d = a.dst0 + q;
    const int K = a.K;
    for (int e = 0; e < ntri(K); ++e) a.pL[(int64_t)e * a.R + d] = a.L[(int64_t)e * a.R + s];
    for (int i = 0; i < K; ++i) a.pb[(int64_t)i * a.R + d] = a.b[(int64_t)i * a.R + s];
    GT *g = static_cast<GT *>(a.Xg) + d * a.ldg;
    for (int i = 0; i < a.ldg; ++i) {
        const double x = i < K ? a.mu[s * K + i] : 0.0;
        if (i < K) a.X[d * K + i] = x;
        if constexpr (sizeof(GT) == 2)
            g[i] = __double2bfloat16(x);
        else
            g[i] = (GT)x;
    }
}

void launch_propagate(const PropParams &a, cudaStream_t st)
{
    if (a.n <= 0) return;
    const int grid = (int)((a.n + 127) / 128);
    if (a.prec == BMF_FP64)
        propagate_kernel<double><<<grid, 128, 0, st>>>(a);
    else if (a.prec == BMF_FP32)
        propagate_kernel<float><<<grid, 128, 0, st>>>(a);
    else
        propagate_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>(a);
}

// ------------------------------------------------------------------------------------------
// Algorithm 2 (Eq. 14 with the eigenvalue correction), thread per row.
// ------------------------------------------------------------------------------------------

// Smallest eigenvalue of the symmetric matrix held packed-lower in A (interleaved; destroyed):
// Householder reduction to tridiagonal form T = Q^T A Q (Golub & Van Loan, Algorithm 8.3.1),
// then bisection on the Sturm count of T (the sign changes of the leading principal minors of
// T - x I equal the number of eigenvalues below x; Golub & Van Loan, Section 8.4.1) to an
// interval of 2^-50 |T|, the rounding level of the count.  The result is the smallest
// eigenvalue to O(2^-50 |A|).  v: K scratch slots, dg / of: the K diagonal and K - 1
// off-diagonal entries of T (of: their squares, scaled, after the reduction).
__device__ double min_eig_tridiag(double *A, double *v, double *dg, double *of, int K, int rb)
{
#define AP(i, j) RS(A, (i) >= (j) ? tri(i, j) : tri(j, i))
    for (int k = 0; k + 2 < K; ++k) {
        // Householder vector of the column below the diagonal, x = A(k+1 .., k)
        double nrm2 = 0.0;
        for (int i = k + 1; i < K; ++i) nrm2 = fma(AP(i, k), AP(i, k), nrm2);
        RS(dg, k) = AP(k, k);
        const double x0 = AP(k + 1, k);
        if (nrm2 == 0.0) {
            RS(of, k) = 0.0;
            continue;
        }
        const double nrm = sqrt(nrm2);
        const double alpha = x0 >= 0.0 ? -nrm : nrm;   // H x = alpha e_1
        RS(of, k) = alpha;
        const double beta = 1.0 / (nrm2 - x0 * alpha);  // 2 / (v^T v), v = x - alpha e_1
        for (int i = k + 1; i < K; ++i) RS(v, i) = AP(i, k);
        RS(v, k + 1) = x0 - alpha;
        // p = beta B v (B the trailing block), then w = p - (beta p^T v / 2) v; the w values
        // replace column k of A, which is not read again
        double pv = 0.0;
        for (int i = k + 1; i < K; ++i) {
            double s = 0.0;
            for (int j = k + 1; j < K; ++j) s = fma(AP(i, j), RS(v, j), s);
            s *= beta;
            RS(A, tri(i, k)) = s;
            pv = fma(s, RS(v, i), pv);
        }
        const double kk = 0.5 * beta * pv;
        for (int i = k + 1; i < K; ++i) RS(A, tri(i, k)) = fma(-kk, RS(v, i), RS(A, tri(i, k)));
        // B -= v w^T + w v^T (lower triangle)
        for (int i = k + 1; i < K; ++i) {
            const double vi = RS(v, i), wi = RS(A, tri(i, k));
            for (int j = k + 1; j <= i; ++j)
                RS(A, tri(i, j)) = fma(-vi, RS(A, tri(j, k)), fma(-wi, RS(v, j), RS(A, tri(i, j))));
        }
    }
    if (K >= 2) {
        RS(dg, K - 2) = AP(K - 2, K - 2);
        RS(of, K - 2) = AP(K - 1, K - 2);
    }
    RS(dg, K - 1) = AP(K - 1, K - 1);
#undef AP
    // Gershgorin interval of T; lambda_min <= min_i T_ii (the Rayleigh quotient of e_i) lowers
    // its top end
    double lo = 0.0, hi = 0.0, dmin = 0.0;
    for (int i = 0; i < K; ++i) {
        const double r = (i > 0 ? fabs(RS(of, i - 1)) : 0.0) + (i + 1 < K ? fabs(RS(of, i)) : 0.0);
        const double a = RS(dg, i) - r, b = RS(dg, i) + r;
        lo = i == 0 ? a : fmin(lo, a);
        hi = i == 0 ? b : fmax(hi, b);
        dmin = i == 0 ? RS(dg, i) : fmin(dmin, RS(dg, i));
    }
    const double nrm = fmax(fabs(lo), fabs(hi));
    if (!(nrm > 0.0)) return 0.0;
    // T / s with s the power of two at or above the norm bound (exact scaling): entries and the
    // bisection interval within [-1, 1], so the Sturm sequence below neither overflows nor, short
    // of K near-coincident eigenvalues, underflows
    const int se = ilogb(nrm) + 1;
    for (int i = 0; i < K; ++i) RS(dg, i) = scalbn(RS(dg, i), -se);
    for (int i = 0; i + 1 < K; ++i) {
        const double e = scalbn(RS(of, i), -se);
        RS(of, i) = e * e;
    }
    lo = scalbn(lo, -se);
    hi = fmin(scalbn(hi, -se), scalbn(dmin, -se) + 0x1.0p-44);
    // bisection on the Sturm count: the number of sign changes of p_0 = 1, p_1 = d_0 - x,
    // p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1} (the leading principal minors of T - x I, a zero
    // taking the sign opposite to its predecessor) is the number of eigenvalues below x
    // (Golub & Van Loan, Section 8.4.1); no division, signs read from the bit patterns
    for (int it = 0; it < 100 && hi - lo > 0x1.0p-50; ++it) {
        const double x = 0.5 * (lo + hi);
        double pm = 1.0, pc = RS(dg, 0) - x;
        long long bc = __double_as_longlong(pc);
        unsigned sc = (bc << 1) == 0 ? 1u : (unsigned)((unsigned long long)bc >> 63);
        unsigned below = sc;
        for (int i = 1; i < K; ++i) {
            double pn = fma(RS(dg, i) - x, pc, -RS(of, i - 1) * pm);
            const int em = max((int)((__double_as_longlong(pn) >> 52) & 0x7ff),
                               (int)((__double_as_longlong(pc) >> 52) & 0x7ff));
            if (em < 1023 - 600) {
                // both terms below 2^-600: rescale them by the same power of two (exact)
                const double f = scalbn(1.0, 1023 - max(em, 1));
                pn *= f;
                pc *= f;
            }
            const long long b2 = __double_as_longlong(pn);
            const unsigned sn = (b2 << 1) == 0 ? (sc ^ 1u) : (unsigned)((unsigned long long)b2 >> 63);
            below += sn ^ sc;
            pm = pc;
            pc = pn;
            sc = sn;
        }
        if (below >= 1)
            hi = x;
        else
            lo = x;
    }
    return scalbn(0.5 * (lo + hi), se);
}

// Algorithm 2 in two passes.  Pass 1, one thread per (row n, submodel j >= 1): the difference
// Lambda^(j) - Lambda^(1) is tested for positive definiteness by a Cholesky factorisation; if a
// pivot is not > 0, corr = |lambda_min| + eps (> 0), else corr = 0.  Pass 2, one thread per row:
// Lambda* = (2 - J) Lambda^(1) + sum_j Lambda*^(j) with Lambda*^(j) = Lambda^(j) when corr = 0,
// else (Lambda^(j) - Lambda^(1) + corr I) + Lambda^(1); the same for the right-hand side
// Lambda* mu* = (2 - J) Lambda^(1) mu^(1) + sum_j Lambda*^(j) mu^(j); then Cholesky and solve.
// Splitting keeps few slots per thread in shared memory, so several warps share an SM.

// In-place packed lower Cholesky used only as a positive-definiteness test (pivot > 0 at every
// step), scaling by one reciprocal per column.
__device__ bool row_pd_test(double *P, int K, int rb)
{
    for (int j = 0; j < K; ++j) {
        const int jj = tri(j, 0);
        double d = RS(P, jj + j);
        for (int k = 0; k < j; ++k) d = fma(-RS(P, jj + k), RS(P, jj + k), d);
        if (!(d > 0.0)) return false;
        const double r = rsqrt(d);
        for (int i = j + 1; i < K; ++i) {
            const int ii = tri(i, 0);
            double s = RS(P, ii + j);
            for (int k = 0; k < j; ++k) s = fma(-RS(P, ii + k), RS(P, jj + k), s);
            RS(P, ii + j) = s * r;
        }
    }
    return true;
}

static inline size_t agg_pd_slots(int K) { return (size_t)ntri(K); }
static inline size_t agg_corr_slots(int K) { return (size_t)ntri(K) + 3 * K; }

// Pass 1a, one thread per (row n, submodel j >= 1): corr = 0 where the difference is positive
// definite, else the pair is appended to a list for pass 1b (one atomic per warp).  Splitting
// the eigenvalue off keeps pass 1b's warps free of pairs that need none (otherwise a warp's
// positive-definite pairs idle while its others take the eigenvalue path).
__global__ void __launch_bounds__(kRowBlock) aggregate_pd_kernel(AggParams a, int64_t n_pairs)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x, rb = blockDim.x;
    const int64_t q = (int64_t)blockIdx.x * rb + t;
    bool listed = false;
    if (q < n_pairs) {
        const int K = a.K, NT = ntri(K);
        const int j = 1 + (int)(q / a.n_rows);
        const int64_t n = q % a.n_rows;
        double *Fm = sm + t;
        const int64_t r1 = a.sub_base[0] + n, rj = a.sub_base[j] + n;
        for (int e = 0; e < NT; ++e) RS(Fm, e) = a.L[(int64_t)e * a.R + rj] - a.L[(int64_t)e * a.R + r1];
        if (row_pd_test(Fm, K, rb))
            a.corr[q] = 0.0;
        else
            listed = true;
    }
    const unsigned am = __activemask();
    const unsigned votes = __ballot_sync(am, listed);
    const int lane = t & 31, leader = __ffs(am) - 1;
    unsigned base = 0;
    if (lane == leader && votes) base = atomicAdd(a.list_n, (unsigned)__popc(votes));
    base = __shfl_sync(am, base, leader);
    if (listed) a.list[base + __popc(votes & ((1u << lane) - 1u))] = (int32_t)q;
}

// Pass 1b, one thread per listed pair: corr = |lambda_min| + eps (Algorithm 2).
__global__ void __launch_bounds__(kRowBlock) aggregate_eig_kernel(AggParams a)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x, rb = blockDim.x;
    const int64_t k = (int64_t)blockIdx.x * rb + t;
    if ((int64_t)blockIdx.x * rb >= (int64_t)*a.list_n) return;    // the whole block is past the list
    unsigned long long nc = 0;
    if (k < (int64_t)*a.list_n) {
        const int K = a.K, NT = ntri(K);
        const int64_t q = a.list[k];
        const int j = 1 + (int)(q / a.n_rows);
        const int64_t n = q % a.n_rows;
        double *Fm = sm + t, *v = Fm + NT * rb, *dg = v + K * rb, *of = dg + K * rb;
        const int64_t r1 = a.sub_base[0] + n, rj = a.sub_base[j] + n;
        double mean_diag = 0.0;
        for (int i = 0; i < K; ++i) mean_diag += a.L[(int64_t)tri(i, i) * a.R + r1];
        mean_diag /= (double)K;
        const double eps = a.eps_rel * (mean_diag > 1.0 ? mean_diag : 1.0);
        for (int e = 0; e < NT; ++e) RS(Fm, e) = a.L[(int64_t)e * a.R + rj] - a.L[(int64_t)e * a.R + r1];
        a.corr[q] = fabs(min_eig_tridiag(Fm, v, dg, of, K, rb)) + eps;
        nc = 1;
    }
    // one atomic per warp (the block may end in a partial warp: only its existing lanes vote)
    const unsigned am = __activemask();
    const unsigned votes = __ballot_sync(am, nc != 0);
    if ((t & 31) == __ffs(am) - 1 && votes) atomicAdd(a.n_corrected, (unsigned long long)__popc(votes));
}

static inline size_t agg_slots(int K) { return (size_t)2 * ntri(K) + 2 * K; }

__global__ void __launch_bounds__(kRowBlock) aggregate_kernel(AggParams a)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x, rb = blockDim.x;
    const int64_t n = (int64_t)blockIdx.x * rb + t;
    if (n >= a.n_rows) return;
    const int K = a.K, NT = ntri(K), J = a.J;
    double *Ls = sm + t, *Dm = Ls + NT * rb, *h = Dm + NT * rb, *ri = h + K * rb;
    const int64_t r1 = a.sub_base[0] + n;
    const double c0 = 2.0 - (double)J;
    for (int e = 0; e < NT; ++e) RS(Ls, e) = c0 * a.L[(int64_t)e * a.R + r1];
    for (int i = 0; i < K; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k)
            s = fma(a.L[(int64_t)(i >= k ? tri(i, k) : tri(k, i)) * a.R + r1], a.mu[r1 * K + k], s);
        RS(h, i) = c0 * s;
    }
    for (int j = 1; j < J; ++j) {
        const int64_t rj = a.sub_base[j] + n;
        const double corr = a.corr[(int64_t)(j - 1) * a.n_rows + n];
        if (corr > 0.0) {
            for (int i = 0; i < K; ++i)
                for (int k = 0; k <= i; ++k) {
                    const int e = tri(i, k);
                    const double l1 = a.L[(int64_t)e * a.R + r1];
                    double dd = a.L[(int64_t)e * a.R + rj] - l1;
                    if (i == k) dd += corr;
                    RS(Dm, e) = dd + l1;
                }
        } else {
            for (int e = 0; e < NT; ++e) RS(Dm, e) = a.L[(int64_t)e * a.R + rj];
        }
        for (int e = 0; e < NT; ++e) RS(Ls, e) += RS(Dm, e);
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int k = 0; k < K; ++k)
                s = fma(RS(Dm, i >= k ? tri(i, k) : tri(k, i)), a.mu[rj * K + k], s);
            RS(h, i) += s;
        }
    }
    if (!row_chol(Ls, ri, K, rb)) {
        atomicOr(&a.err->flags, ERR_NOT_PD);
        atomicMin(&a.err->first_bad_row, (int)n);
        return;
    }
    row_solve(Ls, ri, h, K, rb);
    for (int i = 0; i < K; ++i) a.out[n * K + i] = RS(h, i);
}

// Threads per block for a thread-per-row kernel with `per_row` shared slots: at most
// kRowBlock, fewer when the block would not leave room for four blocks per SM.
static int row_block_small(size_t per_row)
{
    const size_t fit = (size_t)(220 * 1024 / 4) / (per_row * sizeof(double));
    return (int)(fit >= (size_t)kRowBlock ? kRowBlock : (fit < 1 ? 1 : fit));
}

void launch_aggregate(const AggParams &a, cudaStream_t st)
{
    if (a.n_rows <= 0) return;
    const int64_t n_pairs = a.n_rows * (int64_t)(a.J - 1);
    if (n_pairs > 0) {
        cudaMemsetAsync(a.list_n, 0, sizeof(unsigned), st);
        {
            const size_t per = agg_pd_slots(a.K);
            const int rb = row_block_small(per);
            const size_t smem = per * rb * sizeof(double);
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(aggregate_pd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            aggregate_pd_kernel<<<(int)((n_pairs + rb - 1) / rb), rb, smem, st>>>(a, n_pairs);
        }
        const size_t per = agg_corr_slots(a.K);
        const int rb = row_block_small(per);
        const size_t smem = per * rb * sizeof(double);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(aggregate_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        aggregate_eig_kernel<<<(int)((n_pairs + rb - 1) / rb), rb, smem, st>>>(a);
    }
    const size_t per = agg_slots(a.K);
    const int rb = row_block_small(per);
    const size_t smem = per * rb * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(aggregate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    aggregate_kernel<<<(int)((a.n_rows + rb - 1) / rb), rb, smem, st>>>(a);
}

// ------------------------------------------------------------------------------------------
// Posterior-mean prediction (Section 5.2) and the chain-restart gather.
// ------------------------------------------------------------------------------------------
// One factor block with a single submodel: its posterior mean is the mean of the retained
// samples, out[r][k] = S1[k][base + r] * inv_kept.
__global__ void mean_rows_kernel(int K, int64_t n, const double *S1, int64_t R, int64_t base,
                                 double inv_kept, double *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * K) return;
    const int64_t r = q / K;
    const int k = (int)(q % K);
    out[q] = S1[(int64_t)k * R + base + r] * inv_kept;
}

void launch_mean_rows(int K, int64_t n, const double *S1, int64_t R, int64_t base,
                      double inv_kept, double *out, cudaStream_t st)
{
    if (n <= 0) return;
    const int64_t m = n * K;
    mean_rows_kernel<<<(int)((m + 255) / 256), 256, 0, st>>>(K, n, S1, R, base, inv_kept, out);
}

// y_hat = offset + Xm[row]^T Wm[col] (indices mapped through the rank arrays when given), and
// with y the per-block sums of (y - y_hat)^2 (each thread a fixed strided subset, then a fixed
// tree: deterministic).
__global__ void __launch_bounds__(256) predict_sq_kernel(PredictParams p)
{
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < p.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rr = p.row_rank ? p.row_rank[p.row[e]] : (int64_t)p.row[e];
        const int64_t cc = p.col_rank ? p.col_rank[p.col[e]] : (int64_t)p.col[e];
        const double *x = p.Xm + rr * p.K, *w = p.Wm + cc * p.K;
        double d = 0.0;
        for (int k = 0; k < p.K; ++k) d = fma(x[k], w[k], d);
        const double yh = p.offset + d;
        if (p.yhat) p.yhat[e] = yh;
        if (p.y) {
            const double r = p.y[e] - yh;
            s = fma(r, r, s);
        }
    }
    if (!p.partial) return;
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        p.partial[2 * blockIdx.x] = red[0];
        p.partial[2 * blockIdx.x + 1] = 0.0;
    }
}

void launch_predict_sq(const PredictParams &p, int blocks, cudaStream_t st)
{
    predict_sq_kernel<<<blocks, 256, 0, st>>>(p);
}

// out[a][k] = in[src[a]][k]: every subset's block of a factor arena from a factor in the
// original order.
__global__ void gather_rows_kernel(int K, int64_t R, const int64_t *src, const double *in,
                                   double *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R * K) return;
    const int64_t a = q / K;
    const int k = (int)(q % K);
    out[q] = in[src[a] * K + k];
}

void launch_gather_rows(int K, int64_t R, const int64_t *src, const double *in, double *out,
                        cudaStream_t st)
{
    const int64_t m = R * K;
    if (m <= 0) return;
    gather_rows_kernel<<<(int)((m + 255) / 256), 256, 0, st>>>(K, R, src, in, out);
}

template <typename GT>
__global__ void fill_gather_kernel(int K, int64_t R, const double *X, GT *Xg, int ldg)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R * ldg) return;
    const int64_t r = q / ldg;
    const int i = (int)(q % ldg);
    const double x = i < K ? X[r * K + i] : 0.0;
    if constexpr (sizeof(GT) == 2)
        Xg[q] = __double2bfloat16(x);
    else
        Xg[q] = (GT)x;
}

void launch_fill_gather(int K, int prec, int64_t R, const double *X, void *Xg, int ldg,
                        cudaStream_t st)
{
    const int64_t n = R * ldg;
    if (n <= 0) return;
    const int grid = (int)((n + 255) / 256);
    if (prec == BMF_FP64)
        fill_gather_kernel<double><<<grid, 256, 0, st>>>(K, R, X, (double *)Xg, ldg);
    else if (prec == BMF_FP32)
        fill_gather_kernel<float><<<grid, 256, 0, st>>>(K, R, X, (float *)Xg, ldg);
    else
        fill_gather_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(K, R, X, (__nv_bfloat16 *)Xg, ldg);
}

}  // namespace bmf
