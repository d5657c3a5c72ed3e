// noise.cu -- the sampled noise precision (Section 2.1: one precision tau_d per column, or one
// per chain, with conjugate Gamma(a0, b0) priors, shape and rate):
//   tau_d | X, W ~ Gamma(a0 + n_d / 2, b0 + SSE_d / 2),  SSE_d = sum_{n in Omega_d} (y_nd -
//   x_n^T w_d)^2,  drawn as c / (2 b0 + SSE_d) from a chi-square variate c with 2 a0 + n_d
//   degrees of freedom (one precision: the subset's entries and summed SSE).
// The row-side Gram pass takes the per-column precisions through scaled copies: partner rows
// sqrt(tau_d) w_d and values sqrt(tau_d) y_nd, so that sum (sqrt(tau) w)(sqrt(tau) w)^T =
// sum tau w w^T and sum (sqrt(tau) y)(sqrt(tau) w) = sum tau y w.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

template <typename VT>
__global__ void noise_sse_kernel(int K, int64_t r0, int64_t r1, const int64_t *ptr,
                                 const int32_t *idx, const VT *val, const double *X,
                                 const double *W, double *sse)
{
    const int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const double *w = W + r * K;
    double s = 0.0;
    for (int64_t q = ptr[r]; q < ptr[r + 1]; ++q) {
        const double *x = X + (int64_t)idx[q] * K;
        double pr = 0.0;
        for (int k = 0; k < K; ++k) pr = fma(x[k], w[k], pr);
        const double e = (double)val[q] - pr;
        s = fma(e, e, s);
    }
    sse[r] = s;
}

void launch_noise_sse(int K, int64_t r0, int64_t r1, const int64_t *ptr, const int32_t *idx,
                      const void *val, int prec, const double *X, const double *W, double *sse,
                      cudaStream_t st)
{
    if (r1 <= r0) return;
    const int grid = (int)((r1 - r0 + 127) / 128);
    if (prec == BMF_FP64)
        noise_sse_kernel<double><<<grid, 128, 0, st>>>(K, r0, r1, ptr, idx,
                                                       static_cast<const double *>(val), X, W, sse);
    else
        noise_sse_kernel<float><<<grid, 128, 0, st>>>(K, r0, r1, ptr, idx,
                                                      static_cast<const float *>(val), X, W, sse);
}

// One block per subset: column mode writes each row's precision; global mode sums the block's
// SSE (a fixed tree over a fixed strided split) and writes one precision to every row.
__global__ void __launch_bounds__(256) noise_tau_kernel(int mode, double b0, const NoiseBlock *blocks,
                                                        const double *draws, const double *sse,
                                                        double *tau)
{
    const NoiseBlock b = blocks[blockIdx.x];
    if (mode == 2) {
        for (int64_t r = b.r0 + threadIdx.x; r < b.r1; r += blockDim.x)
            tau[r] = draws[b.draw + (r - b.r0)] / (2.0 * b0 + sse[r]);
        return;
    }
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t r = b.r0 + threadIdx.x; r < b.r1; r += blockDim.x) s += sse[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double t = draws[b.draw] / (2.0 * b0 + red[0]);
    for (int64_t r = b.r0 + threadIdx.x; r < b.r1; r += blockDim.x) tau[r] = t;
}

void launch_noise_tau(int mode, double b0, const NoiseBlock *blocks, int n_blocks,
                      const double *draws, const double *sse, double *tau, cudaStream_t st)
{
    if (n_blocks <= 0) return;
    noise_tau_kernel<<<n_blocks, 256, 0, st>>>(mode, b0, blocks, draws, sse, tau);
}

template <typename GT>
__device__ __forceinline__ GT to_g(double x);
template <>
__device__ __forceinline__ double to_g<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_g<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_g<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

template <typename GT, typename VT>
__global__ void noise_scale_kernel(int K, int64_t r0, int64_t r1, const double *tau, const double *W,
                                   GT *Ws, int ldg, int64_t q0, int64_t q1, const int32_t *idx,
                                   const VT *val_orig, VT *val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nrow = (r1 - r0) * ldg;
    if (i < nrow) {
        const int64_t r = r0 + i / ldg;
        const int k = (int)(i % ldg);
        Ws[r * ldg + k] = to_g<GT>(k < K ? sqrt(tau[r]) * W[r * K + k] : 0.0);
        return;
    }
    const int64_t q = q0 + (i - nrow);
    if (q < q1) val[q] = (VT)((double)val_orig[q] * sqrt(tau[idx[q]]));
}

void launch_noise_scale(int K, int prec, int64_t r0, int64_t r1, const double *tau,
                        const double *W, void *Ws, int ldg, int64_t q0, int64_t q1,
                        const int32_t *idx, const void *val_orig, void *val, cudaStream_t st)
{
    const int64_t n = (r1 - r0) * ldg + (q1 - q0);
    if (n <= 0) return;
    const int grid = (int)((n + 255) / 256);
    if (prec == BMF_FP64)
        noise_scale_kernel<double, double><<<grid, 256, 0, st>>>(
            K, r0, r1, tau, W, (double *)Ws, ldg, q0, q1, idx, (const double *)val_orig, (double *)val);
    else if (prec == BMF_FP32)
        noise_scale_kernel<float, float><<<grid, 256, 0, st>>>(
            K, r0, r1, tau, W, (float *)Ws, ldg, q0, q1, idx, (const float *)val_orig, (float *)val);
    else
        noise_scale_kernel<__nv_bfloat16, float><<<grid, 256, 0, st>>>(
            K, r0, r1, tau, W, (__nv_bfloat16 *)Ws, ldg, q0, q1, idx, (const float *)val_orig,
            (float *)val);
}

}  // namespace bmf
