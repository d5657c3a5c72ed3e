// cond.cu -- the conditional draw of every row given its partners (BPMF Gibbs step for x_n | W,
// and symmetrically w_d | X; Eqs. 2-4, the (N+D)K^3 term of the cost model of Section 4.3):
//   Lambda_n = Lambda_p + tau G_n,   b_n = Lambda_p mu_p + tau r_n,
//   Lambda_n = L L^T (FP64 Cholesky),  x_n = L^{-T} (L^{-1} b_n + z_n),
// followed by the write of the FP64 state and of its gathered copy, and the moment sums of the
// moment-matching approximation (Section 4.1).
//
// FP64 throughout (the Gram partials are summed in FP64).  One thread per row: the FP64 pipe is
// the bottleneck on this GPU (about two FP64 FMA per clock per SM), and a thread-per-row
// factorisation keeps all 32 lanes busy with independent FP64 work.  The packed matrix of each
// thread lives in shared memory, interleaved across the block so that consecutive threads touch
// consecutive words; loops run over the runtime K (address arithmetic and shared-memory loads
// issue in the shadow of the FP64 pipe).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

template <typename GT>
__device__ __forceinline__ GT to_gather(double x);
template <>
__device__ __forceinline__ double to_gather<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_gather<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_gather<__nv_bfloat16>(double x)
{
    return __double2bfloat16(x);
}


// Interleave stride of the per-thread shared-memory slots: one past the block size, so that the
// statistics epilogue (thread e reading entry i of every row) touches a different bank for each
// entry instead of the same bank for all.
constexpr int kCondStride = kCondBlock + 1;

// Shared-memory slots per thread: the packed matrix (ntri(K)), the right-hand side / solution
// (K) and the reciprocal pivots (K).
static inline int cond_slots(int K) { return ntri(K) + 2 * K; }

template <typename GT, typename AT>
__global__ void __launch_bounds__(kCondBlock) cond_kernel(CondParams a)
{
    extern __shared__ double sm[];
    const int t = threadIdx.x;
    const CondBlock blk = a.blocks[blockIdx.x];
    const int64_t r = blk.row0 + t;
    const bool active = t < blk.n;
    const int K = a.K;
    const int NT = ntri(K);
    const int64_t R = a.R;
    double *M = sm + t;                       // M[e * kCondStride] is entry e of this thread
#define SM(e) M[(e) * kCondStride]
    const int B0 = NT, RI = NT + K;           // rhs/solution at B0 + i, reciprocal pivot at RI + i
    bool ok = active;
    if (active) {
        // 1. G_n and r_n: the row's single Gram partial, or the FP64 sum of its partials made by
        //    the Gram pass for rows split over several items.  The partial entries use the packed
        //    index of the padded width; tri(i, j) does not depend on it.
        const int prhs = a.part_rhs;
        const int64_t i0 = a.item_ptr[r], i1 = a.item_ptr[r + 1];
        const int mi = a.multi_idx[r];
        if (mi >= 0) {
            const double *p = a.rowsum + (int64_t)mi * a.ld_sum;
            for (int e = 0; e < NT; ++e) SM(e) = p[e];
            for (int i = 0; i < K; ++i) SM(B0 + i) = p[prhs + i];
        } else if (i1 > i0) {
            const AT *p = static_cast<const AT *>(a.part) + (i0 - a.item0) * (int64_t)a.ld;
            for (int e = 0; e < NT; ++e) SM(e) = widen(p[e]);
            for (int i = 0; i < K; ++i) SM(B0 + i) = widen(p[prhs + i]);
        } else {
            for (int e = 0; e < NT + K; ++e) SM(e) = 0.0;
        }
        // 2. assemble with the prior: a shared hyperparameter slot or a per-row propagated prior
        const int h = a.row_hslot[r];
        const double tau = a.tau_row ? a.tau_row[r] : a.tau;
        if (h >= 0) {
            const double *hp = a.hyper + (int64_t)h * hyper_slot_len(K);
            for (int e = 0; e < NT; ++e) SM(e) = fma(tau, SM(e), hp[K + e]);
            for (int i = 0; i < K; ++i) SM(B0 + i) = fma(tau, SM(B0 + i), hp[K + NT + i]);
        } else {
            for (int e = 0; e < NT; ++e) SM(e) = fma(tau, SM(e), a.prior_L[(int64_t)e * R + r]);
            for (int i = 0; i < K; ++i)
                SM(B0 + i) = fma(tau, SM(B0 + i), a.prior_b[(int64_t)i * R + r]);
        }
        // 3. Cholesky (Crout order: column j from the columns before it)
        for (int j = 0; j < K && ok; ++j) {
            const int jj = tri(j, 0);
            double d = SM(jj + j);
            for (int k = 0; k < j; ++k) {
                const double l = SM(jj + k);
                d = fma(-l, l, d);
            }
            if (!pivot_ok(d)) {
                atomicOr(&a.err->flags, ERR_NOT_PD);
                atomicMin(&a.err->first_bad_row, (int)r);
                ok = false;
                break;
            }
            // only 1 / L_jj is used from here on (the solves scale by it)
            const double rs = pivot_rsqrt<GT>(d);
            SM(RI + j) = rs;
            for (int i = j + 1; i < K; ++i) {
                const int ii = tri(i, 0);
                double s = SM(ii + j);
                for (int k = 0; k < j; ++k) s = fma(-SM(ii + k), SM(jj + k), s);
                SM(ii + j) = s * rs;
            }
        }
    }
    if (ok) {
        // 4. forward solve L y = b
        for (int i = 0; i < K; ++i) {
            const int ii = tri(i, 0);
            double s = SM(B0 + i);
            for (int k = 0; k < i; ++k) s = fma(-SM(ii + k), SM(B0 + k), s);
            SM(B0 + i) = s * SM(RI + i);
        }
        // 5. back solve L^T x = y + z
        const double *z = a.z + (r - a.row0) * K;
        for (int i = K - 1; i >= 0; --i) {
            double s = SM(B0 + i) + z[i];
            for (int k = i + 1; k < K; ++k) s = fma(-SM(tri(k, i)), SM(B0 + k), s);
            SM(B0 + i) = s * SM(RI + i);
        }
        // 6. state, gathered copy, moment sums
        double *xr = a.X + r * K;
        GT *g = static_cast<GT *>(a.Xg) + r * a.ldg;
        for (int i = 0; i < K; ++i) {
            const double xi = SM(B0 + i);
            xr[i] = xi;
            g[i] = to_gather<GT>(xi);
        }
        for (int i = K; i < a.ldg; ++i) g[i] = to_gather<GT>(0.0);
        if (a.keep) {
            for (int i = 0; i < K; ++i) {
                const double xi = SM(B0 + i);
                a.S1[(int64_t)i * R + r] += xi;
                if (a.full)
                    for (int j = 0; j <= i; ++j) a.S2[(int64_t)tri(i, j) * R + r] += xi * SM(B0 + j);
            }
        }
    } else {
        for (int i = 0; i < K; ++i) SM(B0 + i) = 0.0;
    }
    // 7. statistics of the new state for the next hyperparameter draw: per block, sum x and
    //    the packed lower sum x x^T over the block's rows (thread e computes entry e, in row
    //    order); skipped when the caller computes them on another stream (stats == nullptr)
    // (only blocks whose factor draws its hyperparameters need them: a block of rows with
    // propagated per-row priors skips them; every row of a block shares its subset's prior)
    if (a.stats == nullptr || a.row_hslot[blk.row0] < 0) return;
    __syncthreads();
    const int NS = K + NT;
    double *out = a.stats + (a.blk0 + blockIdx.x) * (int64_t)NS;
    for (int e = t; e < NS; e += kCondBlock) {
        double s = 0.0;
        if (e < K) {
            for (int q = 0; q < blk.n; ++q) s += sm[(B0 + e) * kCondStride + q];
        } else {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e - K) ++i;
            const int j = e - K - i * (i + 1) / 2;
            for (int q = 0; q < blk.n; ++q)
                s = fma(sm[(B0 + i) * kCondStride + q], sm[(B0 + j) * kCondStride + q], s);
        }
        out[e] = s;
    }
#undef SM
}

// ------------------------------------------------------------------------------------------
// The same conditional with K known at compile time: the packed matrix, right-hand side and
// pivots live in registers (fully unrolled loops with constant indices), so the FP64 chain is
// not interleaved with shared-memory loads.  Instantiated for K = 1, 3, 4, 5, 10, 11, 12, the
// sizes the compiler keeps entirely in registers (for K = 2 and 6-9 it places the matrix in
// local memory, so those take cond_kernel).  Same operations in the same order as cond_kernel;
// shared memory holds only the block's new rows for the statistics epilogue.
// ------------------------------------------------------------------------------------------
template <int K, typename GT, typename AT>
__global__ void __launch_bounds__(kCondBlock) cond_kernel_k(CondParams a)
{
    constexpr int NT = ntri(K);
    __shared__ double XS[K][kCondStride];
    const int t = threadIdx.x;
    const CondBlock blk = a.blocks[blockIdx.x];
    const int64_t r = blk.row0 + t;
    const bool active = t < blk.n;
    const int64_t R = a.R;
    double M[NT], B[K], RI[K];
    bool ok = active;
    if (active) {
        const int prhs = a.part_rhs;
        const int64_t i0 = a.item_ptr[r], i1 = a.item_ptr[r + 1];
        const int mi = a.multi_idx[r];
        if (mi >= 0) {
            const double *p = a.rowsum + (int64_t)mi * a.ld_sum;
#pragma unroll
            for (int e = 0; e < NT; ++e) M[e] = p[e];
#pragma unroll
            for (int i = 0; i < K; ++i) B[i] = p[prhs + i];
        } else if (i1 > i0) {
            const AT *p = static_cast<const AT *>(a.part) + (i0 - a.item0) * (int64_t)a.ld;
#pragma unroll
            for (int e = 0; e < NT; ++e) M[e] = widen(p[e]);
#pragma unroll
            for (int i = 0; i < K; ++i) B[i] = widen(p[prhs + i]);
        } else {
#pragma unroll
            for (int e = 0; e < NT; ++e) M[e] = 0.0;
#pragma unroll
            for (int i = 0; i < K; ++i) B[i] = 0.0;
        }
        const int h = a.row_hslot[r];
        const double tau = a.tau_row ? a.tau_row[r] : a.tau;
        if (h >= 0) {
            const double *hp = a.hyper + (int64_t)h * hyper_slot_len(K);
#pragma unroll
            for (int e = 0; e < NT; ++e) M[e] = fma(tau, M[e], hp[K + e]);
#pragma unroll
            for (int i = 0; i < K; ++i) B[i] = fma(tau, B[i], hp[K + NT + i]);
        } else {
#pragma unroll
            for (int e = 0; e < NT; ++e) M[e] = fma(tau, M[e], a.prior_L[(int64_t)e * R + r]);
#pragma unroll
            for (int i = 0; i < K; ++i) B[i] = fma(tau, B[i], a.prior_b[(int64_t)i * R + r]);
        }
        // Cholesky (Crout order), as in cond_kernel
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double d = M[tri(j, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) d = fma(-M[tri(j, k)], M[tri(j, k)], d);
            if (!pivot_ok(d)) ok = false;
            const double rs = pivot_rsqrt<GT>(d);
            RI[j] = rs;
            M[tri(j, j)] = d * rs;
#pragma unroll
            for (int i = j + 1; i < K; ++i) {
                double s2 = M[tri(i, j)];
#pragma unroll
                for (int k = 0; k < j; ++k) s2 = fma(-M[tri(i, k)], M[tri(j, k)], s2);
                M[tri(i, j)] = s2 * rs;
            }
        }
        if (!ok) {
            atomicOr(&a.err->flags, ERR_NOT_PD);
            atomicMin(&a.err->first_bad_row, (int)r);
        }
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            double s2 = B[i];
#pragma unroll
            for (int k = 0; k < i; ++k) s2 = fma(-M[tri(i, k)], B[k], s2);
            B[i] = s2 * RI[i];
        }
        const double *z = a.z + (r - a.row0) * K;
#pragma unroll
        for (int i = K - 1; i >= 0; --i) {
            double s2 = B[i] + z[i];
#pragma unroll
            for (int k = i + 1; k < K; ++k) s2 = fma(-M[tri(k, i)], B[k], s2);
            B[i] = s2 * RI[i];
        }
        double *xr = a.X + r * K;
        GT *g = static_cast<GT *>(a.Xg) + r * a.ldg;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            xr[i] = B[i];
            g[i] = to_gather<GT>(B[i]);
        }
        for (int i = K; i < a.ldg; ++i) g[i] = to_gather<GT>(0.0);
        if (a.keep) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                a.S1[(int64_t)i * R + r] += B[i];
                if (a.full)
#pragma unroll
                    for (int j = 0; j <= i; ++j) a.S2[(int64_t)tri(i, j) * R + r] += B[i] * B[j];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) B[i] = 0.0;
    }
    if (a.stats == nullptr || a.row_hslot[blk.row0] < 0) return;   // as in cond_kernel
#pragma unroll
    for (int i = 0; i < K; ++i) XS[i][t] = B[i];
    __syncthreads();
    constexpr int NS = K + NT;
    double *out = a.stats + (a.blk0 + blockIdx.x) * (int64_t)NS;
    for (int e = t; e < NS; e += kCondBlock) {
        double s2 = 0.0;
        if (e < K) {
            for (int q = 0; q < blk.n; ++q) s2 += XS[e][q];
        } else {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e - K) ++i;
            const int j = e - K - i * (i + 1) / 2;
            for (int q = 0; q < blk.n; ++q) s2 = fma(XS[i][q], XS[j][q], s2);
        }
        out[e] = s2;
    }
}

template <typename GT, typename AT>
static bool launch_cond_fixed(const CondParams &a, int n_blocks, cudaStream_t st)
{
    switch (a.K) {
    case 1: cond_kernel_k<1, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 3: cond_kernel_k<3, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 4: cond_kernel_k<4, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 5: cond_kernel_k<5, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 10: cond_kernel_k<10, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 11: cond_kernel_k<11, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    case 12: cond_kernel_k<12, GT, AT><<<n_blocks, kCondBlock, 0, st>>>(a); return true;
    default: return false;
    }
}

template <typename GT, typename AT>
static void launch_cond_t(const CondParams &a, int n_blocks, cudaStream_t st)
{
    if (launch_cond_fixed<GT, AT>(a, n_blocks, st)) return;
    const size_t smem = (size_t)cond_slots(a.K) * kCondStride * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(cond_kernel<GT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    cond_kernel<GT, AT><<<n_blocks, kCondBlock, smem, st>>>(a);
}

void launch_cond(int prec, const CondParams &a, int n_blocks, cudaStream_t st)
{
    if (n_blocks <= 0) return;
    if (prec == BMF_FP64)
        launch_cond_t<double, double>(a, n_blocks, st);
    else if (prec == BMF_FP32)
        launch_cond_t<float, float>(a, n_blocks, st);
    else
        launch_cond_t<__nv_bfloat16, float>(a, n_blocks, st);
}

}  // namespace bmf
