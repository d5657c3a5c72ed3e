// adjoint.cu -- the adjoint of the masked log-joint of one data subset (an addition of this
// project; the paper samples with Gibbs only):
//   l(X, W, log a) = -(a/2) sum_{(n,d) in Omega} r_nd^2 + (|Omega|/2) log a
//                    - 1/2 sum_n (x_n - mu_n)^T L_n (x_n - mu_n) - 1/2 sum_d (w_d - mu_d)^T L_d (w_d - mu_d),
//   r_nd = y_nd - x_n^T w_d,
//   grad_x_n = a sum_{d in Omega_n} r_nd w_d - L_n (x_n - mu_n)   (and symmetrically for w_d),
//   dl/dlog a = |Omega|/2 - (a/2) sum r^2,
// where (mu_n, L_n) is the row's prior in the subset (the subset's hyperparameters, or the row's
// propagated Gaussian); terms constant in X, W and a are dropped from the value.
//
// FP32 arithmetic on FP32 factors, FP64 scalar sums.  Pass 1 (per side): one warp per work
// item (at most 1024 observations of one row), lanes over observations; each lane gathers the
// partner row twice in 16-float chunks (dot product, then accumulation) so K = 64 fits in
// registers; a butterfly reduce-scatter writes the item's K gradient entries and its sum of r^2.
// Pass 2: one thread per row sums the row's item partials in item order and adds the prior
// term; per-block FP64 sums of r^2 and of the prior quadratic forms.  Deterministic.
#include "common.cuh"
#include "kernels.h"

namespace bmf {

int adjoint_kt(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : K <= 16 ? 16 : K <= 32 ? 32 : 64; }
int adjoint_ld(int K) { return (adjoint_kt(K) + 1 + 31) / 32 * 32; }

template <int C, int N>
__device__ __forceinline__ void rs_stepf(float (&acc)[N], int lane, int o)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        float lo = acc[i], hi = acc[i + C / 2];
        float send = up ? lo : hi;
        float keep = up ? hi : lo;
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

// Pass 1.  Row `row` of the "self" factor (arena numbering) is local row row - self0 of the
// caller's array; partner index idx (arena numbering of the other factor) is local idx - other0.
template <int KT>
__global__ void __launch_bounds__(256) adjoint_items_kernel(AdjointParams a)
{
    constexpr int LD = (KT + 1 + 31) / 32 * 32;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int K = a.K;
    for (int64_t it = warp; it < a.n_items; it += nw) {
        const GramItem m = a.items[it];
        float x[KT];
        const float4 *xs = reinterpret_cast<const float4 *>(a.self + (int64_t)(m.row - a.self0) * a.ld);
#pragma unroll
        for (int v = 0; v < KT / 4; ++v) {
            const float4 q = __ldg(xs + v);
            x[4 * v] = 4 * v < K ? q.x : 0.f;
            x[4 * v + 1] = 4 * v + 1 < K ? q.y : 0.f;
            x[4 * v + 2] = 4 * v + 2 < K ? q.z : 0.f;
            x[4 * v + 3] = 4 * v + 3 < K ? q.w : 0.f;
        }
        float acc[LD];
#pragma unroll
        for (int v = 0; v < LD; ++v) acc[v] = 0.f;
        for (int e = lane; e < m.count; e += 32) {
            const int64_t q = m.begin + e;
            const int c = __ldg(a.idx + q) - a.other0;
            const float y = __ldg(a.val + q);
            const float4 *ps = reinterpret_cast<const float4 *>(a.other + (int64_t)c * a.ld);
            float dot = 0.f;
#pragma unroll
            for (int v = 0; v < KT / 4; ++v) {
                const float4 p = __ldg(ps + v);
                dot = fmaf(x[4 * v], p.x, dot);
                dot = fmaf(x[4 * v + 1], p.y, dot);
                dot = fmaf(x[4 * v + 2], p.z, dot);
                dot = fmaf(x[4 * v + 3], p.w, dot);
            }
            const float r = y - dot;
#pragma unroll
            for (int v = 0; v < KT / 4; ++v) {
                const float4 p = __ldg(ps + v);
                acc[4 * v] = fmaf(r, p.x, acc[4 * v]);
                acc[4 * v + 1] = fmaf(r, p.y, acc[4 * v + 1]);
                acc[4 * v + 2] = fmaf(r, p.z, acc[4 * v + 2]);
                acc[4 * v + 3] = fmaf(r, p.w, acc[4 * v + 3]);
            }
            acc[KT] = fmaf(r, r, acc[KT]);
        }
        rs_stepf<LD, LD>(acc, lane, 16);
        rs_stepf<LD / 2, LD>(acc, lane, 8);
        rs_stepf<LD / 4, LD>(acc, lane, 4);
        rs_stepf<LD / 8, LD>(acc, lane, 2);
        rs_stepf<LD / 16, LD>(acc, lane, 1);
        constexpr int PER = LD / 32;
        float *dst = a.part + it * (int64_t)LD + lane * PER;
#pragma unroll
        for (int v = 0; v < PER; ++v) dst[v] = acc[v];
    }
}

// Pass 2: one thread per local row of the self factor.
constexpr int kAdjRows = 128;

__global__ void __launch_bounds__(kAdjRows) adjoint_rows_kernel(AdjointParams a)
{
    const int t = threadIdx.x;
    const int64_t n = (int64_t)blockIdx.x * kAdjRows + t;
    const int K = a.K, KT = a.kt, LD = a.ldp;
    double r2 = 0.0, quad = 0.0;
    if (n < a.n_rows) {
        const int64_t row = a.self0 + n;
        const int64_t i0 = a.item_ptr[row], i1 = a.item_ptr[row + 1];
        const float *x = a.self + n * a.ld;
        float *g = a.grad + n * a.ld;
        const int h = a.row_hslot[row];
        const double *hp = h >= 0 ? a.hyper + (int64_t)h * hyper_slot_len(K) : nullptr;
        float qrow = 0.f;
        for (int i = 0; i < K; ++i) {
            float s = 0.f;
            for (int64_t it = i0; it < i1; ++it) s += a.part[(it - a.item_base) * (int64_t)LD + i];
            // prior term L (x - mu) = L x - b, in FP32 like the data term
            float lx = 0.f;
            for (int k = 0; k < K; ++k) {
                const int e = i >= k ? tri(i, k) : tri(k, i);
                const float l = (float)(hp ? hp[K + e] : a.prior_L[(int64_t)e * a.R + row]);
                lx = fmaf(l, x[k], lx);
            }
            const float b = (float)(hp ? hp[K + ntri(K) + i] : a.prior_b[(int64_t)i * a.R + row]);
            g[i] = (float)a.alpha * s - (lx - b);
            // (x - mu)^T L (x - mu) = x^T L x - 2 x^T b + mu^T b: the last term is constant
            qrow = fmaf(x[i], lx - 2.f * b, qrow);
        }
        quad = (double)qrow;
        for (int i = K; i < a.ld; ++i) g[i] = 0.f;
        if (a.count_r2)
            for (int64_t it = i0; it < i1; ++it) r2 += (double)a.part[(it - a.item_base) * (int64_t)LD + KT];
    }
    __shared__ double red[2][kAdjRows];
    red[0][t] = r2;
    red[1][t] = quad;
    __syncthreads();
    for (int o = kAdjRows / 2; o > 0; o >>= 1) {
        if (t < o) {
            red[0][t] += red[0][t + o];
            red[1][t] += red[1][t + o];
        }
        __syncthreads();
    }
    if (t == 0) {
        a.block_sums[2 * blockIdx.x] = red[0][0];
        a.block_sums[2 * blockIdx.x + 1] = red[1][0];
    }
}

template <int KT>
static void launch_items_t(const AdjointParams &a, int grid, cudaStream_t st)
{
    adjoint_items_kernel<KT><<<grid, 256, 0, st>>>(a);
}

void launch_adjoint(const AdjointParams &a, int grid, cudaStream_t st)
{
    if (a.n_items > 0) {
        switch (a.kt) {
        case 4: launch_items_t<4>(a, grid, st); break;
        case 8: launch_items_t<8>(a, grid, st); break;
        case 12: launch_items_t<12>(a, grid, st); break;
        case 16: launch_items_t<16>(a, grid, st); break;
        case 32: launch_items_t<32>(a, grid, st); break;
        default: launch_items_t<64>(a, grid, st); break;
        }
    }
    if (a.n_rows > 0)
        adjoint_rows_kernel<<<(int)((a.n_rows + kAdjRows - 1) / kAdjRows), kAdjRows, 0, st>>>(a);
}

int adjoint_row_blocks(int64_t n_rows) { return (int)((n_rows + kAdjRows - 1) / kAdjRows); }

// Langevin move on FP32 factors: theta <- theta + (eps/2) grad + sqrt(eps) xi (padding kept 0).
__global__ void langevin_kernel(float *theta, const float *grad, const float *xi, int64_t n_rows,
                                int K, int ld, float eps)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_rows * K) return;
    const int64_t r = q / K;
    const int k = (int)(q % K);
    const int64_t o = r * ld + k;
    theta[o] = theta[o] + 0.5f * eps * grad[o] + sqrtf(eps) * xi[r * K + k];
}

void launch_langevin(float *theta, const float *grad, const float *xi, int64_t n_rows, int K,
                     int ld, float eps, cudaStream_t st)
{
    const int64_t n = n_rows * K;
    if (n <= 0) return;
    langevin_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(theta, grad, xi, n_rows, K, ld, eps);
}

// FP32 copy of FP64 observation values (for contexts that gather in FP64).
__global__ void to_float_kernel(const double *in, float *out, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = (float)in[q];
}

void launch_to_float(const double *in, float *out, int64_t n, cudaStream_t st)
{
    if (n > 0) to_float_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(in, out, n);
}

// Per-block FP64 sums of sum_k (a - b - coef g)^2 over rows x K (row pitch ld).
__global__ void __launch_bounds__(256) sqdiff_kernel(const float *a, const float *b, const float *g,
                                                     double coef, int64_t n_rows, int K,
                                                     int64_t ld, double *block_sums)
{
    double s = 0.0;
    const int64_t n = n_rows * K;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (q / K) * ld + q % K;
        const double d = (double)a[o] - (double)b[o] - coef * (double)g[o];
        s += d * d;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = red[0];
}

void launch_sqdiff(const float *a, const float *b, const float *g, double coef, int64_t n_rows,
                   int K, int64_t ld, double *block_sums, int blocks, cudaStream_t st)
{
    sqdiff_kernel<<<blocks, 256, 0, st>>>(a, b, g, coef, n_rows, K, ld, block_sums);
}

}  // namespace bmf
