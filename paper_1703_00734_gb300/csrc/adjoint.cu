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
// item (at most 1024 observations of one row).  K <= 16: lanes over observations, each lane
// gathers its partner row twice (dot product, then accumulation) and a butterfly
// reduce-scatter writes the item's K gradient entries and its sum of r^2.  K > 16: groups of
// 4 (K <= 32) or 8 (K <= 64) lanes per observation, eight features per lane, so that a partner
// row is read once, as consecutive 16-byte pieces; the dot product is reduced within the group
// and the gradient partial across the groups at the end of the item.  Pass 2: one warp per row
// (lanes over features) sums the row's item partials in item order and adds the prior term,
// with the block's shared prior precision staged once in shared memory as FP32; per-block
// FP64 sums of r^2 and of the prior quadratic forms.  Deterministic.
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

// Pass 1 for K > 16 (KT = 32 or 64): F = 8 features per lane, G = KT / F lanes per
// observation, 32 / G observations per warp step and two steps in flight.  Lane li of a group
// owns features 8 li .. 8 li + 7 as two 16-byte pieces; a piece whose first feature is past K
// is not loaded (rows are 16-byte aligned with a pitch that is a multiple of 4 floats and at
// least K, so every piece that is loaded lies inside its row).
template <int KT>
__global__ void __launch_bounds__(256) adjoint_items_grouped_kernel(AdjointParams a)
{
    constexpr int F = 8, PC = F / 4, G = KT / F, NG = 32 / G, LD = (KT + 1 + 31) / 32 * 32;
    static_assert(G * NG == 32 && G * F == KT, "group shape");
    const int lane = threadIdx.x & 31, g = lane / G, li = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int K = a.K, f0 = F * li;
    for (int64_t it = warp; it < a.n_items; it += nw) {
        const GramItem m = a.items[it];
        float x[F];
        const float *xs = a.self + (int64_t)(m.row - a.self0) * a.ld + f0;
#pragma unroll
        for (int j = 0; j < PC; ++j) {
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (f0 + 4 * j < K) q = __ldg(reinterpret_cast<const float4 *>(xs + 4 * j));
            x[4 * j] = q.x;
            x[4 * j + 1] = q.y;
            x[4 * j + 2] = q.z;
            x[4 * j + 3] = q.w;
        }
#pragma unroll
        for (int f = 0; f < F; ++f)
            if (f0 + f >= K) x[f] = 0.f;   // padding of the caller's rows is not read as data
        float acc[F];
#pragma unroll
        for (int f = 0; f < F; ++f) acc[f] = 0.f;
        float r2 = 0.f;
        for (int e0 = 0; e0 < m.count; e0 += 2 * NG) {
            const int ea = e0 + g, eb = e0 + NG + g;
            const bool va = ea < m.count, vb = eb < m.count;
            float ya = 0.f, yb = 0.f, pa[F], pb[F];
            const float *ra_row = nullptr, *rb_row = nullptr;
            if (va) {
                const int64_t q = m.begin + ea;
                ya = __ldg(a.val + q);
                ra_row = a.other + (int64_t)(__ldg(a.idx + q) - a.other0) * a.ld + f0;
            }
            if (vb) {
                const int64_t q = m.begin + eb;
                yb = __ldg(a.val + q);
                rb_row = a.other + (int64_t)(__ldg(a.idx + q) - a.other0) * a.ld + f0;
            }
#pragma unroll
            for (int j = 0; j < PC; ++j) {
                float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
                if (va && f0 + 4 * j < K) u = __ldg(reinterpret_cast<const float4 *>(ra_row + 4 * j));
                if (vb && f0 + 4 * j < K) v = __ldg(reinterpret_cast<const float4 *>(rb_row + 4 * j));
                pa[4 * j] = u.x;
                pa[4 * j + 1] = u.y;
                pa[4 * j + 2] = u.z;
                pa[4 * j + 3] = u.w;
                pb[4 * j] = v.x;
                pb[4 * j + 1] = v.y;
                pb[4 * j + 2] = v.z;
                pb[4 * j + 3] = v.w;
            }
            float da = 0.f, db = 0.f;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                da = fmaf(x[f], pa[f], da);
                db = fmaf(x[f], pb[f], db);
            }
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) {
                da += __shfl_xor_sync(0xffffffffu, da, o);
                db += __shfl_xor_sync(0xffffffffu, db, o);
            }
            // past the end of the item y = 0 and p = 0, so r = 0 adds nothing
            const float ra = ya - da, rb = yb - db;
#pragma unroll
            for (int f = 0; f < F; ++f) acc[f] = fmaf(rb, pb[f], fmaf(ra, pa[f], acc[f]));
            r2 = fmaf(rb, rb, fmaf(ra, ra, r2));
        }
        // sum over the groups (every lane of a group holds the group's r^2)
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
#pragma unroll
            for (int f = 0; f < F; ++f) acc[f] += __shfl_xor_sync(0xffffffffu, acc[f], o);
            r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        }
        if (g == 0) {
            float *dst = a.part + it * (int64_t)LD + f0;
#pragma unroll
            for (int j = 0; j < PC; ++j)
                *reinterpret_cast<float4 *>(dst + 4 * j) =
                    make_float4(acc[4 * j], acc[4 * j + 1], acc[4 * j + 2], acc[4 * j + 3]);
            if (li == 0) a.part[it * (int64_t)LD + KT] = r2;
        }
    }
}

// Pass 2: one warp per local row of the self factor (kAdjRows rows per block, lanes over the
// features).  The prior precision and Lambda mu of the hyperparameter slot of the block's first
// row are staged as FP32 in shared memory, zero-padded to KT columns (all rows of one side of a
// subset share the slot); a row with another slot, or with its own propagated prior, reads and
// converts its prior from global memory.
constexpr int kAdjRows = 128;
constexpr int kAdjWarps = 8;

template <int KT>
__global__ void __launch_bounds__(32 * kAdjWarps) adjoint_rows_kernel(AdjointParams a)
{
    constexpr int KP = KT + 1;    // odd pitch: lanes reading one column hit distinct banks
    __shared__ float Lf[KT * KP], bf[KT], xs[kAdjWarps][KT];
    const int K = a.K, LD = a.ldp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n0 = (int64_t)blockIdx.x * kAdjRows;
    const int64_t n1 = min(n0 + (int64_t)kAdjRows, a.n_rows);
    const int hb = a.row_hslot[a.self0 + n0];
    if (hb >= 0) {
        const double *hp = a.hyper + (int64_t)hb * hyper_slot_len(K);
        for (int q = threadIdx.x; q < KT * KT; q += blockDim.x) {
            const int i = q / KT, k = q % KT;
            Lf[i * KP + k] = (i < K && k < K) ? (float)hp[K + (i >= k ? tri(i, k) : tri(k, i))] : 0.f;
        }
        for (int q = threadIdx.x; q < KT; q += blockDim.x) bf[q] = q < K ? (float)hp[K + ntri(K) + q] : 0.f;
    }
    __syncthreads();
    float *xw = xs[warp];
    double r2 = 0.0, quad = 0.0;
    for (int64_t n = n0 + warp; n < n1; n += kAdjWarps) {
        const int64_t row = a.self0 + n;
        const int64_t i0 = a.item_ptr[row], i1 = a.item_ptr[row + 1];
        const float *x = a.self + n * a.ld;
        float *g = a.grad + n * a.ld;
        for (int k = lane; k < KT; k += 32) xw[k] = k < K ? x[k] : 0.f;
        __syncwarp();
        const int h = a.row_hslot[row];
        float qlane = 0.f;
        for (int i = lane; i < K; i += 32) {
            float s = 0.f;
            for (int64_t it = i0; it < i1; ++it) s += a.part[(it - a.item_base) * (int64_t)LD + i];
            // prior term L (x - mu) = L x - b, in FP32 like the data term
            float lx, b;
            if (h == hb && h >= 0) {
                float l0 = 0.f, l1 = 0.f;
#pragma unroll
                for (int k = 0; k < KT; k += 2) {
                    l0 = fmaf(Lf[i * KP + k], xw[k], l0);
                    l1 = fmaf(Lf[i * KP + k + 1], xw[k + 1], l1);
                }
                lx = l0 + l1;
                b = bf[i];
            } else {
                const double *hp = h >= 0 ? a.hyper + (int64_t)h * hyper_slot_len(K) : nullptr;
                lx = 0.f;
                for (int k = 0; k < K; ++k) {
                    const int e = i >= k ? tri(i, k) : tri(k, i);
                    const float l = (float)(hp ? hp[K + e] : a.prior_L[(int64_t)e * a.R + row]);
                    lx = fmaf(l, xw[k], lx);
                }
                b = (float)(hp ? hp[K + ntri(K) + i] : a.prior_b[(int64_t)i * a.R + row]);
            }
            g[i] = (float)a.alpha * s - (lx - b);
            // (x - mu)^T L (x - mu) = x^T L x - 2 x^T b + mu^T b: the last term is constant
            qlane = fmaf(xw[i], lx - 2.f * b, qlane);
        }
        for (int i = K + lane; i < a.ld; i += 32) g[i] = 0.f;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) qlane += __shfl_xor_sync(0xffffffffu, qlane, o);
        if (lane == 0) {
            quad += (double)qlane;
            if (a.count_r2)
                for (int64_t it = i0; it < i1; ++it) r2 += (double)a.part[(it - a.item_base) * (int64_t)LD + KT];
        }
        __syncwarp();   // xw is rewritten for the next row
    }
    __shared__ double red[2][kAdjWarps];
    if (lane == 0) {
        red[0][warp] = r2;
        red[1][warp] = quad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < kAdjWarps; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        a.block_sums[2 * blockIdx.x] = s0;
        a.block_sums[2 * blockIdx.x + 1] = s1;
    }
}

template <int KT>
static void launch_items_t(const AdjointParams &a, int grid, cudaStream_t st)
{
    if constexpr (KT >= 32)
        adjoint_items_grouped_kernel<KT><<<grid, 256, 0, st>>>(a);
    else
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
    if (a.n_rows > 0) {
        const int blocks = (int)((a.n_rows + kAdjRows - 1) / kAdjRows);
        switch (a.kt) {
        case 4: adjoint_rows_kernel<4><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        case 8: adjoint_rows_kernel<8><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        case 12: adjoint_rows_kernel<12><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        case 16: adjoint_rows_kernel<16><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        case 32: adjoint_rows_kernel<32><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        default: adjoint_rows_kernel<64><<<blocks, 32 * kAdjWarps, 0, st>>>(a); break;
        }
    }
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
