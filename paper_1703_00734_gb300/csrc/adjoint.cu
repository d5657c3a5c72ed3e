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
// K/4 lanes (rounded up to 8 or 16) per observation, four features per lane, so that a partner
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

// Pass 1 for K > 16 (KT = 32 or 64): G = KT / 4 lanes per observation, 32 / G observations per
// warp step and two steps in flight.  Lane li of a group owns features 4 li .. 4 li + 3; a lane
// whose first feature is past K loads nothing (rows are 16-byte aligned with a pitch that is a
// multiple of 4 floats and at least K, so every piece a lane does load lies inside its row).
template <int KT>
__global__ void __launch_bounds__(256) adjoint_items_grouped_kernel(AdjointParams a)
{
    constexpr int G = KT / 4, NG = 32 / G, LD = (KT + 1 + 31) / 32 * 32;
    static_assert(G * NG == 32, "group width must divide the warp");
    const int lane = threadIdx.x & 31, g = lane / G, li = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int K = a.K, f0 = 4 * li;
    const bool mine = f0 < K;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t it = warp; it < a.n_items; it += nw) {
        const GramItem m = a.items[it];
        float4 x = zero;
        if (mine) {
            x = __ldg(reinterpret_cast<const float4 *>(a.self + (int64_t)(m.row - a.self0) * a.ld + f0));
            if (f0 + 1 >= K) x.y = 0.f;
            if (f0 + 2 >= K) x.z = 0.f;
            if (f0 + 3 >= K) x.w = 0.f;
        }
        float4 acc = zero;
        float r2 = 0.f;
        for (int e0 = 0; e0 < m.count; e0 += 2 * NG) {
            const int ea = e0 + g, eb = e0 + NG + g;
            const bool va = ea < m.count, vb = eb < m.count;
            float ya = 0.f, yb = 0.f;
            float4 pa = zero, pb = zero;
            if (va) {
                const int64_t q = m.begin + ea;
                ya = __ldg(a.val + q);
                if (mine)
                    pa = __ldg(reinterpret_cast<const float4 *>(
                        a.other + (int64_t)(__ldg(a.idx + q) - a.other0) * a.ld + f0));
            }
            if (vb) {
                const int64_t q = m.begin + eb;
                yb = __ldg(a.val + q);
                if (mine)
                    pb = __ldg(reinterpret_cast<const float4 *>(
                        a.other + (int64_t)(__ldg(a.idx + q) - a.other0) * a.ld + f0));
            }
            float da = x.x * pa.x, db = x.x * pb.x;
            da = fmaf(x.y, pa.y, da);
            db = fmaf(x.y, pb.y, db);
            da = fmaf(x.z, pa.z, da);
            db = fmaf(x.z, pb.z, db);
            da = fmaf(x.w, pa.w, da);
            db = fmaf(x.w, pb.w, db);
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) {
                da += __shfl_xor_sync(0xffffffffu, da, o);
                db += __shfl_xor_sync(0xffffffffu, db, o);
            }
            // past the end of the item y = 0 and p = 0, so r = 0 adds nothing
            const float ra = ya - da, rb = yb - db;
            acc.x = fmaf(ra, pa.x, acc.x);
            acc.y = fmaf(ra, pa.y, acc.y);
            acc.z = fmaf(ra, pa.z, acc.z);
            acc.w = fmaf(ra, pa.w, acc.w);
            acc.x = fmaf(rb, pb.x, acc.x);
            acc.y = fmaf(rb, pb.y, acc.y);
            acc.z = fmaf(rb, pb.z, acc.z);
            acc.w = fmaf(rb, pb.w, acc.w);
            r2 = fmaf(ra, ra, r2);
            r2 = fmaf(rb, rb, r2);
        }
        // sum over the groups (every lane of a group holds the group's r^2)
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
            r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        }
        if (g == 0) {
            float *dst = a.part + it * (int64_t)LD;
            *reinterpret_cast<float4 *>(dst + f0) = acc;
            if (li == 0) dst[KT] = r2;
        }
    }
}

// Pass 2: one warp per local row of the self factor (kAdjRows rows per block, lanes over the
// features).  The prior precision and Lambda mu of the hyperparameter slot of the block's first
// row are staged as FP32 in shared memory (all rows of one side of a subset share it); a row
// with another slot reads and converts its prior from global memory.
constexpr int kAdjRows = 128;
constexpr int kAdjWarps = 4;

__global__ void __launch_bounds__(32 * kAdjWarps) adjoint_rows_kernel(AdjointParams a)
{
    extern __shared__ float adj_sm[];
    const int K = a.K, KT = a.kt, LD = a.ldp, KP = K | 1;   // odd pitch: no bank conflicts
    float *Lf = adj_sm, *bf = Lf + K * KP, *xs = bf + K;     // Lf [K][KP], bf [K], xs [warps][KT]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n0 = (int64_t)blockIdx.x * kAdjRows;
    const int64_t n1 = min(n0 + (int64_t)kAdjRows, a.n_rows);
    const int hb = a.row_hslot[a.self0 + n0];
    if (hb >= 0) {
        const double *hp = a.hyper + (int64_t)hb * hyper_slot_len(K);
        for (int q = threadIdx.x; q < K * K; q += blockDim.x) {
            const int i = q / K, k = q % K;
            Lf[i * KP + k] = (float)hp[K + (i >= k ? tri(i, k) : tri(k, i))];
        }
        for (int q = threadIdx.x; q < K; q += blockDim.x) bf[q] = (float)hp[K + ntri(K) + q];
    }
    __syncthreads();
    float *xw = xs + warp * KT;
    double r2 = 0.0, quad = 0.0;
    for (int64_t n = n0 + warp; n < n1; n += kAdjWarps) {
        const int64_t row = a.self0 + n;
        const int64_t i0 = a.item_ptr[row], i1 = a.item_ptr[row + 1];
        const float *x = a.self + n * a.ld;
        float *g = a.grad + n * a.ld;
        for (int k = lane; k < K; k += 32) xw[k] = x[k];
        __syncwarp();
        const int h = a.row_hslot[row];
        const double *hp = h >= 0 ? a.hyper + (int64_t)h * hyper_slot_len(K) : nullptr;
        float qlane = 0.f;
        for (int i = lane; i < K; i += 32) {
            float s = 0.f;
            for (int64_t it = i0; it < i1; ++it) s += a.part[(it - a.item_base) * (int64_t)LD + i];
            // prior term L (x - mu) = L x - b, in FP32 like the data term
            float lx = 0.f, b;
            if (h == hb && h >= 0) {
                for (int k = 0; k < K; ++k) lx = fmaf(Lf[i * KP + k], xw[k], lx);
                b = bf[i];
            } else {
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
        const size_t smem = ((size_t)a.K * (a.K | 1) + a.K + (size_t)kAdjWarps * a.kt) * sizeof(float);
        adjoint_rows_kernel<<<(int)((a.n_rows + kAdjRows - 1) / kAdjRows), 32 * kAdjWarps, smem, st>>>(a);
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
