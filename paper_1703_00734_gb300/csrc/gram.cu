// gram.cu -- the Gram-gather pass of the Gibbs sweep: for every arena row n (or a chunk of a
// long row), G_n = sum_{d in Omega_n} p_d p_d^T and r_n = sum_{d in Omega_n} y_nd p_d, where p_d
// are the gathered latent vectors of the observed partners (the row-side and column-side
// conditionals of BPMF, Eqs. 2-4; the MK^2 term of the cost model of Section 4.3).
//
// One warp per work item; lanes stride over the item's observations and gather one partner row
// each, accumulating the packed-lower Gram entries and the right-hand side in registers; a
// butterfly reduce-scatter then leaves each lane with a contiguous slice of the summed entries,
// written with coalesced stores.  Entries are split into parts of EP values when they do not fit
// in registers (each part is a separate slice of work over the same items).  The reduction order
// is fixed, so results are deterministic.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

int padded_k(int K) { return K <= 1 ? 2 : (K + 1) / 2 * 2; }

int gather_ld(int K, int prec)
{
    int KT = padded_k(K);
    int per16 = prec == BMF_FP64 ? 2 : (prec == BMF_BF16 ? 8 : 4);
    return (KT + per16 - 1) / per16 * per16;
}

// Entries per part: registers hold EP accumulators per lane (FP32: up to 160, FP64: 32).
__host__ __device__ constexpr int ep_of(int KT, bool fp64)
{
    return fp64 ? 32 : (gram_nv(KT) <= 96 ? 96 : 160);
}

static int ep_for(int KT, int prec) { return ep_of(KT, prec == BMF_FP64); }

int gram_parts(int K, int prec)
{
    int KT = padded_k(K), ep = ep_for(KT, prec);
    return (gram_nv(KT) + ep - 1) / ep;
}

int gram_part_ld(int K, int prec) { return gram_parts(K, prec) * ep_for(padded_k(K), prec); }

__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }

// Load KT elements of a gathered row (16-byte vector loads) into AT registers.
template <int KT>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&w)[KT])
{
    constexpr int NV4 = (KT + 3) / 4;
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int v = 0; v < NV4; ++v) {
        float4 a = __ldg(q + v);
        if (4 * v + 0 < KT) w[4 * v + 0] = a.x;
        if (4 * v + 1 < KT) w[4 * v + 1] = a.y;
        if (4 * v + 2 < KT) w[4 * v + 2] = a.z;
        if (4 * v + 3 < KT) w[4 * v + 3] = a.w;
    }
}
template <int KT>
__device__ __forceinline__ void load_row(const double *__restrict__ p, double (&w)[KT])
{
    constexpr int NV2 = (KT + 1) / 2;
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int v = 0; v < NV2; ++v) {
        double2 a = __ldg(q + v);
        if (2 * v + 0 < KT) w[2 * v + 0] = a.x;
        if (2 * v + 1 < KT) w[2 * v + 1] = a.y;
    }
}
template <int KT>
__device__ __forceinline__ void load_row(const __nv_bfloat16 *__restrict__ p, float (&w)[KT])
{
    constexpr int NV8 = (KT + 7) / 8;
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int v = 0; v < NV8; ++v) {
        uint4 a = __ldg(q + v);
        uint32_t u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            __nv_bfloat162 b2 = *reinterpret_cast<__nv_bfloat162 *>(&u[h]);
            float2 f = __bfloat1622float2(b2);
            if (8 * v + 2 * h + 0 < KT) w[8 * v + 2 * h + 0] = f.x;
            if (8 * v + 2 * h + 1 < KT) w[8 * v + 2 * h + 1] = f.y;
        }
    }
}

// One butterfly step of the reduce-scatter over C values: the lane half selected by bit `o`
// keeps the upper half of the values, the other the lower half; each adds its partner's copy.
template <int C, int N, typename AT>
__device__ __forceinline__ void rs_step(AT (&acc)[N], int lane, int o)
{
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        AT lo = acc[i], hi = acc[i + C / 2];
        AT send = up ? lo : hi;
        AT keep = up ? hi : lo;
        acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

// Value of Gram entry `e` (global index within the item's entries) for one observation.
template <int KT, int E, typename AT>
__device__ __forceinline__ void accum_entry(AT &acc, const AT (&w)[KT], AT y)
{
    constexpr int NT = ntri(KT);
    if constexpr (E < NT) {
        // decode packed lower (i, j) at compile time
        constexpr int i = [] {
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= E) ++r;
            return r;
        }();
        constexpr int j = E - i * (i + 1) / 2;
        acc = madd(w[i], w[j], acc);
    } else if constexpr (E < NT + KT) {
        acc = madd(y, w[E - NT], acc);
    }
}

template <int KT, int EP, int BASE, int I, typename AT>
__device__ __forceinline__ void accum_all(AT (&acc)[EP], const AT (&w)[KT], AT y)
{
    if constexpr (I < EP) {
        accum_entry<KT, BASE + I, AT>(acc[I], w, y);
        accum_all<KT, EP, BASE, I + 1, AT>(acc, w, y);
    }
}

template <int KT, typename GT, typename AT, int EP, int PART>
__device__ __forceinline__ void gram_body(const GramParams &a)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const GT *__restrict__ P = static_cast<const GT *>(a.P);
    const AT *__restrict__ val = static_cast<const AT *>(a.val);
    AT *__restrict__ part = static_cast<AT *>(a.part);
    for (int64_t it = warp; it < a.n_items; it += nwarps) {
        const GramItem m = a.items[it];
        AT acc[EP];
#pragma unroll
        for (int v = 0; v < EP; ++v) acc[v] = AT(0);
        for (int e = lane; e < m.count; e += 32) {
            const int64_t q = m.begin + e;
            const int c = __ldg(a.idx + q);
            const AT y = __ldg(val + q);
            AT w[KT];
            load_row<KT>(P + (int64_t)c * a.ldP, w);
            accum_all<KT, EP, PART * EP, 0, AT>(acc, w, y);
        }
        rs_step<EP, EP, AT>(acc, lane, 16);
        rs_step<EP / 2, EP, AT>(acc, lane, 8);
        rs_step<EP / 4, EP, AT>(acc, lane, 4);
        rs_step<EP / 8, EP, AT>(acc, lane, 2);
        rs_step<EP / 16, EP, AT>(acc, lane, 1);
        constexpr int PER = EP / 32;
        AT *dst = part + it * (int64_t)a.ld + PART * EP + lane * PER;
#pragma unroll
        for (int v = 0; v < PER; ++v) dst[v] = acc[v];
    }
}

template <int KT, typename GT, typename AT, int EP, int PART, int NP>
__device__ __forceinline__ void gram_dispatch(int part, const GramParams &a)
{
    if constexpr (PART < NP) {
        if (part == PART)
            gram_body<KT, GT, AT, EP, PART>(a);
        else
            gram_dispatch<KT, GT, AT, EP, PART + 1, NP>(part, a);
    }
}

template <int KT, typename GT, typename AT, int EP>
__global__ void __launch_bounds__(256) gram_kernel(GramParams a)
{
    constexpr int NP = (gram_nv(KT) + EP - 1) / EP;
    gram_dispatch<KT, GT, AT, EP, 0, NP>(blockIdx.y, a);
}

template <int KT, typename GT, typename AT>
static void launch_gram_t(const GramParams &a, int grid, int nparts, int, cudaStream_t st)
{
    constexpr int EP = ep_of(KT, sizeof(AT) == 8);
    dim3 g(grid, nparts);
    gram_kernel<KT, GT, AT, EP><<<g, 256, 0, st>>>(a);
}

template <typename GT, typename AT>
static void launch_gram_k(int KT, const GramParams &a, int grid, int nparts, int ep,
                          cudaStream_t st)
{
    switch (KT) {
    case 2: launch_gram_t<2, GT, AT>(a, grid, nparts, ep, st); break;
    case 4: launch_gram_t<4, GT, AT>(a, grid, nparts, ep, st); break;
    case 6: launch_gram_t<6, GT, AT>(a, grid, nparts, ep, st); break;
    case 8: launch_gram_t<8, GT, AT>(a, grid, nparts, ep, st); break;
    case 10: launch_gram_t<10, GT, AT>(a, grid, nparts, ep, st); break;
    case 12: launch_gram_t<12, GT, AT>(a, grid, nparts, ep, st); break;
    case 14: launch_gram_t<14, GT, AT>(a, grid, nparts, ep, st); break;
    case 16: launch_gram_t<16, GT, AT>(a, grid, nparts, ep, st); break;
    default: break;
    }
}

void launch_gram(int K, int prec, const GramParams &a, int grid, cudaStream_t st)
{
    if (a.n_items == 0) return;
    int KT = padded_k(K), ep = ep_for(KT, prec), np = gram_parts(K, prec);
    if (prec == BMF_FP64)
        launch_gram_k<double, double>(KT, a, grid, np, ep, st);
    else if (prec == BMF_FP32)
        launch_gram_k<float, float>(KT, a, grid, np, ep, st);
    else
        launch_gram_k<__nv_bfloat16, float>(KT, a, grid, np, ep, st);
}

}  // namespace bmf
