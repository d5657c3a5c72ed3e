// gram.cu -- the Gram-gather pass of the Gibbs sweep: for every arena row n (or a chunk of a
// long row), G_n = sum_{d in Omega_n} p_d p_d^T and r_n = sum_{d in Omega_n} y_nd p_d, where p_d
// are the gathered latent vectors of the observed partners (the row-side and column-side
// conditionals of BPMF, Eqs. 2-4; the MK^2 term of the cost model of Section 4.3).
//
// A warp task is one long work item (32 lanes) or several short rows (groups of 16 or 8 lanes,
// one row per group).  Lanes of a group stride over the row's observations and gather one
// partner row each with vector loads (the number of scattered load requests, not bytes, bounds
// a gather on this GPU), accumulating the packed-lower Gram entries and the right-hand side in
// registers; a butterfly reduce-scatter within the group then leaves each lane with a contiguous
// slice of the summed entries, written with coalesced stores.  Entries are split into parts of
// EP values when they do not fit in registers.  Rows longer than one item are finished by the
// warp that completes their last item.  Every sum has a fixed order: results are deterministic.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

int padded_k(int K) { return K <= 1 ? 2 : (K + 1) / 2 * 2; }

// Gathered rows start on 16-byte boundaries (128-bit loads).
int gather_ld(int K, int prec)
{
    if (K > 16) return wide_kt(K);   // rows of 32, 48 or 64 elements (16-byte multiples)
    const int KT = padded_k(K);
    const int per16 = prec == BMF_FP64 ? 2 : (prec == BMF_BF16 ? 8 : 4);
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

// Lanes per row by its observation count: fewer lanes per row means more rows per warp and a
// shorter reduce-scatter per row; measured on this GPU (69,878 x 10,677 Zipf workload, K = 10)
// the X-side pass took 118 us with these thresholds against 140 us with (16, 48).
int gram_group(int64_t count) { return count <= 64 ? 8 : (count <= 256 ? 16 : 32); }

__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return fma(a, b, c); }

// ------------------------------------------------------------------------------------------
// Row gathers: the first BYTES bytes of a 16-byte aligned row with 128-bit loads (a tail of at
// most 8 bytes with one 64-bit load).  Measured on this GPU: 256-bit loads at a 32-byte row
// pitch were slower here than 128-bit loads at the tighter 16-byte pitch (fewer L1 hits on the
// frequently gathered rows).
// ------------------------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void load_bits(const void *__restrict__ p, uint32_t (&u)[(BYTES + 3) / 4])
{
    constexpr int NW = (BYTES + 3) / 4;
    const uint4 *q = static_cast<const uint4 *>(p);
    constexpr int FULL = BYTES / 16, REM = BYTES - 16 * FULL;
    constexpr int N16 = FULL + (REM > 8 ? 1 : 0);
#pragma unroll
    for (int c = 0; c < N16; ++c) {
        const uint4 v = __ldg(q + c);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * c + k < NW) u[4 * c + k] = w[k];
    }
    if constexpr (REM > 0 && REM <= 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(q + FULL));
        u[4 * FULL] = v.x;
        if (4 * FULL + 1 < NW) u[4 * FULL + 1] = v.y;
    }
}

template <int KT>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&w)[KT])
{
    uint32_t u[KT];
    load_bits<4 * KT>(p, u);
#pragma unroll
    for (int k = 0; k < KT; ++k) w[k] = __uint_as_float(u[k]);
}
template <int KT>
__device__ __forceinline__ void load_row(const double *__restrict__ p, double (&w)[KT])
{
    uint32_t u[2 * KT];
    load_bits<8 * KT>(p, u);
#pragma unroll
    for (int k = 0; k < KT; ++k) w[k] = __hiloint2double((int)u[2 * k + 1], (int)u[2 * k]);
}
template <int KT>
__device__ __forceinline__ void load_row(const __nv_bfloat16 *__restrict__ p, float (&w)[KT])
{
    uint32_t u[KT / 2];
    load_bits<2 * KT>(p, u);
#pragma unroll
    for (int k = 0; k < KT / 2; ++k) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u[k]));
        w[2 * k] = f.x;
        w[2 * k + 1] = f.y;
    }
}

// ------------------------------------------------------------------------------------------
// Accumulation and the in-group reduce-scatter
// ------------------------------------------------------------------------------------------

// One butterfly step over C values: the lane half selected by bit `o` keeps the upper half of
// the values, the other the lower half; each adds its partner's copy.
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

// Steps with offsets O, O/2, ..., 1 (a group of 2*O lanes); afterwards lane li of the group
// holds the entries [li * C0 / (2*O), (li + 1) * C0 / (2*O)) of the group's sum.
template <int C, int O, int N, typename AT>
__device__ __forceinline__ void rs_group(AT (&acc)[N], int lane)
{
    if constexpr (O >= 1) {
        rs_step<C, N, AT>(acc, lane, O);
        rs_group<C / 2, O / 2, N, AT>(acc, lane);
    }
}

// Gram entry E (packed lower (i, j), then right-hand side) for one observation.
template <int KT, int E, typename AT>
__device__ __forceinline__ void accum_entry(AT &acc, const AT (&w)[KT], AT y)
{
    constexpr int NT = ntri(KT);
    if constexpr (E < NT) {
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

// One warp task with groups of G lanes: group g handles item tk.item0 + g (g < tk.n).
template <int KT, typename GT, typename AT, int EP, int PART, int G>
__device__ __forceinline__ void gram_task(const GramParams &a, const GramTask &tk, int lane)
{
    const GT *__restrict__ P = static_cast<const GT *>(a.P);
    const AT *__restrict__ val = static_cast<const AT *>(a.val);
    AT *__restrict__ part = static_cast<AT *>(a.part);
    const int g = lane / G, li = lane % G;
    const bool has = g < tk.n;
    const int64_t item = tk.item0 + (has ? g : 0);
    const GramItem m = a.items[item - a.item0];
    const int cnt = has ? m.count : 0;
    // accumulators of this group width: the entries rounded up to a multiple of G (the
    // reduce-scatter halves the set log2(G) times), not to the part width, when one part holds
    // all of them
    constexpr int NV = gram_nv(KT);
    constexpr int EPG = NV <= EP ? (NV + G - 1) / G * G : EP;
    AT acc[EPG];
#pragma unroll
    for (int v = 0; v < EPG; ++v) acc[v] = AT(0);
    // two observations per lane per iteration (lane order li, li+G, li+2G, ... is kept), so
    // that two gathers are in flight before either is consumed
    int e = li;
    for (; e + G < cnt; e += 2 * G) {
        const int64_t q0 = m.begin + e, q1 = q0 + G;
        const int c0 = __ldg(a.idx + q0), c1 = __ldg(a.idx + q1);
        const AT y0 = __ldg(val + q0), y1 = __ldg(val + q1);
        AT w0[KT], w1[KT];
        load_row<KT>(P + (int64_t)c0 * a.ldP, w0);
        load_row<KT>(P + (int64_t)c1 * a.ldP, w1);
        accum_all<KT, EPG, PART * EP, 0, AT>(acc, w0, y0);
        accum_all<KT, EPG, PART * EP, 0, AT>(acc, w1, y1);
    }
    if (e < cnt) {
        const int64_t q = m.begin + e;
        const int c = __ldg(a.idx + q);
        const AT y = __ldg(val + q);
        AT w[KT];
        load_row<KT>(P + (int64_t)c * a.ldP, w);
        accum_all<KT, EPG, PART * EP, 0, AT>(acc, w, y);
    }
    rs_group<EPG, G / 2, EPG, AT>(acc, lane);
    constexpr int PER = EPG / G;
    if (has) {
        AT *dst = part + (item - a.item0) * (int64_t)a.ld + PART * EP + li * PER;
#pragma unroll
        for (int v = 0; v < PER; ++v) dst[v] = acc[v];
    }
    if constexpr (G == 32) {
        // A row split over several items: the warp that completes the row's last item sums all
        // of the row's partials (FP64, item order) into the row's slot.  Publication order:
        // partial stores, fence, counter increment (no warp ever waits on another).
        const int mi = a.multi_idx[m.row];
        if (mi >= 0) {
            __threadfence();
            int last = 0;
            const int64_t r_i0 = a.item_ptr[m.row], r_i1 = a.item_ptr[m.row + 1];
            if (lane == 0) {
                const int old = atomicAdd(a.counters + (int64_t)mi * a.nparts + PART, 1);
                last = old == (int)(r_i1 - r_i0) - 1;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                const int e1 = min((PART + 1) * EP, a.nv);
                for (int q = PART * EP + lane; q < e1; q += 32) {
                    double sum = 0.0;
                    for (int64_t it = r_i0; it < r_i1; ++it)
                        sum += (double)__ldcg(part + (it - a.item0) * (int64_t)a.ld + q);
                    a.rowsum[(int64_t)mi * a.ld_sum + q] = sum;
                }
                if (lane == 0) a.counters[(int64_t)mi * a.nparts + PART] = 0;
            }
        }
    }
}

template <int KT, typename GT, typename AT, int EP, int PART>
__device__ __forceinline__ void gram_body(const GramParams &a)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < a.n_tasks; t += nwarps) {
        const GramTask tk = a.tasks[t];
        if (tk.G == 8)
            gram_task<KT, GT, AT, EP, PART, 8>(a, tk, lane);
        else if (tk.G == 16)
            gram_task<KT, GT, AT, EP, PART, 16>(a, tk, lane);
        else
            gram_task<KT, GT, AT, EP, PART, 32>(a, tk, lane);
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
__global__ void __launch_bounds__(256, (EP > 96 ? 1 : 2)) gram_kernel(GramParams a)
{
    constexpr int NP = (gram_nv(KT) + EP - 1) / EP;
    gram_dispatch<KT, GT, AT, EP, 0, NP>(blockIdx.y, a);
}

template <int KT, typename GT, typename AT>
static void launch_gram_t(const GramParams &a, int grid, int nparts, cudaStream_t st)
{
    constexpr int EP = ep_of(KT, sizeof(AT) == 8);
    dim3 g(grid, nparts);
    gram_kernel<KT, GT, AT, EP><<<g, 256, 0, st>>>(a);
}

template <typename GT, typename AT>
static void launch_gram_k(int KT, const GramParams &a, int grid, int nparts, cudaStream_t st)
{
    switch (KT) {
    case 2: launch_gram_t<2, GT, AT>(a, grid, nparts, st); break;
    case 4: launch_gram_t<4, GT, AT>(a, grid, nparts, st); break;
    case 6: launch_gram_t<6, GT, AT>(a, grid, nparts, st); break;
    case 8: launch_gram_t<8, GT, AT>(a, grid, nparts, st); break;
    case 10: launch_gram_t<10, GT, AT>(a, grid, nparts, st); break;
    case 12: launch_gram_t<12, GT, AT>(a, grid, nparts, st); break;
    case 14: launch_gram_t<14, GT, AT>(a, grid, nparts, st); break;
    case 16: launch_gram_t<16, GT, AT>(a, grid, nparts, st); break;
    default: break;
    }
}

void launch_gram(int K, int prec, const GramParams &a, int grid, cudaStream_t st)
{
    if (a.n_tasks == 0) return;
    const int KT = padded_k(K), np = gram_parts(K, prec);
    if (prec == BMF_FP64)
        launch_gram_k<double, double>(KT, a, grid, np, st);
    else if (prec == BMF_FP32)
        launch_gram_k<float, float>(KT, a, grid, np, st);
    else
        launch_gram_k<__nv_bfloat16, float>(KT, a, grid, np, st);
}

}  // namespace bmf
