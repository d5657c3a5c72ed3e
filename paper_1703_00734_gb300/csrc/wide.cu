// wide.cu -- the Gram-gather pass and the conditional draw for K > 16 (same mathematics as
// gram.cu and cond.cu; Eqs. 2-4 and the cost terms of Section 4.3).
//
// Gram: one warp per work item; 32 gathered partner rows are staged in shared memory per step
// and contracted on the tensor cores:
//   * BF16 gathers: mma.sync m16n8k16 (BF16 x BF16 -> FP32), fragments by ldmatrix.trans from
//     row-major staged rows; the right-hand side sum y p rides along as two extra columns holding
//     y split into BF16 high and low parts (so y keeps about 16 bits);
//   * FP32 gathers: split TF32 (p = hi + lo, three m16n8k8 products hi.hi + hi.lo + lo.hi),
//     which keeps close to FP32 accuracy;
//   * FP64 gathers: lanes over the Gram entries with FP64 FMAs (the FP64 pipe is the bound).
// Only the lower-triangular 16 x 8 tiles are computed.  Partials use the packed-lower layout of
// the exact K followed by the K right-hand-side entries; rows split over several items are
// finished by the warp that completes the last item (fence + counter, no waiting).
//
// Conditional: one warp per row, the packed matrix in shared memory; right-looking FP64
// Cholesky with the trailing update spread over the lanes element by element; column-oriented
// forward and back solves.  Per-block statistics of the new state for the next hyperparameter
// draw, as in cond.cu.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

constexpr int kWideObs = 32;     // staged observations per step
constexpr int kWideWarps = 4;    // warps per block (conditional kernel)

// ------------------------------------------------------------------------------------------
// tensor-core helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                          uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t addr, uint32_t &r0, uint32_t &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, "
                 "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t tf32_of(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Lower-triangular tile list of an M x N grid of 16 x 8 tiles plus one right-hand-side tile
// per 16-row block: tile t of block row mi covers rows 16 mi.., columns 8 nj.. (nj <= 2 mi + 1),
// and the extra tile nj = KT / 8 holds the right-hand side.
template <int KT>
struct WideTiles {
    static constexpr int M = KT / 16;
    static constexpr int NT = M * (M + 1) + M;  // sum_{mi} (2 mi + 2) lower tiles + M rhs tiles
};

__device__ __forceinline__ int tile_mi(int t, int &nj, int M)
{
    // tiles of block row mi: 2 mi + 2 lower tiles, then one rhs tile
    int mi = 0, base = 0;
    while (t >= base + 2 * mi + 3) {
        base += 2 * mi + 3;
        ++mi;
    }
    const int off = t - base;
    nj = off < 2 * mi + 2 ? off : -1;   // -1: the rhs tile
    return mi;
}

// Write one item's accumulators to its partial (packed lower entries, then the rhs).
template <int KT>
__device__ __forceinline__ void store_tiles(float *dst, const float (&acc)[WideTiles<KT>::NT][4],
                                            int lane, int K)
{
    constexpr int M = WideTiles<KT>::M;
    const int g = lane >> 2, tig = lane & 3;
    const int NTK = ntri(K);
#pragma unroll
    for (int t = 0; t < WideTiles<KT>::NT; ++t) {
        int nj;
        const int mi = tile_mi(t, nj, M);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int i = 16 * mi + g + (h >= 2 ? 8 : 0);
            const int cc = 2 * tig + (h & 1);
            if (i >= K) continue;
            if (nj >= 0) {
                const int j = 8 * nj + cc;
                if (j <= i && j < K) dst[tri(i, j)] = acc[t][h];
            } else if (cc == 0) {
                // rhs: column 0 = y high part, column 1 = y low part -> combine
                dst[NTK + i] = acc[t][h] + acc[t][h + 1];
            }
        }
    }
}

// Rows split over several items: the warp completing the last item sums the partials (FP64).
__device__ __forceinline__ void finish_row(const GramParams &a, const GramItem &m, float *part,
                                           int lane)
{
    const int mi = a.multi_idx[m.row];
    if (mi < 0) return;
    __threadfence();
    int last = 0;
    const int64_t r0 = a.item_ptr[m.row], r1 = a.item_ptr[m.row + 1];
    if (lane == 0) last = atomicAdd(a.counters + mi, 1) == (int)(r1 - r0) - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    for (int q = lane; q < a.nv; q += 32) {
        double s = 0.0;
        for (int64_t it = r0; it < r1; ++it) s += (double)__ldcg(part + (it - a.item0) * (int64_t)a.ld + q);
        a.rowsum[(int64_t)mi * a.ld_sum + q] = s;
    }
    if (lane == 0) a.counters[mi] = 0;
}

// ------------------------------------------------------------------------------------------
// BF16 Gram: rows [obs][KT + 8] in shared memory (columns KT, KT+1: y high/low, then zeros)
// ------------------------------------------------------------------------------------------
template <int KT>
__global__ void __launch_bounds__(128) gram_wide_bf16(GramParams a)
{
    constexpr int LDS = KT + 8;           // bf16 per staged row (bank-conflict free for ldmatrix)
    constexpr int M = WideTiles<KT>::M, NTL = WideTiles<KT>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __nv_bfloat16 *S = reinterpret_cast<__nv_bfloat16 *>(smraw) + wib * kWideObs * LDS;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(S);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const __nv_bfloat16 *P = static_cast<const __nv_bfloat16 *>(a.P);
    const float *val = static_cast<const float *>(a.val);
    float *part = static_cast<float *>(a.part);
    const int K = a.K;
    for (int64_t it = warp; it < a.n_items; it += nwarps) {
        const GramItem m = a.items[it];
        float acc[NTL][4];
#pragma unroll
        for (int t = 0; t < NTL; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
        // software pipeline: lane o holds in registers the rows and values of observation
        // o0 + o + 32 d for the next D steps d = 0..D-1 (gathered while the tensor cores work on
        // earlier steps) and the index of observation o0 + o + 32 D; D = 2 while the registers
        // allow it (KT <= 48), else 1
        constexpr int D = KT <= 48 ? 2 : 1;
        uint4 nxt[D][KT / 8];
        float ny[D];
        bool nvalid[D];
        int cnext = 0;
#pragma unroll
        for (int dd = 0; dd < D; ++dd) {
            const int od = dd * kWideObs + lane;
            nvalid[dd] = od < m.count;
            ny[dd] = 0.f;
            const int cd = nvalid[dd] ? __ldg(a.idx + m.begin + od) : 0;
            if (nvalid[dd]) {
                ny[dd] = __ldg(val + m.begin + od);
                const uint4 *src = reinterpret_cast<const uint4 *>(P + (int64_t)cd * a.ldP);
#pragma unroll
                for (int v = 0; v < KT / 8; ++v) nxt[dd][v] = __ldg(src + v);
            }
        }
        cnext = D * kWideObs + lane < m.count ? __ldg(a.idx + m.begin + D * kWideObs + lane) : 0;
        for (int o0 = 0; o0 < m.count; o0 += kWideObs) {
            // stage: lane o writes observation o0 + o (zero row past the end)
            __nv_bfloat16 *row = S + lane * LDS;
            if (nvalid[0]) {
#pragma unroll
                for (int v = 0; v < KT / 8; ++v) reinterpret_cast<uint4 *>(row)[v] = nxt[0][v];
                const __nv_bfloat16 hi = __float2bfloat16_rn(ny[0]);
                const __nv_bfloat16 lo = __float2bfloat16_rn(ny[0] - __bfloat162float(hi));
                uint4 tail = make_uint4(0u, 0u, 0u, 0u);
                tail.x = (uint32_t)__bfloat16_as_ushort(hi) | ((uint32_t)__bfloat16_as_ushort(lo) << 16);
                reinterpret_cast<uint4 *>(row)[KT / 8] = tail;
            } else {
#pragma unroll
                for (int v = 0; v <= KT / 8; ++v) reinterpret_cast<uint4 *>(row)[v] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncwarp();
            {
#pragma unroll
                for (int dd = 0; dd + 1 < D; ++dd) {
                    nvalid[dd] = nvalid[dd + 1];
                    ny[dd] = ny[dd + 1];
#pragma unroll
                    for (int v = 0; v < KT / 8; ++v) nxt[dd][v] = nxt[dd + 1][v];
                }
                const int o1 = o0 + D * kWideObs + lane;
                nvalid[D - 1] = o1 < m.count;
                if (nvalid[D - 1]) {
                    ny[D - 1] = __ldg(val + m.begin + o1);
                    const uint4 *src = reinterpret_cast<const uint4 *>(P + (int64_t)cnext * a.ldP);
#pragma unroll
                    for (int v = 0; v < KT / 8; ++v) nxt[D - 1][v] = __ldg(src + v);
                }
                cnext = o1 + kWideObs < m.count ? __ldg(a.idx + m.begin + o1 + kWideObs) : 0;
            }
            // two k-steps of 16 observations
#pragma unroll
            for (int ks = 0; ks < kWideObs / 16; ++ks) {
                const int kb = ks * 16;
                // ldmatrix row addresses: lanes 0-7 / 8-15 / 16-23 / 24-31 give the 8 rows of
                // sub-matrices (k 0-7, cols c..c+7), (k 0-7, c+8..), (k 8-15, c..), (k 8-15, c+8..)
                const int r8 = lane & 7, sub = lane >> 3;
                uint32_t afr[M][4];
#pragma unroll
                for (int mi = 0; mi < M; ++mi) {
                    const int krow = kb + r8 + ((sub & 2) ? 8 : 0);
                    const int col = 16 * mi + ((sub & 1) ? 8 : 0);
                    ldsm_x4_t(sbase + (uint32_t)((krow * LDS + col) * 2), afr[mi][0], afr[mi][1],
                              afr[mi][2], afr[mi][3]);
                }
#pragma unroll
                for (int t = 0; t < NTL; ++t) {
                    int nj;
                    const int mi = tile_mi(t, nj, M);
                    const int col = nj >= 0 ? 8 * nj : KT;
                    uint32_t b0, b1;
                    // x2: lanes 0-7 rows k 0-7, lanes 8-15 rows k 8-15 of columns col..col+7
                    const int krow = kb + r8 + ((sub & 1) ? 8 : 0);
                    ldsm_x2_t(sbase + (uint32_t)((krow * LDS + col) * 2), b0, b1);
                    mma_bf16(acc[t], afr[mi], b0, b1);
                }
            }
            __syncwarp();
        }
        store_tiles<KT>(part + it * (int64_t)a.ld, acc, lane, K);
        finish_row(a, m, part, lane);
    }
}

// ------------------------------------------------------------------------------------------
// FP32 Gram by split TF32 (SPLIT: hi.hi + hi.lo + lo.hi per tile) or single-pass TF32 (hi.hi):
// rows [obs][KT + 4] floats in shared memory (column KT holds y)
// ------------------------------------------------------------------------------------------
template <int KT, bool SPLIT>
__global__ void __launch_bounds__(128) gram_wide_tf32(GramParams a)
{
    constexpr int LDS = KT + 8;           // conflict-free fragment loads; column KT holds y
    constexpr int M = WideTiles<KT>::M, NTL = WideTiles<KT>::NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *S = reinterpret_cast<float *>(smraw) + wib * kWideObs * LDS;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float *P = static_cast<const float *>(a.P);
    const float *val = static_cast<const float *>(a.val);
    float *part = static_cast<float *>(a.part);
    const int K = a.K;
    const int g = lane >> 2, tig = lane & 3;
    for (int64_t it = warp; it < a.n_items; it += nwarps) {
        const GramItem m = a.items[it];
        float acc[NTL][4];
#pragma unroll
        for (int t = 0; t < NTL; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
        for (int o0 = 0; o0 < m.count; o0 += kWideObs) {
            const int o = lane;
            float *row = S + o * LDS;
            if (o0 + o < m.count) {
                const int64_t q = m.begin + o0 + o;
                const int c = __ldg(a.idx + q);
                const float4 *src = reinterpret_cast<const float4 *>(P + (int64_t)c * a.ldP);
#pragma unroll
                for (int v = 0; v < KT / 4; ++v) reinterpret_cast<float4 *>(row)[v] = __ldg(src + v);
                reinterpret_cast<float4 *>(row)[KT / 4] = make_float4(__ldg(val + q), 0.f, 0.f, 0.f);
                reinterpret_cast<float4 *>(row)[KT / 4 + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
#pragma unroll
                for (int v = 0; v < LDS / 4; ++v) reinterpret_cast<float4 *>(row)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncwarp();
#pragma unroll
            for (int ks = 0; ks < kWideObs / 8; ++ks) {
                const int kb = ks * 8;
                // A = P^T (latent x obs): a0 (g, tig), a1 (g+8, tig), a2 (g, tig+4), a3 (g+8, tig+4)
                uint32_t ah[M][4], al[M][4];
#pragma unroll
                for (int mi = 0; mi < M; ++mi) {
                    const float v[4] = {S[(kb + tig) * LDS + 16 * mi + g], S[(kb + tig) * LDS + 16 * mi + g + 8],
                                        S[(kb + tig + 4) * LDS + 16 * mi + g], S[(kb + tig + 4) * LDS + 16 * mi + g + 8]};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        ah[mi][h] = tf32_of(v[h]);
                        if constexpr (SPLIT) al[mi][h] = tf32_of(v[h] - __uint_as_float(ah[mi][h]));
                    }
                }
#pragma unroll
                for (int t = 0; t < NTL; ++t) {
                    int nj;
                    const int mi = tile_mi(t, nj, M);
                    const int col = nj >= 0 ? 8 * nj : KT;
                    const float bv0 = S[(kb + tig) * LDS + col + g], bv1 = S[(kb + tig + 4) * LDS + col + g];
                    const uint32_t bh0 = tf32_of(bv0), bh1 = tf32_of(bv1);
                    if constexpr (SPLIT) {
                        const uint32_t bl0 = tf32_of(bv0 - __uint_as_float(bh0));
                        const uint32_t bl1 = tf32_of(bv1 - __uint_as_float(bh1));
                        mma_tf32(acc[t], al[mi], bh0, bh1);
                        mma_tf32(acc[t], ah[mi], bl0, bl1);
                    }
                    mma_tf32(acc[t], ah[mi], bh0, bh1);
                }
            }
            __syncwarp();
        }
        store_tiles<KT>(part + it * (int64_t)a.ld, acc, lane, K);
        finish_row(a, m, part, lane);
    }
}

// ------------------------------------------------------------------------------------------
// FP64 Gram: lanes over entries (packed lower, then rhs) of 32 staged rows [obs][K + 1]
// ------------------------------------------------------------------------------------------
template <int MAXP>
__global__ void __launch_bounds__(128) gram_wide_fp64(GramParams a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = a.K, LDS = K + 1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *S = reinterpret_cast<double *>(smraw) + wib * kWideObs * LDS;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const double *P = static_cast<const double *>(a.P);
    const double *val = static_cast<const double *>(a.val);
    double *part = static_cast<double *>(a.part);
    const int NTK = ntri(K), NV = NTK + K;
    for (int64_t it = warp; it < a.n_items; it += nwarps) {
        const GramItem m = a.items[it];
        double acc[MAXP];
#pragma unroll
        for (int u = 0; u < MAXP; ++u) acc[u] = 0.0;
        for (int o0 = 0; o0 < m.count; o0 += kWideObs) {
            const int nobs = min(kWideObs, m.count - o0);
            for (int q = lane; q < nobs * LDS; q += 32) {
                const int o = q / LDS, k = q % LDS;
                const int64_t oq = m.begin + o0 + o;
                S[q] = k < K ? P[(int64_t)__ldg(a.idx + oq) * a.ldP + k] : __ldg(val + oq);
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < MAXP; ++u) {
                const int e = lane + 32 * u;
                if (e >= NV) continue;
                int i, j;
                if (e < NTK) {
                    i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                    while (i * (i + 1) / 2 > e) --i;
                    while ((i + 1) * (i + 2) / 2 <= e) ++i;
                    j = e - i * (i + 1) / 2;
                } else {
                    i = e - NTK;
                    j = K;   // the value column
                }
                double s = acc[u];
                for (int o = 0; o < nobs; ++o) s = fma(S[o * LDS + i], S[o * LDS + j], s);
                acc[u] = s;
            }
            __syncwarp();
        }
        double *dst = part + it * (int64_t)a.ld;
#pragma unroll
        for (int u = 0; u < MAXP; ++u)
            if (lane + 32 * u < NV) dst[lane + 32 * u] = acc[u];
        // split rows
        const int mi = a.multi_idx[m.row];
        if (mi >= 0) {
            __threadfence();
            int last = 0;
            const int64_t r0 = a.item_ptr[m.row], r1 = a.item_ptr[m.row + 1];
            if (lane == 0) last = atomicAdd(a.counters + mi, 1) == (int)(r1 - r0) - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                for (int q = lane; q < NV; q += 32) {
                    double sum = 0.0;
                    for (int64_t j = r0; j < r1; ++j) sum += __ldcg(part + (j - a.item0) * (int64_t)a.ld + q);
                    a.rowsum[(int64_t)mi * a.ld_sum + q] = sum;
                }
                if (lane == 0) a.counters[mi] = 0;
            }
        }
    }
}

int wide_kt(int K) { return K <= 32 ? 32 : (K <= 48 ? 48 : 64); }

// Partial entries per item for K > 16 (exact K layout, padded to a multiple of 4).
int wide_part_ld(int K) { return (ntri(K) + K + 3) / 4 * 4; }

template <int KT, bool SPLIT>
static void launch_tf32_t(const GramParams &a, int grid, cudaStream_t st)
{
    const size_t smem = (size_t)4 * kWideObs * (KT + 8) * 4;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(gram_wide_tf32<KT, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    gram_wide_tf32<KT, SPLIT><<<grid, 128, smem, st>>>(a);
}

template <int KT>
static void launch_wide_t(int prec, const GramParams &a, int grid, cudaStream_t st, bool single)
{
    if (prec == BMF_BF16) {
        const size_t smem = (size_t)4 * kWideObs * (KT + 8) * 2;
        gram_wide_bf16<KT><<<grid, 128, smem, st>>>(a);
    } else if (single) {
        launch_tf32_t<KT, false>(a, grid, st);
    } else {
        launch_tf32_t<KT, true>(a, grid, st);
    }
}

void launch_gram_wide(int K, int prec, const GramParams &a, int grid, cudaStream_t st, bool tf32_single)
{
    if (a.n_items == 0) return;
    if (prec == BMF_FP64) {
        const size_t smem = (size_t)4 * kWideObs * (K + 1) * 8;
        const int nv = ntri(K) + K;
        if (nv <= 18 * 32) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(gram_wide_fp64<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            gram_wide_fp64<18><<<grid, 128, smem, st>>>(a);
        } else if (nv <= 38 * 32) {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(gram_wide_fp64<38>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            gram_wide_fp64<38><<<grid, 128, smem, st>>>(a);
        } else {
            if (smem > 48 * 1024)
                cudaFuncSetAttribute(gram_wide_fp64<67>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            gram_wide_fp64<67><<<grid, 128, smem, st>>>(a);
        }
        return;
    }
    switch (wide_kt(K)) {
    case 32: launch_wide_t<32>(prec, a, grid, st, tf32_single); break;
    case 48: launch_wide_t<48>(prec, a, grid, st, tf32_single); break;
    default: launch_wide_t<64>(prec, a, grid, st, tf32_single); break;
    }
}

// ------------------------------------------------------------------------------------------
// Conditional draw for K >= 13: a team of T lanes per row (T = 4 for K <= 16, 16 for K <= 48,
// 32 above), 32 / T rows per warp at a time; below K = 13 one thread per row (cond.cu) is as
// fast.  Measured on this GPU: equal at K = 10, the team form 18% faster at K = 16; at K = 32
// teams of 16 lanes 7% faster than teams of 8 and 20% faster than 32.
// The row's packed matrix lives in shared memory; the team factors it right-looking (each step:
// the pivot, read by every lane, then the column scaled and the trailing triangle updated with
// the entries spread over the team), then solves column by column.  On this GPU the FP64 pipe
// issues one warp instruction every few dozen cycles per SM partition, so the pivot chain
// (square root, reciprocal) is what one row costs serially; several rows per warp share it,
// while the O(K^3) trailing updates keep all lanes busy.  Every team of a warp runs the same
// number of steps (rows beyond the block and rows that fail the positive-definiteness test
// still run the loop structure), and synchronisation is per team.
// ------------------------------------------------------------------------------------------
template <typename GT>
__device__ __forceinline__ GT to_gather_w(double x);
template <>
__device__ __forceinline__ double to_gather_w<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_gather_w<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_gather_w<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

template <typename AT>
__device__ __forceinline__ AT to_acc(double x) { return x; }
template <typename AT>
__device__ __forceinline__ AT to_acc(float x) { return x; }
template <typename AT>
__device__ __forceinline__ AT to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float acc_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double acc_fma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ void decode_packed(int e, int &i, int &j)
{
    i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    j = e - i * (i + 1) / 2;
}

// Default lanes per row: two (the register-resident pair kernel of cond_pair.cu) up to K = 16,
// then 16, then 32.  Measured on the 100k x 20k, K = 16 PP workload: the pair kernel takes
// 1.10 ms per stage-3 X half against 1.33 ms for four-lane teams.
int cond_team_size(int K) { return K <= 16 ? 2 : (K <= 48 ? 16 : 32); }

// Doubles per team in shared memory: the packed matrix, right-hand side, pivots and (teams of 8
// or more lanes) a contiguous copy of the current column, rounded up to a multiple of 8 doubles
// and offset by T mod 16 doubles (4 for teams of 16 or 32 lanes), so that consecutive teams of
// a warp start in different banks.  Rounding to 8 rather than 16 doubles lets five blocks of
// 4-lane teams share an SM at K = 16 (44 KB each).  The column copy removes the strided reads of
// the trailing update; for 4-lane teams (K <= 16) the extra shared memory would cost a resident
// block per SM, which measured slower.
__host__ __device__ constexpr bool team_colcopy(int T) { return T >= 8; }
__host__ __device__ constexpr int team_stride(int K, int T)
{
    return (ntri(K) + (team_colcopy(T) ? 3 : 2) * K + 7) / 8 * 8 + (T % 16 == 0 ? 4 : T % 16);
}

bool cond_lanes_valid(int K, int lanes)
{
    if (lanes == 2 && K >= 13 && K <= 16) return true;
    if (lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 && lanes != 32) return false;
    const size_t smem = (size_t)(32 * kWideWarps / lanes) * team_stride(K, lanes) * sizeof(double);
    return smem <= 227 * 1024;
}

template <typename GT, typename AT, int T>
__global__ void __launch_bounds__(32 * kWideWarps) cond_team_kernel(CondParams a)
{
    extern __shared__ double smw[];
    constexpr int NTEAM = 32 * kWideWarps / T;
    const int K = a.K, NT = ntri(K);
    const int tl = threadIdx.x % T, tm = threadIdx.x / T;
    const unsigned mask = T == 32 ? 0xffffffffu : (((1u << T) - 1u) << ((threadIdx.x & 31) & ~(T - 1)));
    const int per_team = team_stride(K, T);
    double *M = smw + tm * per_team, *B = M + NT, *RI = B + K, *CK = RI + K;
    const CondBlock blk = a.blocks[blockIdx.x];
    const int64_t R = a.R;
    const double tau = a.tau;
    const int rounds = (blk.n + NTEAM - 1) / NTEAM;
    for (int rd = 0; rd < rounds; ++rd) {
        const int q = rd * NTEAM + tm;
        const bool active = q < blk.n;
        const int64_t r = blk.row0 + (active ? q : 0);
        // 1-2. G, r and the prior
        if (active) {
            const int64_t i0 = a.item_ptr[r], i1 = a.item_ptr[r + 1];
            const int mi = a.multi_idx[r];
            const int h = a.row_hslot[r];
            const double *hp = h >= 0 ? a.hyper + (int64_t)h * hyper_slot_len(K) : nullptr;
            const AT *pp = static_cast<const AT *>(a.part) + (i0 - a.item0) * (int64_t)a.ld;
            const double *ps = mi >= 0 ? a.rowsum + (int64_t)mi * a.ld_sum : nullptr;
            const double tau_r = a.tau_row ? a.tau_row[r] : tau;
            for (int e = tl; e < NT + K; e += T) {
                const int src = e < NT ? e : a.part_rhs + (e - NT);
                double gsum;
                if (mi == kFusedRow) {
                    // a row with few observations: the entry from its list, in list order (the
                    // same operations as the two-lane conditional)
                    int ii, jj;
                    if (e < NT)
                        decode_packed(e, ii, jj);
                    else
                        ii = e - NT, jj = -1;
                    AT acc = AT(0);
                    for (int64_t o = a.obs_ptr[r]; o < a.obs_ptr[r + 1]; ++o) {
                        const GT *pr = static_cast<const GT *>(a.P) + (int64_t)a.obs_idx[o] * a.ldP;
                        const AT pi = to_acc<AT>(pr[ii]);
                        acc = jj >= 0 ? acc_fma(pi, to_acc<AT>(pr[jj]), acc)
                                      : acc_fma(static_cast<const AT *>(a.obs_val)[o], pi, acc);
                    }
                    gsum = widen(acc);
                } else {
                    gsum = ps ? ps[src] : (i1 > i0 ? widen(pp[src]) : 0.0);
                }
                double prior;
                if (e < NT)
                    prior = hp ? hp[K + e] : a.prior_L[(int64_t)e * R + r];
                else
                    prior = hp ? hp[K + NT + (e - NT)] : a.prior_b[(int64_t)(e - NT) * R + r];
                M[e] = fma(tau_r, gsum, prior);   // M[NT + i] is B[i]
            }
        }
        __syncwarp(mask);
        // 3. right-looking Cholesky
        bool ok = active;
        for (int k = 0; k < K; ++k) {
            const int kk = tri(k, k);
            const double d = ok ? M[kk] : 1.0;
            if (!pivot_ok(d)) ok = false;
            const double rs = ok ? pivot_rsqrt<GT>(d) : 0.0;
            __syncwarp(mask);
            if (ok) {
                // the scaled column also goes to CK[i], contiguous, for the trailing update
                for (int i = k + 1 + tl; i < K; i += T) {
                    const double l = M[tri(i, k)] * rs;
                    M[tri(i, k)] = l;
                    if constexpr (team_colcopy(T)) CK[i] = l;
                }
                if (tl == 0) RI[k] = rs;   // the solves scale by 1 / L_kk; L_kk itself is not kept
            }
            __syncwarp(mask);
            if (ok) {
                // trailing triangle rows i = k+1..K-1, columns j = k+1..i, row by row; lane tl
                // takes positions tl, tl + T, ... (row i holds i - k of them)
                int i = k + 1, j = k + 1 + tl;
                while (i < K && j > i) {
                    j -= i - k;
                    ++i;
                }
                while (i < K) {
                    if constexpr (team_colcopy(T))
                        M[tri(i, j)] = fma(-CK[i], CK[j], M[tri(i, j)]);
                    else
                        M[tri(i, j)] = fma(-M[tri(i, k)], M[tri(j, k)], M[tri(i, j)]);
                    j += T;
                    while (i < K && j > i) {
                        j -= i - k;
                        ++i;
                    }
                }
            }
            __syncwarp(mask);
        }
        if (active && !ok && tl == 0) {
            atomicOr(&a.err->flags, ERR_NOT_PD);
            atomicMin(&a.err->first_bad_row, (int)r);
        }
        // 4. forward solve L y = b (column oriented)
        for (int k = 0; k < K; ++k) {
            const double yk = ok ? B[k] * RI[k] : 0.0;
            __syncwarp(mask);
            if (ok) {
                for (int i = k + 1 + tl; i < K; i += T) B[i] = fma(-M[tri(i, k)], yk, B[i]);
                if (tl == 0) B[k] = yk;
            }
            __syncwarp(mask);
        }
        // 5. back solve L^T x = y + z (column oriented)
        if (ok) {
            const double *z = a.z + (r - a.row0) * K;
            for (int i = tl; i < K; i += T) B[i] += z[i];
        }
        __syncwarp(mask);
        for (int i = K - 1; i >= 0; --i) {
            const double xi = ok ? B[i] * RI[i] : 0.0;
            __syncwarp(mask);
            if (ok) {
                for (int k = tl; k < i; k += T) B[k] = fma(-M[tri(i, k)], xi, B[k]);
                if (tl == 0) B[i] = xi;
            }
            __syncwarp(mask);
        }
        // 6. state, gathered copy, moments
        if (active) {
            GT *g = static_cast<GT *>(a.Xg) + r * a.ldg;
            for (int i = tl; i < a.ldg; i += T) {
                const double xi = (ok && i < K) ? B[i] : 0.0;
                if (ok) g[i] = to_gather_w<GT>(xi);
                if (i < K && ok) {
                    a.X[r * K + i] = xi;
                    if (a.keep) a.S1[(int64_t)i * R + r] += xi;
                }
            }
            if (ok && a.keep && a.full)
                for (int e = tl; e < NT; e += T) {
                    int i, j;
                    decode_packed(e, i, j);
                    a.S2[(int64_t)e * R + r] += B[i] * B[j];
                }
        }
        __syncwarp(mask);
    }
    // 7. per-block statistics of the new state (unless computed on another stream), read back
    //    from the state rows this block has just written (visible to the block after the
    //    barrier, and still in L1); no shared-memory copy, so more blocks fit on an SM
    // (only blocks whose factor draws its hyperparameters need them: a block of rows with
    // propagated per-row priors skips them; every row of a block shares its subset's prior)
    if (a.stats == nullptr || a.row_hslot[blk.row0] < 0) return;
    __syncthreads();
    const int NS = K + NT;
    const double *Xb = a.X + blk.row0 * K;
    double *out = a.stats + (a.blk0 + blockIdx.x) * (int64_t)NS;
    for (int e = threadIdx.x; e < NS; e += blockDim.x) {
        double s = 0.0;
        if (e < K) {
            for (int q = 0; q < blk.n; ++q) s += Xb[q * K + e];
        } else {
            int i, j;
            decode_packed(e - K, i, j);
            for (int q = 0; q < blk.n; ++q) s = fma(Xb[q * K + i], Xb[q * K + j], s);
        }
        out[e] = s;
    }
}

template <typename GT, typename AT, int T>
static void launch_cond_team_t(const CondParams &a, int n_blocks, cudaStream_t st)
{
    constexpr int NTEAM = 32 * kWideWarps / T;
    const size_t smem = (size_t)NTEAM * team_stride(a.K, T) * sizeof(double);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(cond_team_kernel<GT, AT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cond_team_kernel<GT, AT, T><<<n_blocks, 32 * kWideWarps, smem, st>>>(a);
}

template <typename GT, typename AT>
static void launch_cond_team_p(const CondParams &a, int n_blocks, int team, cudaStream_t st)
{
    switch (team) {
    case 2: launch_cond_team_t<GT, AT, 2>(a, n_blocks, st); break;
    case 4: launch_cond_team_t<GT, AT, 4>(a, n_blocks, st); break;
    case 8: launch_cond_team_t<GT, AT, 8>(a, n_blocks, st); break;
    case 16: launch_cond_team_t<GT, AT, 16>(a, n_blocks, st); break;
    default: launch_cond_team_t<GT, AT, 32>(a, n_blocks, st); break;
    }
}

void launch_cond_team(int prec, const CondParams &a, int n_blocks, int team, cudaStream_t st)
{
    if (n_blocks <= 0) return;
    if (prec == BMF_FP64)
        launch_cond_team_p<double, double>(a, n_blocks, team, st);
    else if (prec == BMF_FP32)
        launch_cond_team_p<float, float>(a, n_blocks, team, st);
    else
        launch_cond_team_p<__nv_bfloat16, float>(a, n_blocks, team, st);
}

}  // namespace bmf
