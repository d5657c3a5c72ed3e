// cond_pair.cu -- the FP64 conditional draw of a row for 13 <= K <= 16 with the row's matrix in
// registers (the same draw as cond.cu and the team kernel of wide.cu: Eqs. 2-4,
//   Lambda_n = Lambda_p + tau G_n, b_n = Lambda_p mu_p + tau r_n, Lambda_n = L L^T,
//   x_n = L^{-T} (L^{-1} b_n + z_n)).
//
// Two lanes factor one row, 16 rows per warp.  On this GPU a warp's FP64 instruction costs the
// same whatever its active lanes, so what a row costs is the FP64 warp instructions it takes:
// two lanes per row share each pivot's reciprocal square root among 16 rows (four-lane teams:
// 8 rows), and with the matrix in registers the trailing updates read no shared memory.  Lane l
// of a pair owns the rows i with i mod 4 in {0, 3} (l = 0) or {1, 2} (l = 1): slot s of a lane
// holds row 2s + (l xor (s & 1)), so both lanes hold about half of the packed triangle.  Column
// k of L reaches the other lane by shuffles.  Every entry sees the operations of the team kernel
// in the same order (right-looking Cholesky, column-oriented solves), so the values are
// bit-identical to it.  A row with few observations (kFusedRow) forms its own G_n and r_n from
// its list and the gathered partner rows, each entry accumulated in list order in the Gram
// pass's accumulation type, instead of reading Gram partials.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

namespace {

template <typename GT>
__device__ __forceinline__ GT narrow_to(double x);
template <>
__device__ __forceinline__ double narrow_to<double>(double x) { return x; }
template <>
__device__ __forceinline__ float narrow_to<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 narrow_to<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

// Row of slot s of lane l, the lane owning row i, and the entries slot s can hold.
__device__ __forceinline__ int pair_row(int s, int l) { return 2 * s + (l ^ (s & 1)); }
__host__ __device__ constexpr int pair_owner(int i) { return ((i & 3) == 1 || (i & 3) == 2) ? 1 : 0; }
__host__ __device__ constexpr int slot_len(int K, int s) { return 2 * s + 2 < K ? 2 * s + 2 : K; }

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void decode_tri_pair(int e, int &i, int &j)
{
    i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    j = e - i * (i + 1) / 2;
}

}  // namespace

constexpr int kPairThreads = 2 * kCondBlock;   // one conditional block of rows per CUDA block

// Shared-memory prefetch of a row's moment sums (S2 packed, then S1) while the row is factored:
// each lane copies the entries of its own rows and reads only those back, so the copy needs
// only the lane's own wait.
__device__ __forceinline__ void prefetch8(double *dst, const double *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void prefetch_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void prefetch_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

int cond_pair_smem(int K) { return kCondBlock * (ntri(K) + K) * (int)sizeof(double); }

// The first K entries of a gathered partner row (16-byte aligned, at least the padded K
// entries long) with vector loads, in the accumulation type of the Gram sums.
template <int K, typename GT, typename AT>
__device__ __forceinline__ void load_partner(const GT *__restrict__ p, AT (&w)[K])
{
    if constexpr (sizeof(GT) == 8) {
        const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
        for (int c = 0; c < (K + 1) / 2; ++c) {
            const double2 v = __ldg(q + c);
            w[2 * c] = v.x;
            if (2 * c + 1 < K) w[2 * c + 1] = v.y;
        }
    } else if constexpr (sizeof(GT) == 4) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int c = 0; c < (K + 3) / 4; ++c) {
            const float4 v = __ldg(q + c);
            const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (4 * c + u < K) w[4 * c + u] = f[u];
        }
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int c = 0; c < (K + 7) / 8; ++c) {
            const uint4 v = __ldg(q + c);
            const uint32_t u4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u4[u]));
                if (8 * c + 2 * u < K) w[8 * c + 2 * u] = f.x;
                if (8 * c + 2 * u + 1 < K) w[8 * c + 2 * u + 1] = f.y;
            }
        }
    }
}

__device__ __forceinline__ float macc(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double macc(double a, double b, double c) { return fma(a, b, c); }

template <int K, typename GT, typename AT>
__global__ void __launch_bounds__(kPairThreads) cond_pair_kernel(CondParams a)
{
    constexpr int S = (K + 1) / 2;
    constexpr int NT = ntri(K);
    const int lane = threadIdx.x & 31;
    const int l = lane & 1;
    const int pb = lane & ~1;
    const int q = threadIdx.x >> 1;
    const CondBlock blk = a.blocks[blockIdx.x];
    const bool active = q < blk.n;
    const int64_t r = blk.row0 + (active ? q : 0);
    const int64_t R = a.R;
    const double tau = a.tau_row ? a.tau_row[r] : a.tau;
    // the row's indices first, all in flight together (the observation range too, which a row
    // forming its own Gram sums needs before its first gather)
    const int64_t i0 = a.item_ptr[r], i1 = a.item_ptr[r + 1];
    const int mi = a.multi_idx[r];
    const int h = a.row_hslot[r];
    const int64_t o0 = a.obs_ptr[r], o1 = a.obs_ptr[r + 1];
    double M[S][K];
    double B[S], RI[S];
    // the moment sums of this row are fetched now and used after the draw (their global-memory
    // latency hides behind the factorisation)
    extern __shared__ double pre[];
    double *mine = pre + q * (NT + K);
    const bool moments = active && a.keep;
    if (moments) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = pair_row(s, l);
            if (i < K) {
                prefetch8(mine + NT + i, a.S1 + (int64_t)i * R + r);
                if (a.full)
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j)
                        if (j <= i) prefetch8(mine + tri(i, j), a.S2 + (int64_t)tri(i, j) * R + r);
            }
        }
        prefetch_commit();
    }
    // 1-2. G, r and the prior (inactive pairs carry an identity, so their arithmetic stays
    //      finite; they write nothing)
    if (active) {
        const double *hp = h >= 0 ? a.hyper + (int64_t)h * hyper_slot_len(K) : nullptr;
        const AT *pp = static_cast<const AT *>(a.part) + (i0 - a.item0) * (int64_t)a.ld;
        const double *ps = mi >= 0 ? a.rowsum + (int64_t)mi * a.ld_sum : nullptr;
        if (mi == kFusedRow) {
            // a row with few observations: its Gram sums from its own list, each entry
            // accumulated in list order (the Gram pass skips the row)
            AT G[S][K], Rv[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
#pragma unroll
                for (int j = 0; j < slot_len(K, s); ++j) G[s][j] = AT(0);
                Rv[s] = AT(0);
            }
            const int no = (int)(o1 - o0);
            // observations in groups of four: indices and values first, then the partner rows
            constexpr int QG = 4;
            for (int c0 = 0; c0 < no; c0 += QG) {
                int32_t pid[QG];
                AT yv[QG];
#pragma unroll
                for (int q2 = 0; q2 < QG; ++q2)
                    if (c0 + q2 < no) {
                        pid[q2] = a.obs_idx[o0 + c0 + q2];
                        yv[q2] = static_cast<const AT *>(a.obs_val)[o0 + c0 + q2];
                    }
#pragma unroll
                for (int q2 = 0; q2 < QG; ++q2)
                    if (c0 + q2 < no) {
                        AT pv[K];
                        load_partner<K, GT, AT>(static_cast<const GT *>(a.P) + (int64_t)pid[q2] * a.ldP,
                                                pv);
#pragma unroll
                        for (int s = 0; s < S; ++s) {
                            const int i = pair_row(s, l);
                            if (i < K) {
#pragma unroll
                                for (int j = 0; j < slot_len(K, s); ++j)
                                    if (j <= i) G[s][j] = macc(pv[i], pv[j], G[s][j]);
                                Rv[s] = macc(yv[q2], pv[i], Rv[s]);
                            }
                        }
                    }
            }
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int i = pair_row(s, l);
                if (i < K) {
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j)
                        if (j <= i) {
                            const int e = tri(i, j);
                            const double prior = hp ? hp[K + e] : a.prior_L[(int64_t)e * R + r];
                            M[s][j] = fma(tau, widen(G[s][j]), prior);
                        }
                    const double prior = hp ? hp[K + NT + i] : a.prior_b[(int64_t)i * R + r];
                    B[s] = fma(tau, widen(Rv[s]), prior);
                } else {
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j) M[s][j] = 0.0;
                    B[s] = 0.0;
                }
            }
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int i = pair_row(s, l);
                if (i < K) {
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j)
                        if (j <= i) {
                            const int e = tri(i, j);
                            const double gsum = ps ? ps[e] : (i1 > i0 ? widen(pp[e]) : 0.0);
                            const double prior = hp ? hp[K + e] : a.prior_L[(int64_t)e * R + r];
                            M[s][j] = fma(tau, gsum, prior);
                        }
                    const int src = a.part_rhs + i;
                    const double gsum = ps ? ps[src] : (i1 > i0 ? widen(pp[src]) : 0.0);
                    const double prior = hp ? hp[K + NT + i] : a.prior_b[(int64_t)i * R + r];
                    B[s] = fma(tau, gsum, prior);
                } else {
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j) M[s][j] = 0.0;
                    B[s] = 0.0;
                }
            }
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int j = 0; j < slot_len(K, s); ++j) M[s][j] = j == pair_row(s, l) ? 1.0 : 0.0;
            B[s] = 0.0;
        }
    }
    // 3. right-looking Cholesky: pivot k from its owner, column k scaled, trailing triangle
    //    updated with column k broadcast entry by entry
    bool ok = active;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double d = __shfl_sync(kFull, M[k / 2][k], pb + pair_owner(k));
        if (!pivot_ok(d)) ok = false;
        const double rs = ok ? pivot_rsqrt<GT>(d) : 0.0;
        if (l == pair_owner(k)) RI[k / 2] = rs;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (2 * s + 1 > k) {
                const int i = pair_row(s, l);
                if (i > k && i < K) M[s][k] = M[s][k] * rs;
            }
#pragma unroll
        for (int j = k + 1; j < K; ++j) {
            const double cj = __shfl_sync(kFull, M[j / 2][k], pb + pair_owner(j));
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (2 * s + 1 >= j) {
                    const int i = pair_row(s, l);
                    if (j <= i && i < K) M[s][j] = fma(-M[s][k], cj, M[s][j]);
                }
        }
    }
    if (active && !ok && l == 0) {
        atomicOr(&a.err->flags, ERR_NOT_PD);
        atomicMin(&a.err->first_bad_row, (int)r);
    }
    // 4. forward solve L y = b (column oriented)
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double yk = ok ? B[k / 2] * RI[k / 2] : 0.0;
        yk = __shfl_sync(kFull, yk, pb + pair_owner(k));
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (2 * s + 1 > k) {
                const int i = pair_row(s, l);
                if (ok && i > k && i < K) B[s] = fma(-M[s][k], yk, B[s]);
            }
        if (ok && l == pair_owner(k)) B[k / 2] = yk;
    }
    // 5. back solve L^T x = y + z (column oriented): x_i from its owner, then row i of L
    //    broadcast to update the rows below i
    if (ok) {
        const double *z = a.z + (r - a.row0) * K;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = pair_row(s, l);
            if (i < K) B[s] += z[i];
        }
    }
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        double xi = ok ? B[i / 2] * RI[i / 2] : 0.0;
        xi = __shfl_sync(kFull, xi, pb + pair_owner(i));
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (2 * s < i) {
                const double l0 = __shfl_sync(kFull, M[i / 2][2 * s], pb + pair_owner(i));
                const double l1 =
                    2 * s + 1 < i ? __shfl_sync(kFull, M[i / 2][2 * s + 1], pb + pair_owner(i)) : 0.0;
                const int k = pair_row(s, l);
                if (ok && k < i) B[s] = fma(-(k == 2 * s ? l0 : l1), xi, B[s]);
            }
        if (ok && l == pair_owner(i)) B[i / 2] = xi;
    }
    // 6. state, gathered copy, moments
    double xall[K];
#pragma unroll
    for (int j = 0; j < K; ++j) xall[j] = __shfl_sync(kFull, B[j / 2], pb + pair_owner(j));
    if (moments) prefetch_wait();
    if (active && ok) {
        GT *g = static_cast<GT *>(a.Xg) + r * a.ldg;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int i = pair_row(s, l);
            if (i < K) {
                a.X[r * K + i] = B[s];
                g[i] = narrow_to<GT>(B[s]);
                if (a.keep) a.S1[(int64_t)i * R + r] = mine[NT + i] + B[s];
            }
        }
        for (int i = K + l; i < a.ldg; i += 2) g[i] = narrow_to<GT>(0.0);
        if (a.keep && a.full) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int i = pair_row(s, l);
                if (i < K) {
#pragma unroll
                    for (int j = 0; j < slot_len(K, s); ++j)
                        if (j <= i) a.S2[(int64_t)tri(i, j) * R + r] = mine[tri(i, j)] + B[s] * xall[j];
                }
            }
        }
    }
    // 7. per-block statistics of the new state (unless computed on another stream), read back
    //    from the state rows this block has just written, each entry over the rows in order
    // (only blocks whose factor draws its hyperparameters need them: a block of rows with
    // propagated per-row priors skips them; every row of a block shares its subset's prior)
    if (a.stats == nullptr || a.row_hslot[blk.row0] < 0) return;
    __syncthreads();
    constexpr int NS = K + NT;
    const double *Xb = a.X + blk.row0 * K;
    double *out = a.stats + (a.blk0 + blockIdx.x) * (int64_t)NS;
    for (int e = threadIdx.x; e < NS; e += blockDim.x) {
        double s = 0.0;
        if (e < K) {
            for (int qq = 0; qq < blk.n; ++qq) s += Xb[qq * K + e];
        } else {
            int i, j;
            decode_tri_pair(e - K, i, j);
            for (int qq = 0; qq < blk.n; ++qq) s = fma(Xb[qq * K + i], Xb[qq * K + j], s);
        }
        out[e] = s;
    }
}

template <int K, typename GT, typename AT>
static void launch_pair_k(const CondParams &a, int n_blocks, cudaStream_t st)
{
    const int smem = a.keep ? cond_pair_smem(K) : 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(cond_pair_kernel<K, GT, AT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             cond_pair_smem(K));
    cond_pair_kernel<K, GT, AT><<<n_blocks, kPairThreads, smem, st>>>(a);
}

template <typename GT, typename AT>
static bool launch_pair_t(const CondParams &a, int n_blocks, cudaStream_t st)
{
    switch (a.K) {
    case 13: launch_pair_k<13, GT, AT>(a, n_blocks, st); return true;
    case 14: launch_pair_k<14, GT, AT>(a, n_blocks, st); return true;
    case 15: launch_pair_k<15, GT, AT>(a, n_blocks, st); return true;
    case 16: launch_pair_k<16, GT, AT>(a, n_blocks, st); return true;
    default: return false;
    }
}

bool launch_cond_pair(int prec, const CondParams &a, int n_blocks, cudaStream_t st)
{
    if (n_blocks <= 0) return true;
    if (prec == BMF_FP64) return launch_pair_t<double, double>(a, n_blocks, st);
    if (prec == BMF_FP32) return launch_pair_t<float, float>(a, n_blocks, st);
    return launch_pair_t<__nv_bfloat16, float>(a, n_blocks, st);
}

}  // namespace bmf
