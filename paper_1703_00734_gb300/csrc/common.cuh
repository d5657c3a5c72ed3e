// common.cuh -- internal definitions shared by the library's kernels and its runtime.
// Not part of the public ABI (include/bmf.h is).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "bmf.h"

namespace bmf {

constexpr int kWarp = 32;

// Packed lower-triangular index of (i, j), i >= j, row by row.
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }
__host__ __device__ constexpr int ntri(int K) { return K * (K + 1) / 2; }
// Gram partial of one work item: the K(K+1)/2 packed-lower entries of sum p p^T followed by
// the K entries of sum y p, padded to a multiple of 32 (the warp reduce-scatter width).
__host__ __device__ constexpr int gram_nv(int K) { return ntri(K) + K; }
__host__ __device__ constexpr int gram_ld(int K) { return (gram_nv(K) + 31) / 32 * 32; }
// Hyperparameter draw block: chi2[K], K(K-1)/2 normals, z_mu[K].
__host__ __device__ constexpr int hyper_len(int K) { return K + K * (K - 1) / 2 + K; }

// A work item of the Gram-gather pass: `count` consecutive observations of arena row `row`
// starting at position `begin` of the observation lists.
struct GramItem {
    int64_t begin;
    int32_t count;
    int32_t row;
};

// A warp task of the Gram-gather pass: items item0 .. item0 + n - 1, one per group of G lanes
// (G = 32 with n = 1 for long rows and row chunks; G = 16 or 8 with n = 32 / G short rows).
struct GramTask {
    int64_t item0;
    int32_t n;
    int32_t G;
};

// Device error word bits (set by kernels, read by the host at sync points).
enum : uint32_t {
    ERR_NOT_PD = 1u << 0,
    ERR_NONFINITE = 1u << 1,
    ERR_TIMEOUT = 1u << 2,
    ERR_ARG = 1u << 3,
    ERR_RNG = 1u << 4,      // chi-square rejection limit of the device generator
};

struct DevError {
    uint32_t flags;
    int32_t first_bad_row;  // arena row of the first non-PD conditional (atomicMin)
};

// Hyperparameters of one (subset, factor): mu[K], Lambda packed lower, b = Lambda mu.
// Laid out contiguously per slot: [mu (K)][Lambda (ntri)][b (K)].
__host__ __device__ constexpr int hyper_slot_len(int K) { return K + ntri(K) + K; }

// FP32 -> FP64 by rebuilding the IEEE-754 fields on the integer pipe, without a branch: exact
// for every normal float, zero, infinity and NaN; a subnormal float (below 1.2e-38 in
// magnitude) reads as a zero of its sign.  On this GPU the conversion instruction occupies the
// FP64 pipe, which the conditional draw is bound by, and a branch to it would still issue a
// predicated conversion for the whole warp.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t s = u & 0x80000000u, t = u & 0x7f800000u;
    // exponent rebased from 127 to 1023: + (1023 - 127) << 20 in the high word
    uint32_t hi = s + ((u & 0x7fffffffu) >> 3) + 0x38000000u;
    hi = t == 0u ? s : (t == 0x7f800000u ? hi + 0x38000000u : hi);
    const uint32_t lo = t == 0u ? 0u : u << 29;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double widen(double d) { return d; }

// A pivot the FP64 Cholesky of the conditional draw can take: positive, finite and normal (a
// pivot below the smallest normal double, 2.2e-308, leaves the row numerically singular and
// counts as not positive definite).  Integer compares of the bit pattern.
__device__ __forceinline__ bool pivot_ok(double d)
{
    const long long b = __double_as_longlong(d);
    return b >= 0x0010000000000000ll && b < 0x7ff0000000000000ll;
}

// 1 / sqrt(d) for a pivot of the FP64 Cholesky in the reduced-precision modes (FP32 or BF16
// Gram entries, relative error ~1e-7 already); d must pass pivot_ok.  With d = m 2^E, m in
// [1, 2) and E = 2h + p (p in {0, 1}): the FP32 unit gives 1/sqrt(m 2^p) for a float built from
// d's top mantissa bits (relative error below 2^-21 with the truncation), widened and scaled by
// 2^-h on the integer pipe, then one Newton step in FP64, y <- y + (y / 2)(1 - d y^2) (y / 2 by
// the exponent too): relative error below 1e-12 with three FP64 operations and no branch.
__device__ __forceinline__ double rsqrt_refined(double d)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int E = (int)(u >> 52) - 1023;
    const int p = E & 1, h = (E - p) / 2;
    const uint32_t fb = ((uint32_t)(127 + p) << 23) | (uint32_t)((u >> 29) & 0x7fffffull);
    const uint32_t yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));   // in (0.5, 1]
    const int hi = (int)(((yb & 0x7fffffffu) >> 3) + 0x38000000u);
    const int lo = (int)(yb << 29);
    const double y = __hiloint2double(hi - h * (1 << 20), lo);
    const double y2 = __hiloint2double(hi - (h + 1) * (1 << 20), lo);
    const double r = fma(-(d * y), y, 1.0);
    return fma(y2, r, y);
}

// Pivot reciprocal square root of the conditional draw: full FP64 in the FP64 mode (gathered
// type double), refined FP32 otherwise.
template <typename GT>
__device__ __forceinline__ double pivot_rsqrt(double d)
{
    if constexpr (sizeof(GT) == 8)
        return rsqrt(d);
    else
        return rsqrt_refined(d);
}

}  // namespace bmf
