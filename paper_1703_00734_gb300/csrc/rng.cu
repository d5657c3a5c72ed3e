// rng.cu -- the device generator of the Gibbs sweep's random numbers.
//
// Counter-based: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11) with key (seed, 0) and counter (index, t, tag, attempt), t the 1-based
// sweep number of the subset's chain and tag = subset id * 256 + factor * 16 + kind.  Every
// number is a pure function of its position, so the draws do not depend on batching, on the
// launch shape or on how sweeps are split across calls.
//   kind 2 (hyperparameter normals) and kind 3 (z of the rows): element e of the stream comes
//     from call e / 4; words (0, 1) give elements 4q, 4q + 1 and words (2, 3) elements
//     4q + 2, 4q + 3 by Box-Muller (cosine, sine), u1 = (top 53 bits + 1) 2^-53 in (0, 1] and
//     u2 = top 53 bits 2^-53 in [0, 1);
//   kind 1 (chi-square, dof nu0 + n - k for diagonal entry k): 2 Gamma(dof / 2) by Marsaglia &
//     Tsang (ACM TOMS 2000), attempt j on counter (k, t, tag, j): a candidate from the
//     cosine normal of words (0, 1), the acceptance uniform from word 2 and, for shape < 1,
//     the U^(1/a) boost from word 3.  64 rejections in a row set an error flag;
//   kind 4 (chi-square of a sampled noise precision, factor W): variate k drawn the same way
//     with dof 2 a0 + the entries of column k of the subset (one precision per column) or
//     2 a0 + the subset's entries (one precision per subset, k = 0).
// One thread per Philox call (normal streams) or per variate (chi-square).
#include "common.cuh"
#include "kernels.h"

namespace bmf {

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
        const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
        const uint64_t n0 = hi1 ^ x[1] ^ k0, n2 = hi0 ^ x[3] ^ k1;
        x[0] = n0;
        x[1] = lo1;
        x[2] = n2;
        x[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

__device__ __forceinline__ double u_closed0(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double u_open0(uint64_t w) { return (double)((w >> 11) + 1) * 0x1.0p-53; }

__device__ __forceinline__ void box_muller(uint64_t a, uint64_t b, double &z0, double &z1)
{
    const double r = sqrt(-2.0 * log(u_open0(a)));
    double s, c;
    sincos(6.283185307179586 * u_closed0(b), &s, &c);
    z0 = r * c;
    z1 = r * s;
}

__global__ void __launch_bounds__(256) gen_kernel(GenParams p)
{
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= p.n_units) return;
    int lo = 0, hi = p.n_segs - 1;           // last segment with unit0 <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.segs[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    const GenSeg sg = p.segs[lo];
    const int64_t l = u - sg.unit0;
    double *out = p.out + sg.out;
    if (sg.kind == 1 || sg.kind == 4) {
        // kind 1: the Bartlett diagonal, dof0 - k; kind 4: the noise precision of a column
        // (dof0 + its entries) or of a subset (dof0)
        const double dof = sg.kind == 1 ? sg.dof0 - (double)l
                                        : sg.dof0 + (sg.row0 >= 0
                                                         ? (double)(p.cnt_ptr[sg.row0 + l + 1] -
                                                                    p.cnt_ptr[sg.row0 + l])
                                                         : 0.0);
        const double a = 0.5 * dof;
        const bool boost = a < 1.0;
        const double d = (boost ? a + 1.0 : a) - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
        double res = __longlong_as_double(0x7ff8000000000000ll);
        bool ok = false;
        for (int j = 0; j < 64 && dof > 0.0; ++j) {
            uint64_t w[4] = {(uint64_t)l, (uint64_t)p.t, sg.tag, (uint64_t)j};
            philox4x64_10(w, p.seed, 0);
            double x, unused;
            box_muller(w[0], w[1], x, unused);
            double v = 1.0 + c * x;
            if (!(v > 0.0)) continue;
            v = v * v * v;
            const double uu = u_open0(w[2]);
            if (uu < 1.0 - 0.0331 * (x * x) * (x * x) ||
                log(uu) < 0.5 * x * x + d * (1.0 - v + log(v))) {
                double g = d * v;
                if (boost) g *= pow(u_open0(w[3]), 1.0 / a);
                res = 2.0 * g;
                ok = true;
                break;
            }
        }
        if (!ok) atomicOr(&p.err->flags, ERR_RNG);
        out[l] = res;
        return;
    }
    uint64_t w[4] = {(uint64_t)l, (uint64_t)p.t, sg.tag, 0};
    philox4x64_10(w, p.seed, 0);
    double z[4];
    box_muller(w[0], w[1], z[0], z[1]);
    box_muller(w[2], w[3], z[2], z[3]);
    const int64_t e0 = 4 * l;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (e0 + q < sg.count) out[e0 + q] = z[q];
}

void launch_gen(const GenParams &p, cudaStream_t st)
{
    if (p.n_units <= 0) return;
    gen_kernel<<<(unsigned)((p.n_units + 255) / 256), 256, 0, st>>>(p);
}

// Host side: the segments of one sweep's draw buffer for a batch (layout of the public header).
int64_t gen_segments(const std::vector<GenSubset> &subs, int K, double nu0, int noise, double a0,
                     std::vector<GenSeg> &segs)
{
    segs.clear();
    const int64_t HN = (int64_t)K * (K - 1) / 2 + K;
    int64_t unit = 0, off = 0;
    auto add = [&](int kind, int64_t count, uint64_t tag, double dof0, int64_t row0 = -1) {
        if (count <= 0) return;
        GenSeg s;
        s.unit0 = unit;
        s.count = count;
        s.out = off;
        s.tag = tag;
        s.dof0 = dof0;
        s.kind = kind;
        s.row0 = row0;
        segs.push_back(s);
        unit += (kind == 1 || kind == 4) ? count : (count + 3) / 4;
        off += count;
    };
    auto tag = [](int sid, int f, int kind) {
        return ((uint64_t)(uint32_t)sid << 8) | ((uint64_t)f << 4) | (uint64_t)kind;
    };
    for (const GenSubset &s : subs)
        for (int f = 0; f < 2; ++f) {
            const int64_t m = f == 0 ? s.n : s.d;
            add(1, K, tag(s.sid, f, 1), nu0 + (double)m);
            add(2, HN, tag(s.sid, f, 2), 0.0);
        }
    for (int f = 0; f < 2; ++f)
        for (const GenSubset &s : subs) add(3, (f == 0 ? s.n : s.d) * K, tag(s.sid, f, 3), 0.0);
    // noise precisions: one chi-square per column (dof 2 a0 + the column's entries) or one per
    // subset (dof 2 a0 + its entries), stream (subset, W, kind 4)
    if (noise == 2)
        for (const GenSubset &s : subs) add(4, s.d, tag(s.sid, 1, 4), 2.0 * a0, s.woff);
    else if (noise == 1)
        for (const GenSubset &s : subs) add(4, 1, tag(s.sid, 1, 4), 2.0 * a0 + (double)s.nnz, -1);
    return unit;
}

}  // namespace bmf
