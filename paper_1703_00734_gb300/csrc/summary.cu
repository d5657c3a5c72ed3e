// summary.cu -- the subset-posterior summaries beyond moment matching (Section 4.1, "PP DM"
// and "PP GMM"; Section 5.1) and the component choice of a propagated mixture prior.
//
//   * summary_kernel: one warp per row clusters the row's retained samples by lambda-means and
//     fits Gaussians to the largest clusters (dominant mode: the largest one; mixture: the C
//     largest with at least K + 1 samples, weighted by their sizes; a row without such a
//     cluster falls back to one Gaussian over all samples), then the mixture's pooled mean and
//     covariance, which Eq. 14 aggregates (Section 4.2).
//   * mix_choose_kernel: one thread per row picks, before each draw, the component with the
//     largest responsibility pi_c N(x; mu_c, Lambda_c^{-1}) at the row's current value and
//     installs it as the row's prior.
//
// lambda-means follows one fixed procedure (the paper names the method without its details):
// one cluster centred on the first sample; each round visits the samples in order and gives
// each to the nearest centre (lowest index on ties) unless every squared distance exceeds
// lambda, in which case it opens a new cluster centred on itself; then centres move to the
// means of their samples and empty clusters are dropped (renumbered in order); rounds repeat
// until no assignment changes (at most 100).  The warp scores the samples in parallel against
// the existing centres, then walks the samples in order to open new clusters, updating the
// later samples' nearest centre after each opening: the same assignments as the sequential
// visit.  Every sum runs over the samples in order with separate multiplies and adds, so
// assignments and fits do not depend on the launch shape.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace bmf {

namespace {

constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Squared distance of two K-vectors, summed in order.
__device__ double sqdist(const double *p, const double *c, int K)
{
    double d = 0.0;
    for (int k = 0; k < K; ++k) {
        const double e = dsub(p[k], c[k]);
        d = dadd(d, dmul(e, e));
    }
    return d;
}

// Lower Cholesky factor of the K x K row-major matrix A into L (warp; lane i computes row i
// below the pivot, each entry summed in order); false if a pivot is not > 0.
__device__ bool warp_chol(const double *A, double *L, int K, int lane)
{
    for (int e = lane; e < K * K; e += 32) L[e] = 0.0;
    __syncwarp();
    for (int j = 0; j < K; ++j) {
        double d = 0.0;
        if (lane == 0) {
            double s = A[j * K + j];
            for (int k = 0; k < j; ++k) s = dsub(s, dmul(L[j * K + k], L[j * K + k]));
            d = s > 0.0 ? sqrt(s) : -1.0;
            if (s > 0.0) L[j * K + j] = d;
        }
        d = __shfl_sync(kAll, d, 0);
        if (!(d > 0.0)) return false;
        __syncwarp();
        for (int i = j + 1 + lane; i < K; i += 32) {
            double t = A[i * K + j];
            for (int k = 0; k < j; ++k) t = dsub(t, dmul(L[i * K + k], L[j * K + k]));
            L[i * K + j] = t / d;
        }
        __syncwarp();
    }
    return true;
}

// Inverse of the SPD matrix A (K x K) into Ainv from its Cholesky factor L: lane j solves
// L L^T x = e_j (forward then back substitution, in order), then the two triangles are
// averaged.  col: K * 32 scratch (a column per lane).
__device__ bool warp_spd_inverse(const double *A, double *Ainv, double *L, double *col, int K,
                                 int lane)
{
    if (!warp_chol(A, L, K, lane)) return false;
    for (int j = lane; j < K; j += 32) {
        double *y = col + (size_t)lane * K;
        for (int i = 0; i < K; ++i) y[i] = i == j ? 1.0 : 0.0;
        for (int i = 0; i < K; ++i) {
            double t = y[i];
            for (int k = 0; k < i; ++k) t = dsub(t, dmul(L[i * K + k], y[k]));
            y[i] = t / L[i * K + i];
        }
        for (int i = K - 1; i >= 0; --i) {
            double t = y[i];
            for (int k = i + 1; k < K; ++k) t = dsub(t, dmul(L[k * K + i], y[k]));
            y[i] = t / L[i * K + i];
        }
        for (int i = 0; i < K; ++i) Ainv[i * K + j] = y[i];
    }
    __syncwarp();
    for (int e = lane; e < K * K; e += 32) {
        const int i = e / K, j = e % K;
        if (j < i) {
            const double m = dmul(0.5, dadd(Ainv[i * K + j], Ainv[j * K + i]));
            Ainv[i * K + j] = m;
            Ainv[j * K + i] = m;
        }
    }
    __syncwarp();
    return true;
}

}  // namespace

// Shared memory of one row (one warp): samples, centres (at most 2S + 1), per-sample state and
// the fit workspace (which reuses the centre area after the clustering): component means and
// precisions, four K x K work matrices, a column per lane and the pooled mean.
__host__ __device__ static size_t fit_doubles(int K)
{
    return (size_t)kMaxComponents * K + (size_t)kMaxComponents * K * K + (size_t)4 * K * K +
           (size_t)32 * K + K;
}

size_t summary_smem(int K, int S)
{
    const size_t cen = (size_t)(2 * S + 1) * K;
    const size_t fit = fit_doubles(K);
    return ((size_t)S * K + (cen > fit ? cen : fit) + S) * sizeof(double) +
           (size_t)(3 * S + 2 * (2 * S + 1) + 4) * sizeof(int);
}

__global__ void __launch_bounds__(32) summary_kernel(SummaryParams p)
{
    extern __shared__ double sh[];
    const int lane = threadIdx.x;
    const int64_t row = blockIdx.x;
    const int K = p.K, S = p.S, C = p.C;
    const size_t cen_n = (size_t)(2 * S + 1) * K, fit_n = fit_doubles(K);
    double *X = sh;                                   // [S][K]
    double *cen = X + (size_t)S * K;                  // [2S+1][K] (clustering), fit area after
    double *dbest = cen + (cen_n > fit_n ? cen_n : fit_n);   // [S]
    int *assign = reinterpret_cast<int *>(dbest + S);        // [S]
    int *prev = assign + S;                                  // [S]
    int *best = prev + S;                                    // [S]
    int *cnt = best + S;                                     // [2S+1]
    int *map = cnt + 2 * S + 1;                              // [2S+1]
    int *misc = map + 2 * S + 1;                             // [4]
    for (int e = lane; e < S * K; e += 32) {
        const int s = e / K, k = e % K;
        X[e] = p.samples[(int64_t)s * p.sample_stride + (p.row0 + row) * K + k];
    }
    __syncwarp();
    // ---- lambda-means ---------------------------------------------------------------------
    int n = 0;
    if (p.mode != 0 && S > 0) {
        n = 1;
        for (int k = lane; k < K; k += 32) cen[k] = X[k];
        for (int i = lane; i < S; i += 32) prev[i] = -1;
        __syncwarp();
        for (int it = 0; it < 100; ++it) {
            // nearest existing centre of every sample (lowest index on ties)
            for (int i = lane; i < S; i += 32) {
                int b = 0;
                double db = INFINITY;
                for (int c = 0; c < n; ++c) {
                    const double d = sqdist(X + (size_t)i * K, cen + (size_t)c * K, K);
                    if (d < db) {
                        db = d;
                        b = c;
                    }
                }
                best[i] = b;
                dbest[i] = db;
            }
            __syncwarp();
            // samples in order: the next one farther than lambda from every centre opens a
            // cluster; the later samples then compare with the new centre too
            int pos = 0;
            while (pos < S) {
                int found = S;
                for (int base = pos; base < S && found == S; base += 32) {
                    const int i = base + lane;
                    const unsigned v = __ballot_sync(kAll, i < S && dbest[i] > p.lambda);
                    if (v) found = base + __ffs(v) - 1;
                }
                if (found == S) break;
                const int c = n++;
                for (int k = lane; k < K; k += 32) cen[(size_t)c * K + k] = X[(size_t)found * K + k];
                if (lane == 0) best[found] = c;
                __syncwarp();
                for (int j = found + 1 + lane; j < S; j += 32) {
                    const double d = sqdist(X + (size_t)j * K, cen + (size_t)c * K, K);
                    if (d < dbest[j]) {
                        dbest[j] = d;
                        best[j] = c;
                    }
                }
                __syncwarp();
                pos = found + 1;
            }
            for (int i = lane; i < S; i += 32) assign[i] = best[i];
            for (int c = lane; c < n; c += 32) cnt[c] = 0;
            __syncwarp();
            for (int i = lane; i < S; i += 32) atomicAdd(&cnt[assign[i]], 1);
            __syncwarp();
            if (lane == 0) {
                int m = 0;
                for (int c = 0; c < n; ++c) map[c] = cnt[c] > 0 ? m++ : -1;
                misc[0] = m;
            }
            __syncwarp();
            // centres to the means of their samples (in order), compacted in place: the new
            // index never exceeds the old one and the sums read only the samples
            for (int e = lane; e < n * K; e += 32) {
                const int c = e / K, k = e % K;
                if (map[c] < 0) continue;
                double s = 0.0;
                for (int i = 0; i < S; ++i)
                    if (assign[i] == c) s = dadd(s, X[(size_t)i * K + k]);
                cen[(size_t)map[c] * K + k] = s / (double)cnt[c];
            }
            __syncwarp();
            n = misc[0];
            int changed = 0;
            for (int i = lane; i < S; i += 32) {
                const int a = map[assign[i]];
                assign[i] = a;
                changed |= a != prev[i];
                prev[i] = a;
            }
            __syncwarp();
            if (!__any_sync(kAll, changed)) break;
        }
    }
    // cluster sizes under the final numbering
    if (p.mode != 0 && S > 0) {
        __syncwarp();
        for (int c = lane; c < n; c += 32) cnt[c] = 0;
        __syncwarp();
        for (int i = lane; i < S; i += 32) atomicAdd(&cnt[assign[i]], 1);
        __syncwarp();
    }
    if (p.assign)
        for (int i = lane; i < S; i += 32) p.assign[row * S + i] = p.mode != 0 ? assign[i] : 0;
    // ---- fits -----------------------------------------------------------------------------
    double *fmu = cen;                       // [C][K] component means
    double *cL = fmu + (size_t)kMaxComponents * K;    // [C][K][K] component precisions
    double *Sig = cL + (size_t)kMaxComponents * K * K;   // [K][K]
    double *Lw = Sig + (size_t)K * K;        // [K][K]
    double *Lam = Lw + (size_t)K * K;        // [K][K] current component precision
    double *Acc = Lam + (size_t)K * K;       // [K][K] pooled covariance
    double *col = Acc + (size_t)K * K;       // [32][K]
    double *pm = col + (size_t)32 * K;       // [K] pooled mean
    // the chosen clusters, largest first (ties: lowest index), written by lane 0
    int *chosen = best;                      // [C] cluster ids, -1 unused
    int *sizes = cnt;
    int used = 0;
    __syncwarp();
    if (lane == 0) {
        if (p.mode != 0) {
            const int want = p.mode == 1 ? 1 : C;
            for (int t = 0; t < want; ++t) {
                int b = -1;
                for (int c = 0; c < n; ++c)
                    if (sizes[c] >= 0 && (b < 0 || sizes[c] > sizes[b])) b = c;
                if (b < 0) break;
                const int sz = sizes[b];
                sizes[b] = -1;
                if (sz < K + 1) continue;
                chosen[used] = b;
                map[used] = sz;              // component size
                ++used;
            }
        }
        misc[1] = used;
    }
    __syncwarp();
    used = misc[1];
    // Gaussian of the samples of cluster cl (all samples when cl < 0): mean into m, precision
    // (inverse of the 1/n covariance) into Lam; false when fewer than K + 1 samples or singular
    auto fit = [&](int cl, double *m) -> bool {
        int nn = 0;
        for (int i = 0; i < S; ++i) nn += (cl < 0 || assign[i] == cl);
        if (nn < K + 1) return false;
        for (int k = lane; k < K; k += 32) {
            double s = 0.0;
            for (int i = 0; i < S; ++i)
                if (cl < 0 || assign[i] == cl) s = dadd(s, X[(size_t)i * K + k]);
            m[k] = s / (double)nn;
        }
        __syncwarp();
        for (int e = lane; e < K * K; e += 32) {
            const int a = e / K, b = e % K;
            double s = 0.0;
            for (int i = 0; i < S; ++i)
                if (cl < 0 || assign[i] == cl)
                    s = dadd(s, dmul(dsub(X[(size_t)i * K + a], m[a]), dsub(X[(size_t)i * K + b], m[b])));
            Sig[e] = s / (double)nn;
        }
        __syncwarp();
        return warp_spd_inverse(Sig, Lam, Lw, col, K, lane);
    };
    double wts[kMaxComponents] = {0.0, 0.0, 0.0, 0.0};
    int got = 0;
    bool bad = false;
    for (int t = 0; t < used; ++t) {
        const int cl = chosen[t];
        const int sz = map[t];
        __syncwarp();
        if (!fit(cl, fmu + (size_t)got * K)) continue;
        // keep this component's precision for the outputs
        for (int e = lane; e < K * K; e += 32) cL[(size_t)got * K * K + e] = Lam[e];
        wts[got] = (double)sz;
        ++got;
    }
    if (got == 0) {
        // moment matching over all samples
        __syncwarp();
        if (!fit(-1, fmu)) {
            bad = true;
        } else {
            for (int e = lane; e < K * K; e += 32) cL[e] = Lam[e];
            wts[0] = 1.0;
            got = 1;
        }
    }
    if (bad) {
        if (lane == 0) {
            atomicOr(&p.err->flags, ERR_NOT_PD);
            atomicMin(&p.err->first_bad_row, (int)(p.row0 + row));
        }
        return;
    }
    double tot = 0.0;
    for (int c = 0; c < got; ++c) tot = dadd(tot, wts[c]);
    for (int c = 0; c < got; ++c) wts[c] = wts[c] / tot;
    __syncwarp();
    // pooled mean and covariance: sum_c pi_c (Lambda_c^{-1} + (mu_c - m)(mu_c - m)^T)
    for (int k = lane; k < K; k += 32) {
        double s = 0.0;
        for (int c = 0; c < got; ++c) s = dadd(s, dmul(wts[c], fmu[(size_t)c * K + k]));
        pm[k] = s;
    }
    for (int e = lane; e < K * K; e += 32) Acc[e] = 0.0;
    __syncwarp();
    for (int c = 0; c < got; ++c) {
        const double *Lc = cL + (size_t)c * K * K;
        for (int e = lane; e < K * K; e += 32) Sig[e] = Lc[e];
        __syncwarp();
        if (!warp_spd_inverse(Sig, Lam, Lw, col, K, lane)) {
            bad = true;
            break;
        }
        const double *mc = fmu + (size_t)c * K;
        for (int e = lane; e < K * K; e += 32) {
            const int a = e / K, b = e % K;
            Acc[e] = dadd(Acc[e], dmul(wts[c], dadd(Lam[e], dmul(dsub(mc[a], pm[a]), dsub(mc[b], pm[b])))));
        }
        __syncwarp();
    }
    if (!bad) bad = !warp_spd_inverse(Acc, Sig, Lw, col, K, lane);   // pooled precision in Sig
    if (bad) {
        if (lane == 0) {
            atomicOr(&p.err->flags, ERR_NOT_PD);
            atomicMin(&p.err->first_bad_row, (int)(p.row0 + row));
        }
        return;
    }
    // ---- outputs --------------------------------------------------------------------------
    const int64_t KK = (int64_t)K * K;
    if (p.pi) {
        for (int c = lane; c < C; c += 32) p.pi[row * C + c] = c < got ? wts[c] : 0.0;
        for (int e = lane; e < C * K; e += 32) {
            const int c = e / K;
            p.mu[row * C * K + e] = c < got ? fmu[e] : 0.0;
        }
        for (int64_t e = lane; e < C * KK; e += 32) {
            const int c = (int)(e / KK);
            p.Lam[row * C * KK + e] = c < got ? cL[(size_t)c * KK + (e % KK)] : 0.0;
        }
        for (int k = lane; k < K; k += 32) p.pooled_mu[row * K + k] = pm[k];
        for (int e = lane; e < KK; e += 32) p.pooled_Lam[row * KK + e] = Sig[e];
    }
    if (p.mm_mu) {
        // the summary the library propagates and aggregates: the dominant component (mode 1)
        // or the pooled moments (mode 2), as mean, packed precision and precision x mean
        const int64_t ar = p.row0 + row;
        const double *sm = p.mode == 1 ? fmu : pm;
        const double *sL = p.mode == 1 ? cL : Sig;
        for (int k = lane; k < K; k += 32) p.mm_mu[ar * K + k] = sm[k];
        for (int e = lane; e < K * (K + 1) / 2; e += 32) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            const int j = e - i * (i + 1) / 2;
            p.mm_L[(int64_t)e * p.R + ar] = sL[i * K + j];
        }
        for (int i = lane; i < K; i += 32) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc = fma(sL[i * K + k], sm[k], acc);
            p.mm_b[(int64_t)i * p.R + ar] = acc;
        }
        if (p.mix) {
            // mixture store of the row: per component [log pi + log det(Lambda)/2][mu][L packed]
            // [Lambda mu]; unused components get a -infinity score
            const int NT = K * (K + 1) / 2, W = 1 + 2 * K + NT;
            double *mx = p.mix + ar * (int64_t)C * W;
            for (int c = 0; c < C; ++c) {
                double *o = mx + (int64_t)c * W;
                if (c >= got) {
                    if (lane == 0) o[0] = -INFINITY;
                    continue;
                }
                const double *Lc = cL + (size_t)c * KK;
                const double *mc = fmu + (size_t)c * K;
                __syncwarp();
                const bool okc = warp_chol(Lc, Lw, K, lane);
                if (lane == 0) {
                    double logdet = 0.0;
                    for (int k = 0; k < K; ++k) logdet += 2.0 * log(Lw[k * K + k]);
                    o[0] = okc ? log(wts[c]) + 0.5 * logdet : -INFINITY;
                }
                for (int k = lane; k < K; k += 32) o[1 + k] = mc[k];
                for (int e = lane; e < NT; e += 32) {
                    int i = 0;
                    while ((i + 1) * (i + 2) / 2 <= e) ++i;
                    const int j = e - i * (i + 1) / 2;
                    o[1 + K + e] = Lc[i * K + j];
                }
                for (int i = lane; i < K; i += 32) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k) acc = fma(Lc[i * K + k], mc[k], acc);
                    o[1 + K + NT + i] = acc;
                }
            }
        }
    }
}

void launch_summary(const SummaryParams &p, cudaStream_t st)
{
    if (p.n_rows <= 0) return;
    const size_t smem = summary_smem(p.K, p.S);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(summary_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    summary_kernel<<<(unsigned)p.n_rows, 32, smem, st>>>(p);
}

// ------------------------------------------------------------------------------------------
// Component choice of a mixture prior: score_c = log pi_c + log det(Lambda_c)/2
// - (x - mu_c)^T Lambda_c (x - mu_c) / 2 at the row's current x (the quadratic form summed in
// order, separate multiplies and adds); the best (lowest index on ties) becomes the prior.
// ------------------------------------------------------------------------------------------
__global__ void mix_choose_kernel(MixChooseParams p)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= p.n) return;
    const int64_t r = p.r0 + q;
    if (!p.has_mix[r]) return;
    const int K = p.K, C = p.C, NT = K * (K + 1) / 2, W = 1 + 2 * K + NT;
    const double *mx = p.mix + r * (int64_t)C * W;
    const double *x = p.X + r * K;
    int bestc = -1;
    double sbest = -INFINITY;
    for (int c = 0; c < C; ++c) {
        const double *o = mx + (int64_t)c * W;
        if (!(o[0] > -INFINITY)) continue;
        const double *m = o + 1, *L = o + 1 + K;
        double qf = 0.0;
        for (int a = 0; a < K; ++a) {
            double s = 0.0;
            for (int b = 0; b < K; ++b)
                s = dadd(s, dmul(L[a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a], dsub(x[b], m[b])));
            qf = dadd(qf, dmul(dsub(x[a], m[a]), s));
        }
        const double score = o[0] - 0.5 * qf;
        if (bestc < 0 || score > sbest) {
            bestc = c;
            sbest = score;
        }
    }
    if (bestc < 0) {
        atomicOr(&p.err->flags, ERR_NOT_PD);
        atomicMin(&p.err->first_bad_row, (int)r);
        return;
    }
    const double *o = mx + (int64_t)bestc * W;
    for (int e = 0; e < NT; ++e) p.pL[(int64_t)e * p.R + r] = o[1 + K + e];
    for (int i = 0; i < K; ++i) p.pb[(int64_t)i * p.R + r] = o[1 + K + NT + i];
    if (p.chosen) p.chosen[r] = bestc;
}

void launch_mix_choose(const MixChooseParams &p, cudaStream_t st)
{
    if (p.n <= 0) return;
    mix_choose_kernel<<<(unsigned)((p.n + 127) / 128), 128, 0, st>>>(p);
}

}  // namespace bmf
