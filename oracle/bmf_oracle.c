/*
 * bmf_oracle.c -- the ORACLE: a plain, slow, FP64 CPU restatement of the BPMF Gibbs sweep
 * and of the posterior-propagation (PP) approximation and aggregation steps of
 * Qin et al., "Distributed Bayesian Matrix Factorization with Limited Communication"
 * (arXiv 1703.00734).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA library; the library never loads it.
 *
 * Everything is written out from the definitions, in the order the method states them,
 * with sequential loops and no blocking or reordering:
 *   - model: Gaussian likelihood on observed entries with noise precision tau (Eqs. 2-3),
 *     Gaussian row priors (Eqs. 4a/4b), Normal-Wishart hyperpriors (Section 5.1);
 *   - Gibbs conditionals: the textbook conjugate updates of BPMF (Salakhutdinov & Mnih 2008,
 *     cited in Section 5.1), with the centred scatter matrix of the Section 5.1 footnote;
 *   - moment matching (Section 4.1) and the eigenvalue-corrected aggregation of
 *     Algorithm 2 / Eq. 14 (Section 4.2).
 *
 * Conventions fixed here (the paper is silent on them; the CUDA library follows the same
 * conventions, stated in its public header):
 *   - a Gaussian with precision P is drawn as mu + L^{-T} z with P = L L^T (lower, positive
 *     diagonal Cholesky) and z standard normal;
 *   - Wishart(W, nu) is drawn by the Bartlett decomposition on the lower Cholesky factor L of
 *     W: Lambda = (L A)(L A)^T, A lower triangular, A_kk = sqrt(chi2_k) with
 *     chi2_k ~ chi^2(nu - k) (k = 0..K-1), A_kl ~ N(0,1) for k > l;
 *   - one block of hyperparameter draws is laid out as chi2[K], then the K(K-1)/2
 *     below-diagonal normals row by row (k = 1..K-1, l = 0..k-1), then z_mu[K].
 * Matrices are dense, row-major, K x K; vectors are row-major [rows x K].
 *
 * Pinned by tests/test_oracle_*.py against closed forms, identities and brute force
 * (see the tests for which pin covers which function).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_PD 1
#define ORC_ARG 2
#define ORC_NOMEM 3

/* ------------------------------------------------------------------------------------- */
/* Dense FP64 linear algebra (textbook forms).                                           */
/* ------------------------------------------------------------------------------------- */

/* Cholesky factor of a symmetric positive definite A: A = L L^T, L lower with positive
 * diagonal (Cholesky-Crout, column by column).  Returns ORC_NOT_PD if a pivot is not > 0. */
static int chol_lower(int K, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)K * K);
    for (int j = 0; j < K; ++j) {
        double s = A[j * K + j];
        for (int k = 0; k < j; ++k) s -= L[j * K + k] * L[j * K + k];
        if (!(s > 0.0)) return ORC_NOT_PD;
        double d = sqrt(s);
        L[j * K + j] = d;
        for (int i = j + 1; i < K; ++i) {
            double t = A[i * K + j];
            for (int k = 0; k < j; ++k) t -= L[i * K + k] * L[j * K + k];
            L[i * K + j] = t / d;
        }
    }
    return ORC_OK;
}

/* Solve L y = b in place (L lower triangular). */
static void solve_lower(int K, const double *L, double *y)
{
    for (int i = 0; i < K; ++i) {
        double t = y[i];
        for (int k = 0; k < i; ++k) t -= L[i * K + k] * y[k];
        y[i] = t / L[i * K + i];
    }
}

/* Solve L^T x = y in place (L lower triangular, so L^T is upper triangular). */
static void solve_lower_t(int K, const double *L, double *x)
{
    for (int i = K - 1; i >= 0; --i) {
        double t = x[i];
        for (int k = i + 1; k < K; ++k) t -= L[k * K + i] * x[k];
        x[i] = t / L[i * K + i];
    }
}

/* Inverse of a symmetric positive definite matrix through its Cholesky factor:
 * column j of A^{-1} solves L L^T x = e_j. */
static int spd_inverse(int K, const double *A, double *Ainv, double *work /* K*K + K */)
{
    double *L = work, *col = work + (size_t)K * K;
    if (chol_lower(K, A, L)) return ORC_NOT_PD;
    for (int j = 0; j < K; ++j) {
        for (int i = 0; i < K; ++i) col[i] = (i == j) ? 1.0 : 0.0;
        solve_lower(K, L, col);
        solve_lower_t(K, L, col);
        for (int i = 0; i < K; ++i) Ainv[i * K + j] = col[i];
    }
    /* symmetrise (the two triangles agree up to rounding) */
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (Ainv[i * K + j] + Ainv[j * K + i]);
            Ainv[i * K + j] = m;
            Ainv[j * K + i] = m;
        }
    return ORC_OK;
}

/* Smallest eigenvalue of a symmetric matrix by the cyclic Jacobi method
 * (Golub & Van Loan, "Matrix Computations", Section 8.5): rotate away each off-diagonal
 * entry in turn until the off-diagonal mass is negligible; the diagonal then holds the
 * eigenvalues. */
static double jacobi_min_eig(int K, const double *M, double *a /* K*K work */)
{
    memcpy(a, M, sizeof(double) * (size_t)K * K);
    double fro = 0.0;
    for (int i = 0; i < K * K; ++i) fro += a[i] * a[i];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) off += a[p * K + q] * a[p * K + q];
        if (off <= 1e-30 * fro || off == 0.0) break;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                double apq = a[p * K + q];
                if (apq == 0.0) continue;
                double theta = (a[q * K + q] - a[p * K + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < K; ++k) {
                    double akp = a[k * K + p], akq = a[k * K + q];
                    a[k * K + p] = c * akp - s * akq;
                    a[k * K + q] = s * akp + c * akq;
                }
                for (int k = 0; k < K; ++k) {
                    double apk = a[p * K + k], aqk = a[q * K + k];
                    a[p * K + k] = c * apk - s * aqk;
                    a[q * K + k] = s * apk + c * aqk;
                }
            }
    }
    double m = a[0];
    for (int i = 1; i < K; ++i)
        if (a[i * K + i] < m) m = a[i * K + i];
    return m;
}

/* ------------------------------------------------------------------------------------- */
/* Normal-Wishart hyperparameter update (Section 5.1 and its footnote).                  */
/* ------------------------------------------------------------------------------------- */

/* Posterior parameters of (mu, Lambda) given the N rows of X under the Normal-Wishart
 * prior (mu0, beta0, nu0, W0):
 *   xbar = (1/N) sum_i x_i,   Sbar = (1/N) sum_i (x_i - xbar)(x_i - xbar)^T   (centred,
 *   as the Section 5.1 footnote corrects),
 *   beta* = beta0 + N, nu* = nu0 + N, mu* = (beta0 mu0 + N xbar) / beta*,
 *   [W*]^{-1} = W0^{-1} + N Sbar + (beta0 N / beta*) (mu0 - xbar)(mu0 - xbar)^T.
 * With N = 0 the posterior equals the prior. */
int orc_nw_posterior(int K, int64_t N, const double *X, const double *mu0, double beta0, double nu0,
                     const double *W0, double *xbar, double *Sbar, double *mu_star, double *beta_star,
                     double *nu_star, double *Wstar_inv)
{
    double *work = (double *)malloc(sizeof(double) * ((size_t)2 * K * K + K));
    if (!work) return ORC_NOMEM;
    for (int k = 0; k < K; ++k) xbar[k] = 0.0;
    for (int a = 0; a < K * K; ++a) Sbar[a] = 0.0;
    if (N > 0) {
        for (int64_t i = 0; i < N; ++i)
            for (int k = 0; k < K; ++k) xbar[k] += X[i * K + k];
        for (int k = 0; k < K; ++k) xbar[k] /= (double)N;
        for (int64_t i = 0; i < N; ++i)
            for (int a = 0; a < K; ++a)
                for (int b = 0; b < K; ++b)
                    Sbar[a * K + b] += (X[i * K + a] - xbar[a]) * (X[i * K + b] - xbar[b]);
        for (int a = 0; a < K * K; ++a) Sbar[a] /= (double)N;
    }
    double Nd = (double)N;
    *beta_star = beta0 + Nd;
    *nu_star = nu0 + Nd;
    for (int k = 0; k < K; ++k) mu_star[k] = (beta0 * mu0[k] + Nd * xbar[k]) / *beta_star;
    double *W0inv = work + (size_t)K * K + K; /* after the K*K + K scratch used by spd_inverse */
    if (spd_inverse(K, W0, W0inv, work)) {
        free(work);
        return ORC_NOT_PD;
    }
    double c = beta0 * Nd / *beta_star;
    for (int a = 0; a < K; ++a)
        for (int b = 0; b < K; ++b)
            Wstar_inv[a * K + b] = W0inv[a * K + b] + Nd * Sbar[a * K + b]
                                   + c * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b]);
    free(work);
    return ORC_OK;
}

/* One draw of (mu, Lambda) from the Normal-Wishart posterior:
 *   Lambda ~ Wishart(W*, nu*) by the Bartlett decomposition on chol(W*) (draws chi2, nrm),
 *   mu ~ N(mu*, (beta* Lambda)^{-1}) drawn as mu* + chol(beta* Lambda)^{-T} zmu. */
int orc_nw_draw(int K, const double *mu_star, double beta_star, const double *Wstar_inv,
                const double *chi2, const double *nrm, const double *zmu, double *mu_out,
                double *Lam_out)
{
    size_t KK = (size_t)K * K;
    double *w = (double *)malloc(sizeof(double) * (5 * KK + 2 * K));
    if (!w) return ORC_NOMEM;
    double *Wst = w, *L = w + KK, *A = w + 2 * KK, *B = w + 3 * KK, *work = w + 4 * KK;
    double *v = w + 5 * KK + K;
    int st = spd_inverse(K, Wstar_inv, Wst, work);
    if (!st) st = chol_lower(K, Wst, L);
    if (st) {
        free(w);
        return ORC_NOT_PD;
    }
    /* Bartlett factor A */
    memset(A, 0, sizeof(double) * KK);
    for (int k = 0; k < K; ++k) {
        A[k * K + k] = sqrt(chi2[k]);
        for (int l = 0; l < k; ++l) A[k * K + l] = nrm[(size_t)k * (k - 1) / 2 + l];
    }
    /* B = L A */
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += L[i * K + k] * A[k * K + j];
            B[i * K + j] = s;
        }
    /* Lambda = B B^T */
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += B[i * K + k] * B[j * K + k];
            Lam_out[i * K + j] = s;
        }
    /* mu = mu* + chol(beta* Lambda)^{-T} zmu */
    for (int a = 0; a < (int)KK; ++a) A[a] = beta_star * Lam_out[a];
    if (chol_lower(K, A, L)) {
        free(w);
        return ORC_NOT_PD;
    }
    for (int k = 0; k < K; ++k) v[k] = zmu[k];
    solve_lower_t(K, L, v);
    for (int k = 0; k < K; ++k) mu_out[k] = mu_star[k] + v[k];
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Row conditionals (the Gibbs update of every x_n given W; Eqs. 2-4).                   */
/* ------------------------------------------------------------------------------------- */

/* For each row r of a CSR block (ptr/idx/val; idx indexes rows of the partner matrix P):
 *   Lambda_r = Lambda_p + sum_{d in Omega_r} t_rd p_d p_d^T,
 *   b_r      = Lambda_p mu_p + sum_{d in Omega_r} t_rd y_rd p_d,
 *   x_r      = Lambda_r^{-1} b_r + L_r^{-T} z_r,   Lambda_r = L_r L_r^T,
 * with the noise precision t_rd = tau_partner[d] (per-column precisions, row side: the
 * partner is the column), tau_row[r] (column side: the row is the column), or tau (Eq. 3).
 * The prior (mu_p, Lambda_p) is shared by all rows (per_row_prior = 0: mu_p[K],
 * Lam_p[K*K]) or given per row (per_row_prior = 1: mu_p[R*K], Lam_p[R*K*K]).
 * If some Lambda_r is not positive definite, *bad_row = the first such r and ORC_NOT_PD is
 * returned (the serial build stops there).  The rows are independent given P and the draws, so
 * a build with OpenMP (the all-core timing of the oracle) splits them over threads; every row's
 * arithmetic is the same as in the serial build, whose loop compiles as if the OpenMP lines
 * were absent. */
int orc_update_rows(int K, int64_t R, const int64_t *ptr, const int32_t *idx, const double *val,
                    const double *P, double tau, const double *tau_partner, const double *tau_row,
                    int per_row_prior, const double *mu_p, const double *Lam_p, const double *z,
                    double *X_out, int64_t *bad_row)
{
    size_t KK = (size_t)K * K;
#ifdef _OPENMP
    int64_t first_bad = -1;
    int nomem = 0;
#pragma omp parallel
    {
#endif
    double *w = (double *)malloc(sizeof(double) * (2 * KK + 2 * K));
#ifdef _OPENMP
    if (!w) {
#pragma omp atomic write
        nomem = 1;
    }
#else
    if (!w) return ORC_NOMEM;
#endif
    double *A = w, *L = w + KK, *b = w + 2 * KK;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < R; ++r) {
#ifdef _OPENMP
        if (!w) continue;
#endif
        const double *mu = per_row_prior ? mu_p + r * K : mu_p;
        const double *Lam = per_row_prior ? Lam_p + r * (int64_t)KK : Lam_p;
        for (size_t a = 0; a < KK; ++a) A[a] = Lam[a];
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += Lam[i * K + j] * mu[j];
            b[i] = s;
        }
        for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) {
            const double *p = P + (int64_t)idx[e] * K;
            double y = val[e];
            /* noise precision of this observation: the partner column's (row side), the row's
             * own column's (column side), or the shared one */
            const double t = tau_partner ? tau_partner[idx[e]] : (tau_row ? tau_row[r] : tau);
            for (int i = 0; i < K; ++i) {
                for (int j = 0; j < K; ++j) A[i * K + j] += t * p[i] * p[j];
                b[i] += t * y * p[i];
            }
        }
        if (chol_lower(K, A, L)) {
#ifdef _OPENMP
#pragma omp critical(orc_bad_row)
            if (first_bad < 0 || r < first_bad) first_bad = r;
            continue;
#else
            if (bad_row) *bad_row = r;
            free(w);
            return ORC_NOT_PD;
#endif
        }
        solve_lower(K, L, b);                       /* b <- L^{-1} b            */
        for (int i = 0; i < K; ++i) b[i] += z[r * K + i]; /* + z                 */
        solve_lower_t(K, L, b);                     /* x = L^{-T}(L^{-1} b + z) */
        for (int i = 0; i < K; ++i) X_out[r * K + i] = b[i];
    }
    free(w);
#ifdef _OPENMP
    }
    if (nomem) return ORC_NOMEM;
    if (first_bad >= 0) {
        if (bad_row) *bad_row = first_bad;
        return ORC_NOT_PD;
    }
#endif
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------- */
/* One Gibbs sweep of BPMF on one data subset.                                           */
/* ------------------------------------------------------------------------------------- */

/* Order within a sweep: (mu_X, Lambda_X) | X, then (mu_W, Lambda_W) | W, then every x_n | W,
 * then every w_d | X (the new X), then (noise_mode != 0) the noise precisions | X, W
 * (orc_noise_update; tau_col [D] in/out, noise_draw its chi-square variates; noise_mode 0
 * keeps the fixed tau).  A factor whose prior is propagated from an earlier PP stage
 * (prior_x / prior_w = 1) keeps that per-row prior and draws no hyperparameters
 * (Section 5.1); otherwise its hyperparameters are drawn and shared by its rows.
 * hdraw_* = one hyperparameter draw block (chi2[K], nrm[K(K-1)/2], zmu[K]).
 * hyper_out receives mu_X[K], Lambda_X[K*K], mu_W[K], Lambda_W[K*K] (unchanged entries
 * for a propagated factor). */
/* Noise precision update after a sweep's W half (Section 2.1: per-column precisions tau_d, or
 * one precision, with conjugate Gamma(a0, b0) priors, shape-rate):
 *   mode 1 (one precision):  tau | X, W ~ Gamma(a0 + |Omega| / 2, b0 + SSE / 2),
 *   mode 2 (per column):     tau_d | X, W ~ Gamma(a0 + n_d / 2, b0 + SSE_d / 2),
 * SSE_d = sum_{n in Omega_d} (y_nd - x_n^T w_d)^2 over the column's entries in order, SSE the
 * sum of the SSE_d in column order.  A Gamma(a, b) variate is c / (2 b) with c ~ chi^2(2 a),
 * the variate given in draw[] (one per column, or one).  tau[] (D entries) receives the new
 * precisions (mode 1: the same value in every entry). */
int orc_noise_update(int K, int64_t D, const int64_t *cptr, const int32_t *cidx,
                     const double *cval, const double *X, const double *W, int mode, double a0,
                     double b0, const double *draw, double *tau)
{
    (void)a0;
    double total = 0.0;
    for (int64_t d = 0; d < D; ++d) {
        double sse = 0.0;
        for (int64_t e = cptr[d]; e < cptr[d + 1]; ++e) {
            const double *x = X + (int64_t)cidx[e] * K, *w = W + d * K;
            double pr = 0.0;
            for (int k = 0; k < K; ++k) pr += x[k] * w[k];
            const double r = cval[e] - pr;
            sse += r * r;
        }
        if (mode == 2)
            tau[d] = draw[d] / (2.0 * b0 + sse);
        else
            total += sse;
    }
    if (mode == 1) {
        const double t = draw[0] / (2.0 * b0 + total);
        for (int64_t d = 0; d < D; ++d) tau[d] = t;
    }
    return ORC_OK;
}

int orc_sweep(int K, int64_t N, int64_t D, const int64_t *rptr, const int32_t *ridx,
              const double *rval, const int64_t *cptr, const int32_t *cidx, const double *cval,
              double tau, const double *mu0, double beta0, double nu0, const double *W0,
              int prior_x, const double *muX_row, const double *LamX_row, int prior_w,
              const double *muW_row, const double *LamW_row, const double *hdraw_x,
              const double *hdraw_w, const double *zX, const double *zW, double *X, double *W,
              double *hyper_out, int noise_mode, double a0, double b0, const double *noise_draw,
              double *tau_col, int64_t *bad_row)
{
    size_t KK = (size_t)K * K;
    int st;
    double *muX = hyper_out, *LamX = hyper_out + K, *muW = hyper_out + K + KK,
           *LamW = hyper_out + 2 * K + KK;
    double *w = (double *)malloc(sizeof(double) * (3 * KK + 3 * K));
    if (!w) return ORC_NOMEM;
    double *xbar = w, *Sbar = w + K, *mus = w + K + KK, *Wsi = w + 2 * K + KK;
    double bs, ns;
    size_t nlow = (size_t)K * (K - 1) / 2;
    if (!prior_x) {
        st = orc_nw_posterior(K, N, X, mu0, beta0, nu0, W0, xbar, Sbar, mus, &bs, &ns, Wsi);
        if (!st) st = orc_nw_draw(K, mus, bs, Wsi, hdraw_x, hdraw_x + K, hdraw_x + K + nlow, muX, LamX);
        if (st) goto done;
    }
    if (!prior_w) {
        st = orc_nw_posterior(K, D, W, mu0, beta0, nu0, W0, xbar, Sbar, mus, &bs, &ns, Wsi);
        if (!st) st = orc_nw_draw(K, mus, bs, Wsi, hdraw_w, hdraw_w + K, hdraw_w + K + nlow, muW, LamW);
        if (st) goto done;
    }
    /* with sampled noise precisions the rows see their columns' current values (one shared
     * value in mode 1 is stored per column too) */
    st = orc_update_rows(K, N, rptr, ridx, rval, W, tau, noise_mode ? tau_col : NULL, NULL,
                         prior_x, prior_x ? muX_row : muX, prior_x ? LamX_row : LamX, zX, X,
                         bad_row);
    if (st) goto done;
    st = orc_update_rows(K, D, cptr, cidx, cval, X, tau, NULL, noise_mode ? tau_col : NULL,
                         prior_w, prior_w ? muW_row : muW, prior_w ? LamW_row : LamW, zW, W,
                         bad_row);
    if (st) goto done;
    if (noise_mode)
        st = orc_noise_update(K, D, cptr, cidx, cval, X, W, noise_mode, a0, b0, noise_draw, tau_col);
done:
    free(w);
    return st;
}

/* ------------------------------------------------------------------------------------- */
/* Moment matching (Section 4.1, "PP MM").                                               */
/* ------------------------------------------------------------------------------------- */

/* Running sums over retained samples: S1_r += x_r, S2_r += x_r x_r^T. */
void orc_moments_accumulate(int K, int64_t R, const double *X, double *S1, double *S2)
{
    for (int64_t r = 0; r < R; ++r) {
        const double *x = X + r * K;
        for (int i = 0; i < K; ++i) {
            S1[r * K + i] += x[i];
            for (int j = 0; j < K; ++j) S2[(r * K + i) * K + j] += x[i] * x[j];
        }
    }
}

/* One Gaussian per row fitted to S retained samples by moment matching:
 *   m_r = S1_r / S,   Sigma_r = S2_r / S - m_r m_r^T,   Lambda_r = Sigma_r^{-1}. */
int orc_mm_finalize(int K, int64_t R, int64_t S, const double *S1, const double *S2,
                    double *mu, double *Lam, int64_t *bad_row)
{
    size_t KK = (size_t)K * K;
    double *w = (double *)malloc(sizeof(double) * (2 * KK + K));
    if (!w) return ORC_NOMEM;
    double *Sig = w, *work = w + KK;
    for (int64_t r = 0; r < R; ++r) {
        for (int i = 0; i < K; ++i) mu[r * K + i] = S1[r * K + i] / (double)S;
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j)
                Sig[i * K + j] = S2[(r * K + i) * K + j] / (double)S - mu[r * K + i] * mu[r * K + j];
        if (spd_inverse(K, Sig, Lam + r * (int64_t)KK, work)) {
            if (bad_row) *bad_row = r;
            free(w);
            return ORC_NOT_PD;
        }
    }
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Aggregation of the per-row Gaussians (Eq. 14 with the correction of Algorithm 2).     */
/* ------------------------------------------------------------------------------------- */

/* J submodels hold a Gaussian (mu^(j), Lambda^(j)) for each of R rows; submodel 0 is the
 * one whose posterior was propagated to the others.  For j = 1..J-1:
 *   if Lambda^(j) - Lambda^(0) is positive definite: Lambda*^(j) = Lambda^(j);
 *   else: add |lambda_min| + eps to its diagonal, Lambda*^(j) = corrected + Lambda^(0);
 * then Lambda* = (2 - J) Lambda^(0) + sum_j Lambda*^(j) and
 * mu* = Lambda*^{-1} ((2 - J) Lambda^(0) mu^(0) + sum_j Lambda*^(j) mu^(j)).
 * eps = eps_rel * max(1, mean diagonal of Lambda^(0)).  Positive definiteness is decided by
 * whether the FP64 Cholesky factorisation has all pivots > 0.
 * mu: [J][R][K], Lam: [J][R][K][K]; n_corrected counts corrected (row, j) pairs. */
int orc_aggregate(int K, int64_t R, int J, const double *mu, const double *Lam, double eps_rel,
                  double *mu_star, double *Lam_star, int64_t *n_corrected, int64_t *bad_row)
{
    size_t KK = (size_t)K * K;
    double *w = (double *)malloc(sizeof(double) * (4 * KK + 2 * K));
    if (!w) return ORC_NOMEM;
    double *Dm = w, *L = w + KK, *Lj = w + 2 * KK, *work = w + 3 * KK, *h = w + 4 * KK;
    int64_t ncorr = 0;
    for (int64_t r = 0; r < R; ++r) {
        const double *L0 = Lam + r * (int64_t)KK, *m0 = mu + r * K;
        double *Ls = Lam_star + r * (int64_t)KK;
        double c0 = 2.0 - (double)J;
        double mean_diag = 0.0;
        for (int i = 0; i < K; ++i) mean_diag += L0[i * K + i];
        mean_diag /= (double)K;
        double eps = eps_rel * (mean_diag > 1.0 ? mean_diag : 1.0);
        for (size_t a = 0; a < KK; ++a) Ls[a] = c0 * L0[a];
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += L0[i * K + k] * m0[k];
            h[i] = c0 * s;
        }
        for (int j = 1; j < J; ++j) {
            const double *Lja = Lam + ((int64_t)j * R + r) * (int64_t)KK;
            const double *mj = mu + ((int64_t)j * R + r) * K;
            for (size_t a = 0; a < KK; ++a) Dm[a] = Lja[a] - L0[a];
            if (chol_lower(K, Dm, L) == ORC_OK) {
                for (size_t a = 0; a < KK; ++a) Lj[a] = Lja[a];
            } else {
                double lmin = jacobi_min_eig(K, Dm, work);
                for (int i = 0; i < K; ++i) Dm[i * K + i] += fabs(lmin) + eps;
                for (size_t a = 0; a < KK; ++a) Lj[a] = Dm[a] + L0[a];
                ++ncorr;
            }
            for (size_t a = 0; a < KK; ++a) Ls[a] += Lj[a];
            for (int i = 0; i < K; ++i) {
                double s = 0.0;
                for (int k = 0; k < K; ++k) s += Lj[i * K + k] * mj[k];
                h[i] += s;
            }
        }
        if (chol_lower(K, Ls, L)) {
            if (bad_row) *bad_row = r;
            free(w);
            return ORC_NOT_PD;
        }
        solve_lower(K, L, h);
        solve_lower_t(K, L, h);
        for (int i = 0; i < K; ++i) mu_star[r * K + i] = h[i];
    }
    if (n_corrected) *n_corrected = ncorr;
    free(w);
    return ORC_OK;
}

/* Smallest eigenvalue (exposed for the tests of the correction step). */
double orc_min_eig(int K, const double *M)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)K * K);
    if (!a) return NAN;
    double m = jacobi_min_eig(K, M, a);
    free(a);
    return m;
}

/* ------------------------------------------------------------------------------------- */
/* Prediction with posterior means (Section 5.2: Eq. 1 with the means of X and W).       */
/* ------------------------------------------------------------------------------------- */

void orc_predict(int K, int64_t n, const int32_t *row, const int32_t *col, const double *Xm,
                 const double *Wm, double offset, double *yhat)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += Xm[(int64_t)row[i] * K + k] * Wm[(int64_t)col[i] * K + k];
        yhat[i] = offset + s;
    }
}

/* ------------------------------------------------------------------------------------- */
/* Masked log-joint and its gradient (the differentiation extension).                    */
/* ------------------------------------------------------------------------------------- */

/* l(X, W, log a) = -(a/2) sum_{(n,d) in Omega} (y_nd - x_n^T w_d)^2 + (|Omega|/2) log a
 *                  - 1/2 sum_n (x_n - mu_X)^T Lambda_X (x_n - mu_X)
 *                  - 1/2 sum_d (w_d - mu_W)^T Lambda_W (w_d - mu_W)        (constants dropped)
 * grad_x_n = a sum_{d in Omega_n} r_nd w_d - Lambda_X (x_n - mu_X),   r_nd = y_nd - x_n^T w_d,
 * grad_w_d = a sum_{n in Omega_d} r_nd x_n - Lambda_W (w_d - mu_W),
 * dl/dlog a = |Omega|/2 - (a/2) sum r^2.
 * Observations are given in COO form. */
void orc_logjoint_grad(int K, int64_t N, int64_t D, int64_t nnz, const int32_t *row,
                       const int32_t *col, const double *val, const double *X, const double *W,
                       double log_a, const double *muX, const double *LamX, const double *muW,
                       const double *LamW, double *gX, double *gW, double *g_log_a, double *value)
{
    double a = exp(log_a);
    double sse = 0.0;
    for (int64_t i = 0; i < N * K; ++i) gX[i] = 0.0;
    for (int64_t i = 0; i < D * K; ++i) gW[i] = 0.0;
    for (int64_t e = 0; e < nnz; ++e) {
        const double *x = X + (int64_t)row[e] * K, *w = W + (int64_t)col[e] * K;
        double p = 0.0;
        for (int k = 0; k < K; ++k) p += x[k] * w[k];
        double r = val[e] - p;
        sse += r * r;
        for (int k = 0; k < K; ++k) {
            gX[(int64_t)row[e] * K + k] += a * r * w[k];
            gW[(int64_t)col[e] * K + k] += a * r * x[k];
        }
    }
    double quad = 0.0;
    for (int64_t n = 0; n < N; ++n)
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += LamX[i * K + j] * (X[n * K + j] - muX[j]);
            gX[n * K + i] -= s;
            quad += (X[n * K + i] - muX[i]) * s;
        }
    for (int64_t d = 0; d < D; ++d)
        for (int i = 0; i < K; ++i) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += LamW[i * K + j] * (W[d * K + j] - muW[j]);
            gW[d * K + i] -= s;
            quad += (W[d * K + i] - muW[i]) * s;
        }
    *g_log_a = 0.5 * (double)nnz - 0.5 * a * sse;
    *value = -0.5 * a * sse + 0.5 * (double)nnz * log_a - 0.5 * quad;
}

/* ------------------------------------------------------------------------------------- */
/* Counter-based generator for the draws (the library's device generator draws the same    */
/* numbers): Philox4x64-10 of Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3" (SC'11), and the transforms to normal and chi-square variates.         */
/* ------------------------------------------------------------------------------------- */

/* 64 x 64 -> 128-bit product (hi, lo) from 32-bit halves (schoolbook). */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
    uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    *lo = (mid << 32) | (p00 & 0xffffffffu);
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

/* Philox4x64 with 10 rounds: each round multiplies words 0 and 2 by the two round
 * multipliers, the new words are (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1,
 * lo(M0 x0)), and the key is bumped by the two Weyl constants between rounds. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
        x0 = n0;
        x1 = lo1;
        x2 = n2;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Uniforms from the top 53 bits of a word: [0, 1) and (0, 1]. */
static double u01_closed0(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }
static double u01_open0(uint64_t w) { return (double)((w >> 11) + 1) * 0x1.0p-53; }

/* Box-Muller (1958): two normals from the word pair (a, b). */
static void box_muller(uint64_t a, uint64_t b, double *z0, double *z1)
{
    double r = sqrt(-2.0 * log(u01_open0(a)));
    double th = 6.283185307179586 * u01_closed0(b);
    *z0 = r * cos(th);
    *z1 = r * sin(th);
}

/* Stream tags of the counter's third word. */
#define ORC_KIND_CHI2 1
#define ORC_KIND_NORMAL 2
#define ORC_KIND_Z 3

static uint64_t orc_tag(int32_t sid, int f, int kind)
{
    return ((uint64_t)(uint32_t)sid << 8) | ((uint64_t)f << 4) | (uint64_t)kind;
}

/* Element e of a normal stream: call e / 4 of counter (e / 4, t, tag, 0); the call's words
 * (0, 1) give elements 0 and 1 (cosine, sine), words (2, 3) elements 2 and 3. */
static double stream_normal(const uint64_t key[2], int64_t t, uint64_t tag, int64_t e)
{
    uint64_t ctr[4] = {(uint64_t)(e >> 2), (uint64_t)t, tag, 0}, w[4];
    orc_philox4x64(ctr, key, w);
    int p = (int)((e >> 1) & 1);
    double z0, z1;
    box_muller(w[2 * p], w[2 * p + 1], &z0, &z1);
    return (e & 1) ? z1 : z0;
}

/* chi-square(dof) = 2 Gamma(dof / 2) by Marsaglia & Tsang, "A simple method for generating
 * gamma variables" (ACM TOMS 2000): for shape a >= 1, d = a - 1/3, c = 1 / sqrt(9 d); a
 * candidate x ~ N(0, 1) with v = (1 + c x)^3 > 0 is accepted when u < 1 - 0.0331 x^4 or
 * log u < x^2 / 2 + d (1 - v + log v), giving d v.  For a < 1 the variate for a + 1 is
 * multiplied by U^(1/a).  Attempt j of variate k uses counter (k, t, tag, j): x from words
 * (0, 1) (cosine), u from word 2, U from word 3.  Returns ORC_ARG after 64 rejections. */
static int stream_chi2(const uint64_t key[2], int64_t t, uint64_t tag, int k, double dof,
                       double *out)
{
    if (!(dof > 0.0)) return ORC_ARG;
    double a = 0.5 * dof;
    int boost = a < 1.0;
    double aa = boost ? a + 1.0 : a;
    double d = aa - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
    for (int j = 0; j < 64; ++j) {
        uint64_t ctr[4] = {(uint64_t)k, (uint64_t)t, tag, (uint64_t)j}, w[4];
        orc_philox4x64(ctr, key, w);
        double x, unused;
        box_muller(w[0], w[1], &x, &unused);
        double v = 1.0 + c * x;
        if (!(v > 0.0)) continue;
        v = v * v * v;
        double u = u01_open0(w[2]);
        if (u < 1.0 - 0.0331 * (x * x) * (x * x) ||
            log(u) < 0.5 * x * x + d * (1.0 - v + log(v))) {
            double g = d * v;
            if (boost) g *= pow(u01_open0(w[3]), 1.0 / a);
            *out = 2.0 * g;
            return ORC_OK;
        }
    }
    return ORC_ARG;
}

#define ORC_KIND_NOISE 4

/* The noise-precision variates of sweep t of subset `sid` (Section 2.1 with sampled noise):
 * m chi-square variates, variate k with dof[k], drawn like the hyperparameter chi-squares with
 * tag (sid, W, kind 4) and counter (k, t, tag, attempt). */
int orc_gen_noise(uint64_t seed, int64_t t, int32_t sid, int64_t m, const double *dof,
                  double *out)
{
    const uint64_t key[2] = {seed, 0};
    for (int64_t k = 0; k < m; ++k) {
        int st = stream_chi2(key, t, orc_tag(sid, 1, ORC_KIND_NOISE), (int)k, dof[k], &out[k]);
        if (st) return st;
    }
    return ORC_OK;
}

/* The draws of sweep t (1-based) of subset `sid` with n rows and d columns: the X and W
 * hyperparameter blocks (chi2[K] with dof nu0 + n - k resp. nu0 + d - k, K(K-1)/2 + K normals
 * of the (sid, factor) normal stream) and z of its X rows and W columns (element r K + k of
 * the (sid, factor) z stream).  Key (seed, 0). */
int orc_gen_subset(uint64_t seed, int64_t t, int32_t sid, int K, double nu0, int64_t n,
                   int64_t d, double *hx, double *hw, double *zx, double *zw)
{
    const uint64_t key[2] = {seed, 0};
    const int nn = K * (K - 1) / 2 + K;
    for (int f = 0; f < 2; ++f) {
        double *h = f == 0 ? hx : hw;
        const int64_t m = f == 0 ? n : d;
        for (int k = 0; k < K; ++k) {
            int st = stream_chi2(key, t, orc_tag(sid, f, ORC_KIND_CHI2), k, nu0 + (double)m - k,
                                 &h[k]);
            if (st) return st;
        }
        for (int e = 0; e < nn; ++e)
            h[K + e] = stream_normal(key, t, orc_tag(sid, f, ORC_KIND_NORMAL), e);
        double *z = f == 0 ? zx : zw;
        for (int64_t e = 0; e < m * K; ++e)
            z[e] = stream_normal(key, t, orc_tag(sid, f, ORC_KIND_Z), e);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------- */
/* Summaries beyond moment matching (Section 4.1 "PP DM" and "PP GMM", Section 5.1): the  */
/* retained samples of each row are clustered by lambda-means; the dominant-mode          */
/* approximation fits one Gaussian to the largest cluster, the mixture approximation one  */
/* Gaussian to each of the C largest clusters.                                            */
/* ------------------------------------------------------------------------------------- */

/* lambda-means clustering of S points in R^K (rows of x) with penalty lambda on the squared
 * distance: start from one cluster centred on the first point (the first retained sample; a
 * start at the mean of all points, which lies between the modes of a multimodal posterior,
 * opens spurious clusters on the far sides of the modes that the rounds never merge); then,
 * until no assignment changes (at most max_iter rounds), visit the points in order and give
 * each to the nearest centre (lowest index on ties), unless its squared distance to every
 * centre exceeds lambda, in which case it opens a new cluster centred on itself; after each
 * round move every centre to the mean of its points and drop empty clusters, renumbering the
 * rest in order.
 * assign[S] receives the cluster of each point; returns the number of clusters (>= 1 for
 * S >= 1), or -1 if memory runs out. */
int orc_lambda_means(int K, int S, const double *x, double lambda, int max_iter, int *assign)
{
    if (S <= 0) return 0;
    /* at most S non-empty clusters enter a round, and a round opens at most one per point */
    const size_t cap = 2 * (size_t)S + 1;
    double *cen = (double *)malloc(sizeof(double) * cap * K);
    int *cnt = (int *)malloc(sizeof(int) * cap);
    int *prev = (int *)malloc(sizeof(int) * (size_t)S);
    int *map = (int *)malloc(sizeof(int) * cap);
    if (!cen || !cnt || !prev || !map) {
        free(cen); free(cnt); free(prev); free(map);
        return -1;
    }
    int n = 1;
    for (int k = 0; k < K; ++k) cen[k] = x[k];
    for (int i = 0; i < S; ++i) prev[i] = -1;
    for (int it = 0; it < max_iter; ++it) {
        int changed = 0;
        for (int i = 0; i < S; ++i) {
            const double *p = x + (size_t)i * K;
            int best = 0;
            double dbest = INFINITY;
            for (int c = 0; c < n; ++c) {
                double d = 0.0;
                for (int k = 0; k < K; ++k) {
                    const double e = p[k] - cen[(size_t)c * K + k];
                    d += e * e;
                }
                if (d < dbest) {
                    dbest = d;
                    best = c;
                }
            }
            if (dbest > lambda) {
                best = n++;
                for (int k = 0; k < K; ++k) cen[(size_t)best * K + k] = p[k];
            }
            assign[i] = best;
        }
        /* centres to the means of their points; empty clusters dropped */
        for (int c = 0; c < n; ++c) cnt[c] = 0;
        for (int i = 0; i < S; ++i) cnt[assign[i]]++;
        int m = 0;
        for (int c = 0; c < n; ++c) map[c] = cnt[c] > 0 ? m++ : -1;
        for (int c = 0; c < n; ++c) {
            if (map[c] < 0) continue;
            double *dst = cen + (size_t)map[c] * K;
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int i = 0; i < S; ++i)
                    if (assign[i] == c) s += x[(size_t)i * K + k];
                dst[k] = s / cnt[c];
            }
        }
        n = m;
        for (int i = 0; i < S; ++i) {
            assign[i] = map[assign[i]];
            if (assign[i] != prev[i]) changed = 1;
            prev[i] = assign[i];
        }
        if (!changed) break;
    }
    free(cen); free(cnt); free(prev); free(map);
    return n;
}

/* Mean and precision (inverse of the 1/n covariance) of the points of x (S x K) with
 * assign[i] == c (all points when c < 0); 0, ORC_NOT_PD (fewer than K + 1 points, or a singular
 * covariance) or ORC_NOMEM. */
static int fit_gaussian(int K, int S, const double *x, const int *assign, int c, double *mu,
                        double *Lam)
{
    size_t KK = (size_t)K * K;
    int n = 0;
    for (int k = 0; k < K; ++k) mu[k] = 0.0;
    for (int i = 0; i < S; ++i) {
        if (c >= 0 && assign[i] != c) continue;
        ++n;
        for (int k = 0; k < K; ++k) mu[k] += x[(size_t)i * K + k];
    }
    if (n < K + 1) return ORC_NOT_PD;
    for (int k = 0; k < K; ++k) mu[k] /= n;
    double *w = (double *)malloc(sizeof(double) * (2 * KK + K));
    if (!w) return ORC_NOMEM;
    double *Sig = w, *work = w + KK;
    for (size_t a = 0; a < KK; ++a) Sig[a] = 0.0;
    for (int i = 0; i < S; ++i) {
        if (c >= 0 && assign[i] != c) continue;
        const double *p = x + (size_t)i * K;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) Sig[a * K + b] += (p[a] - mu[a]) * (p[b] - mu[b]);
    }
    for (size_t a = 0; a < KK; ++a) Sig[a] /= n;
    const int st = spd_inverse(K, Sig, Lam, work);
    free(w);
    return st;
}

/* Per-row summaries of R rows from S retained samples (samples [S][R][K]).
 *   mode 0, moment matching: one component fitted to all samples;
 *   mode 1, dominant mode: one component fitted to the largest lambda-means cluster;
 *   mode 2, mixture: one component for each of the C largest clusters (ties: lowest cluster
 *           index) that has at least K + 1 samples, weights proportional to their sizes.
 * A row whose clusters are all too small for a full-rank covariance falls back to moment
 * matching.  Outputs: pi [R][C] (0 for unused components), mu [R][C][K], Lam [R][C][K][K];
 * pooled_mu [R][K] and pooled_Lam [R][K][K], the mean of the fitted mixture and the inverse of
 * its covariance sum_c pi_c (Lam_c^{-1} + (mu_c - m)(mu_c - m)^T), which the aggregation of
 * Eq. 14 takes (Section 4.2, pooled mixture components). */
int orc_fit_summaries(int K, int64_t R, int S, const double *samples, int mode, int C,
                      double lambda, double *pi, double *mu, double *Lam, double *pooled_mu,
                      double *pooled_Lam, int64_t *bad_row)
{
    size_t KK = (size_t)K * K;
    double *x = (double *)malloc(sizeof(double) * (size_t)S * K);
    int *assign = (int *)malloc(sizeof(int) * (size_t)(S > 0 ? S : 1));
    int *size = (int *)malloc(sizeof(int) * (size_t)(S > 0 ? S : 1));
    double *w = (double *)malloc(sizeof(double) * (3 * KK + K));
    if (!x || !assign || !size || !w) {
        free(x); free(assign); free(size); free(w);
        return ORC_NOMEM;
    }
    double *Sig = w, *work = w + KK;   /* Sig [KK]; work [KK + K], or cov [KK] + work [KK + K] */
    int status = ORC_OK;
    for (int64_t r = 0; r < R && status == ORC_OK; ++r) {
        for (int s = 0; s < S; ++s)
            for (int k = 0; k < K; ++k) x[(size_t)s * K + k] = samples[((size_t)s * R + r) * K + k];
        double *pir = pi + r * C, *mur = mu + r * (int64_t)C * K, *Lr = Lam + r * (int64_t)C * KK;
        for (int c = 0; c < C; ++c) pir[c] = 0.0;
        int used = 0;
        if (mode != 0) {
            const int n = orc_lambda_means(K, S, x, lambda, 100, assign);
            if (n < 0) { status = ORC_NOMEM; break; }
            for (int c = 0; c < n; ++c) size[c] = 0;
            for (int s = 0; s < S; ++s) size[assign[s]]++;
            const int want = mode == 1 ? 1 : C;
            for (int t = 0; t < want; ++t) {
                int best = -1;                       /* t-th largest, ties to the lowest index */
                for (int c = 0; c < n; ++c)
                    if (size[c] >= 0 && (best < 0 || size[c] > size[best])) best = c;
                if (best < 0) break;
                const int sz = size[best];
                size[best] = -1;                     /* taken */
                if (sz < K + 1) continue;
                const int st = fit_gaussian(K, S, x, assign, best, mur + (size_t)used * K,
                                            Lr + (size_t)used * KK);
                if (st == ORC_NOMEM) { status = st; break; }
                if (st) continue;
                pir[used++] = sz;
            }
        }
        if (status) break;
        if (used == 0) {                              /* moment matching over all samples */
            const int st = fit_gaussian(K, S, x, NULL, -1, mur, Lr);
            if (st) {
                if (bad_row) *bad_row = r;
                status = st;
                break;
            }
            pir[0] = 1.0;
            used = 1;
        }
        double tot = 0.0;
        for (int c = 0; c < used; ++c) tot += pir[c];
        for (int c = 0; c < used; ++c) pir[c] /= tot;
        /* pooled mean and covariance of the mixture */
        double *pm = pooled_mu + r * K;
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int c = 0; c < used; ++c) s += pir[c] * mur[(size_t)c * K + k];
            pm[k] = s;
        }
        for (size_t a = 0; a < KK; ++a) Sig[a] = 0.0;
        for (int c = 0; c < used; ++c) {
            double *cov = w + KK;                     /* Lam_c^{-1} */
            if (spd_inverse(K, Lr + (size_t)c * KK, cov, w + 2 * KK)) {
                if (bad_row) *bad_row = r;
                status = ORC_NOT_PD;
                break;
            }
            const double *mc = mur + (size_t)c * K;
            for (int a = 0; a < K; ++a)
                for (int b = 0; b < K; ++b)
                    Sig[a * K + b] += pir[c] * (cov[a * K + b] + (mc[a] - pm[a]) * (mc[b] - pm[b]));
        }
        if (status) break;
        if (spd_inverse(K, Sig, pooled_Lam + r * (int64_t)KK, work)) {
            if (bad_row) *bad_row = r;
            status = ORC_NOT_PD;
        }
    }
    free(x); free(assign); free(size); free(w);
    return status;
}

/* Component choice of a mixture prior (Section 5.1, GMM prior): for each row, the component
 * with the largest responsibility pi_c N(x_r; mu_c, Lam_c^{-1}) at the row's current value x_r
 * (log pi_c + (1/2) log det Lam_c - (1/2)(x_r - mu_c)^T Lam_c (x_r - mu_c); ties go to the
 * lowest index; components with pi_c = 0 are skipped); its mean and precision are written to
 * mu_out [R][K] and Lam_out [R][K][K], the per-row prior of the next draw of x_r.
 * chosen [R] (nullable) receives the component. */
int orc_mix_choose(int K, int64_t R, int C, const double *pi, const double *mu, const double *Lam,
                   const double *X, int *chosen, double *mu_out, double *Lam_out)
{
    size_t KK = (size_t)K * K;
    double *L = (double *)malloc(sizeof(double) * (KK + K));
    if (!L) return ORC_NOMEM;
    double *d = L + KK;
    for (int64_t r = 0; r < R; ++r) {
        int best = -1;
        double sbest = -INFINITY;
        for (int c = 0; c < C; ++c) {
            const double p = pi[r * C + c];
            if (!(p > 0.0)) continue;
            const double *m = mu + (r * C + c) * (int64_t)K;
            const double *A = Lam + (r * C + c) * (int64_t)KK;
            if (chol_lower(K, A, L)) { free(L); return ORC_NOT_PD; }
            double logdet = 0.0;
            for (int k = 0; k < K; ++k) logdet += 2.0 * log(L[k * K + k]);
            for (int k = 0; k < K; ++k) d[k] = X[r * K + k] - m[k];
            double q = 0.0;                          /* (x - mu)^T A (x - mu) */
            for (int a = 0; a < K; ++a) {
                double s = 0.0;
                for (int b = 0; b < K; ++b) s += A[a * K + b] * d[b];
                q += d[a] * s;
            }
            const double score = log(p) + 0.5 * logdet - 0.5 * q;
            if (best < 0 || score > sbest) {
                best = c;
                sbest = score;
            }
        }
        if (best < 0) { free(L); return ORC_NOT_PD; }
        if (chosen) chosen[r] = best;
        memcpy(mu_out + r * K, mu + (r * C + best) * (int64_t)K, sizeof(double) * K);
        memcpy(Lam_out + r * (int64_t)KK, Lam + (r * C + best) * (int64_t)KK, sizeof(double) * KK);
    }
    free(L);
    return ORC_OK;
}
