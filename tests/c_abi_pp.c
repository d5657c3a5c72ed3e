/*
 * c_abi_pp.c -- a plain C99 client of libbmf.so (test program).
 *
 * Runs the three stages of posterior propagation (Section 3.2, Algorithm 1) on a 2 x 2 grid
 * with the device generator, then the aggregated posterior means (Eq. 14, Algorithm 2) and the
 * test-set predictions (Section 5.2), through nothing but the C ABI declared in bmf.h.  The
 * problem is read from a binary file written by the test (all little-endian):
 *   int64 N, D, nnz, n_test, K, I, J, sweeps_per_stage, burnin, seed; double tau;
 *   int32 row[nnz], col[nnz]; double val[nnz]; double X0[N*K], W0[D*K];
 *   int32 test_row[n_test], test_col[n_test]; double test_val[n_test].
 * Output file: int64 n_corrected; double rmse, Xm[N*K], Wm[D*K], yhat[n_test].
 * It also checks the host-side error paths that need no data on the GPU (a bad config, a stage
 * opened out of order) and prints "c abi ok" on success; any failure exits non-zero.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "bmf.h"

static void *read_block(FILE *f, size_t n, size_t size) {
    void *p = malloc(n * size + 1);
    if (!p || fread(p, size, n, f) != n) {
        fprintf(stderr, "short read\n");
        exit(2);
    }
    return p;
}

#define CHECK(call)                                                                    \
    do {                                                                               \
        bmf_status s_ = (call);                                                        \
        if (s_ != BMF_OK) {                                                            \
            fprintf(stderr, "%s failed: %d (%s)\n", #call, (int)s_, bmf_last_error(ctx)); \
            return 3;                                                                  \
        }                                                                              \
    } while (0)

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s input.bin output.bin\n", argv[0]);
        return 2;
    }
    FILE *f = fopen(argv[1], "rb");
    if (!f) {
        perror("input");
        return 2;
    }
    int64_t hdr[10];
    double tau;
    if (fread(hdr, sizeof(int64_t), 10, f) != 10 || fread(&tau, sizeof(double), 1, f) != 1) {
        fprintf(stderr, "bad header\n");
        return 2;
    }
    const int64_t N = hdr[0], D = hdr[1], nnz = hdr[2], n_test = hdr[3], K = hdr[4];
    const int32_t I = (int32_t)hdr[5], J = (int32_t)hdr[6], sweeps = (int32_t)hdr[7];
    int32_t *row = read_block(f, (size_t)nnz, sizeof(int32_t));
    int32_t *col = read_block(f, (size_t)nnz, sizeof(int32_t));
    double *val = read_block(f, (size_t)nnz, sizeof(double));
    double *X0 = read_block(f, (size_t)(N * K), sizeof(double));
    double *W0 = read_block(f, (size_t)(D * K), sizeof(double));
    int32_t *trow = read_block(f, (size_t)n_test, sizeof(int32_t));
    int32_t *tcol = read_block(f, (size_t)n_test, sizeof(int32_t));
    double *tval = read_block(f, (size_t)n_test, sizeof(double));
    fclose(f);

    bmf_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.K = (int32_t)K;
    cfg.precision = BMF_FP64;
    cfg.tau = tau;
    cfg.beta0 = 2.0;
    cfg.nu0 = (double)K;
    cfg.order = BMF_ORDER_DECREASING;
    cfg.center = 1;
    cfg.burnin = (int32_t)hdr[8];
    cfg.thin = 1;
    cfg.seed = (uint64_t)hdr[9];
    cfg.eps_rel = 1e-6;
    cfg.moments = BMF_MOMENTS_AUTO;

    bmf_ctx *ctx = NULL;
    /* error path: K = 0 is rejected before anything touches the device */
    bmf_config bad = cfg;
    bad.K = 0;
    if (bmf_init(&ctx, &bad, N, D, nnz, row, col, val, I, NULL, J, NULL, X0, W0, 0, NULL, NULL,
                 NULL, NULL) != BMF_E_ARG || ctx != NULL || bmf_last_error(NULL)[0] == '\0') {
        fprintf(stderr, "K = 0 was not rejected with BMF_E_ARG and a message\n");
        return 4;
    }

    CHECK(bmf_init(&ctx, &cfg, N, D, nnz, row, col, val, I, NULL, J, NULL, X0, W0, n_test, trow,
                   tcol, tval, NULL));
    /* error path: stage 2 cannot open before stage 1 */
    if (bmf_stage(ctx, 2, 1, NULL, NULL) != BMF_E_STATE) {
        fprintf(stderr, "stage 2 before stage 1 was not rejected with BMF_E_STATE\n");
        return 4;
    }
    bmf_sweep_stats st;
    for (int32_t s = 1; s <= 3; ++s) CHECK(bmf_stage(ctx, s, sweeps, NULL, &st));

    double *Xm = malloc((size_t)(N * K) * sizeof(double));
    double *Wm = malloc((size_t)(D * K) * sizeof(double));
    double *yhat = malloc((size_t)n_test * sizeof(double) + 1);
    int64_t n_corr = 0;
    double rmse = 0.0;
    CHECK(bmf_posterior_means(ctx, Xm, Wm, &n_corr));
    CHECK(bmf_predict(ctx, n_test, trow, tcol, tval, yhat, &rmse));
    bmf_destroy(ctx);

    FILE *o = fopen(argv[2], "wb");
    if (!o) {
        perror("output");
        return 2;
    }
    fwrite(&n_corr, sizeof n_corr, 1, o);
    fwrite(&rmse, sizeof rmse, 1, o);
    fwrite(Xm, sizeof(double), (size_t)(N * K), o);
    fwrite(Wm, sizeof(double), (size_t)(D * K), o);
    fwrite(yhat, sizeof(double), (size_t)n_test, o);
    fclose(o);
    printf("c abi ok: rmse %.6f, corrected %lld\n", rmse, (long long)n_corr);
    free(row); free(col); free(val); free(X0); free(W0); free(trow); free(tcol); free(tval);
    free(Xm); free(Wm); free(yhat);
    return 0;
}
