/* A plain C client of the library (C99): it sets up the 4 smallest
 * eigenpairs of a small Dirichlet Laplacian, solves, reads the pairs and
 * destroys the context.  Exit status: 0 solved, 2 the library reported that
 * no usable GPU is present (SAMG_E_CUDA), 1 anything else. */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include "samg.h"

int main(void) {
    enum { N = 12 };
    /* the layout the bindings must mirror */
    printf("sizeof(samg_params) %u offsetof(n_conv) %u\n", (unsigned)sizeof(samg_params),
           (unsigned)offsetof(samg_params, n_conv));
    const int n = N * N;
    int64_t *rp = malloc(sizeof(int64_t) * (n + 1));
    int32_t *col = malloc(sizeof(int32_t) * 5 * n);
    double *val = malloc(sizeof(double) * 5 * n);
    int64_t nnz = 0;
    rp[0] = 0;
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            const int r = j * N + i;
            if (j > 0) { col[nnz] = r - N; val[nnz++] = -1.0; }
            if (i > 0) { col[nnz] = r - 1; val[nnz++] = -1.0; }
            col[nnz] = r; val[nnz++] = 4.0;
            if (i < N - 1) { col[nnz] = r + 1; val[nnz++] = -1.0; }
            if (j < N - 1) { col[nnz] = r + N; val[nnz++] = -1.0; }
            rp[r + 1] = nnz;
        }
    samg_csr A = {n, n, nnz, rp, col, val};
    samg_params p;
    samg_default_params(&p);
    p.coarsest_max = 40;
    samg_ctx *ctx = NULL;
    samg_status st = samg_setup(&A, 4, SAMG_MINIMAL, SAMG_SPD_EIG, &p, NULL, &ctx);
    int rc = 1;
    if (st == SAMG_E_CUDA) {
        fprintf(stderr, "no usable GPU: %s\n", samg_last_error(NULL));
        rc = 2;
    } else if (st == SAMG_OK) {
        int done = 0;
        double sigma[4], resid[4];
        st = samg_solve(ctx, 1e-10, 60, &done);
        if (st == SAMG_OK && samg_get_triplets(ctx, sigma, NULL, NULL, resid) == SAMG_OK) {
            printf("%d iterations, lambda_1 = %.12f\n", done, sigma[0]);
            rc = 0;
        }
        samg_destroy(ctx);
    }
    free(rp);
    free(col);
    free(val);
    return rc;
}
