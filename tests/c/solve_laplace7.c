/*
 * A plain C99 caller of the library's C ABI (include/jacobi.h): builds the
 * 7-point Laplacian on an m^3 grid in CSR form (Sec. 4.1), b = A * ones,
 * solves it by synchronous Jacobi to a relative residual of 1e-8 and checks
 * the solution.  Prints "sweeps=<k> relres=<r> maxerr=<e>" and returns 0, or
 * prints the library's message and returns the jac_status code.
 * Usage: solve_laplace7 [m]   (default 12)
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "jacobi.h"

int main(int argc, char** argv)
{
    const int m = argc > 1 ? atoi(argv[1]) : 12;
    if (m < 1 || m > 200) return 1;
    const int64_t n = (int64_t)m * m * m;
    int32_t* rowptr = malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t* col = malloc(sizeof(int32_t) * (size_t)(7 * n));
    double* val = malloc(sizeof(double) * (size_t)(7 * n));
    double* b = malloc(sizeof(double) * (size_t)n);
    double* x = malloc(sizeof(double) * (size_t)n);
    if (!rowptr || !col || !val || !b || !x) return 2;
    const int off[7][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    int64_t e = 0;
    rowptr[0] = 0;
    for (int k = 0; k < m; ++k)
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) {
                const int64_t r = i + (int64_t)m * (j + (int64_t)m * k);
                double rowsum = 0.0;
                for (int s = 0; s < 7; ++s) {
                    const int ii = i + off[s][0], jj = j + off[s][1], kk = k + off[s][2];
                    if (ii < 0 || ii >= m || jj < 0 || jj >= m || kk < 0 || kk >= m) continue;
                    const int diag = (off[s][0] | off[s][1] | off[s][2]) == 0;
                    col[e] = (int32_t)(ii + (int64_t)m * (jj + (int64_t)m * kk));
                    val[e] = diag ? 6.0 : -1.0;
                    rowsum += val[e];
                    ++e;
                }
                rowptr[r + 1] = (int32_t)e;
                b[r] = rowsum;          /* (A * ones)_r */
            }
    jac_csr A = {n, e, rowptr, col, val, 0, JAC_MEM_HOST};
    jac_opts o;
    jac_opts_default(&o);
    jac_ctx* ctx = NULL;
    jac_status st = jac_setup(&A, b, JAC_BANDROW_NNZ, 4, &o, &ctx);
    if (st != JAC_OK) {
        printf("jac_setup: %s\n", jac_last_error(NULL));
        return (int)st;
    }
    int64_t sweeps = 0;
    double relres = 0.0;
    st = jac_solve(ctx, 1e-8, 100000, &sweeps, &relres);
    if (st == JAC_OK) st = jac_get_x(ctx, x, JAC_MEM_HOST);
    if (st != JAC_OK) {
        printf("jac_solve: %s\n", jac_last_error(ctx));
        jac_free(ctx);
        return (int)st;
    }
    double maxerr = 0.0;
    for (int64_t r = 0; r < n; ++r) maxerr = fmax(maxerr, fabs(x[r] - 1.0));
    printf("sweeps=%lld relres=%.6e maxerr=%.3e\n", (long long)sweeps, relres, maxerr);
    jac_free(ctx);
    free(rowptr); free(col); free(val); free(b); free(x);
    return 0;
}
