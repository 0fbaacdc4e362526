/*
 * Multi-core CPU baseline of the Jacobi sweep: the oracle's plain row loop
 * (Sec. 3, x^{k+1}_i = (1/a_ii)(b_i - sum_{j != i} a_ij x^k_j), with the
 * residual r^k_i = (b_i - s_i) - a_ii x^k_i of the pre-update iterate)
 * spread over the host's cores with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY, and a timing baseline, not a checker: the
 * benchmark times it next to the single-threaded oracle so that the GPU's
 * speed can be read against every core of the host.  Its reductions of
 * sum r_i^2 and max |r_i| run in OpenMP's order, so its norms may differ
 * from the oracle's in the last bits; nothing compares against them.
 *
 * Build:  gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared -o libjacobi_omp.so jacobi_omp.c
 */
#include <math.h>
#include <stdint.h>
#include <omp.h>

/* Threads the parallel regions use (OMP_NUM_THREADS, else every core). */
int jo_omp_threads(void)
{
    return omp_get_max_threads();
}

/* One synchronous sweep over all rows; d, dinv as computed by the oracle. */
void jo_sweep_omp(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                  const double* d, const double* dinv, const double* b, const double* x,
                  double* x_next, double* sumsq, double* maxabs)
{
    double ss = 0.0, mx = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ss) reduction(max : mx)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t j = col[k];
            if (j != i) s = s + val[k] * x[j];
        }
        const double t = b[i] - s;
        x_next[i] = dinv[i] * t;
        const double r = t - d[i] * x[i];
        ss = ss + r * r;
        const double a = fabs(r);
        if (a > mx) mx = a;
    }
    *sumsq = ss;
    *maxabs = mx;
}
