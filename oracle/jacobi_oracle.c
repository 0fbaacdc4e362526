/*
 * CPU oracle for synchronous Jacobi on a CSR matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA path is checked against.  Only tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * library never calls it and shares no code with it.
 *
 * Build:  gcc -O2 -ffp-contract=off -fPIC -shared -o libjacobi_oracle.so jacobi_oracle.c
 * (-ffp-contract=off: every multiply and add is rounded separately, as
 *  written, with no fused multiply-add.)
 *
 * Notation follows the paper (Sec. 3): A = D + L + U, D the diagonal, and the
 * Jacobi iteration  x^{k+1}_i = (1/a_ii) (b_i - sum_{j != i} a_ij x^k_j).
 * The residual of the pre-update iterate is r^k = b - A x^k, evaluated from
 * the same off-diagonal sum:  r^k_i = (b_i - s_i) - a_ii x^k_i.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { JO_OK = 0, JO_EINVAL = 1, JO_ESINGULAR = 2, JO_ENOTCONV = 3, JO_EHALO = 4 };

/* Diagonal of row i (sum of the stored entries with col == i).  0 if none. */
static double row_diag(const int64_t* rowptr, const int32_t* col, const double* val, int64_t i)
{
    double d = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
        if (col[k] == i) d += val[k];
    return d;
}

/*
 * Diagonal extraction and inverse, computed once before the iterations
 * (Algorithm 1: "D^{-1} is computed once").  dinv_i = 1 / a_ii.
 * Returns JO_ESINGULAR if a diagonal entry is missing or zero.
 */
int jo_diag(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
            double* d, double* dinv)
{
    for (int64_t i = 0; i < n; ++i) {
        double di = row_diag(rowptr, col, val, i);
        if (di == 0.0) return JO_ESINGULAR;
        d[i] = di;
        dinv[i] = 1.0 / di;
    }
    return JO_OK;
}

/* One row of the sweep: the Jacobi update of Sec. 3 and the residual of x^k. */
static void sweep_row(const int64_t* rowptr, const int32_t* col, const double* val,
                      const double* d, const double* dinv, const double* b,
                      const double* x, int64_t i, double* xnext_i, double* r_i)
{
    double s = 0.0;                              /* s_i = sum_{j != i} a_ij x_j, stored order */
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        int64_t j = col[k];
        if (j == i) continue;
        double p = val[k] * x[j];
        s = s + p;
    }
    double t = b[i] - s;                         /* b_i - (L+U) x */
    *xnext_i = dinv[i] * t;                      /* x^{k+1}_i = D^{-1} (b - (L+U) x^k) */
    double dx = d[i] * x[i];
    *r_i = t - dx;                               /* r^k_i = b_i - (A x^k)_i */
}

/*
 * One synchronous sweep over all rows in natural order.
 *   x_next  <- D^{-1} (b - (L+U) x)
 *   r       <- b - A x             (may be NULL)
 *   *sumsq  <- sum r_i^2,  *maxabs <- max |r_i|   (of the pre-update iterate)
 */
int jo_sweep(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const double* d, const double* dinv, const double* b, const double* x,
             double* x_next, double* r, double* sumsq, double* maxabs)
{
    double ss = 0.0, mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double xi, ri;
        sweep_row(rowptr, col, val, d, dinv, b, x, i, &xi, &ri);
        x_next[i] = xi;
        if (r) r[i] = ri;
        ss = ss + ri * ri;
        double a = fabs(ri);
        if (a > mx || a != a) mx = a;
    }
    *sumsq = ss;
    *maxabs = mx;
    return JO_OK;
}

/*
 * Algorithm 1 (vectorial Jacobi) with the test made on the residual of the
 * current iterate before it is updated.
 *   norm_kind = 2 : relres_k = ||r^k||_2 / ||b||_2  (||r^k||_2 if b == 0)
 *   norm_kind = 0 : relres_k = ||r^k||_inf          (absolute, the paper's
 *                   experiments' criterion ||D(x^{k+1}-x^k)||_inf, Sec. 5.2)
 * For k = 0, 1, ...: evaluate r^k; stop with x^k if relres_k <= tol, or when
 * k == maxit.  On return x holds x^k, *sweeps = k (updates applied), and
 * hist[0..k] the relres values (hist may be NULL, else it has maxit+1 slots).
 */
int jo_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const double* b, double* x, double tol, int norm_kind, int64_t maxit,
             int64_t* sweeps, double* relres_out, double* hist)
{
    if (n < 0 || maxit < 0 || (norm_kind != 0 && norm_kind != 2)) return JO_EINVAL;
    double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* dinv = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!d || !dinv || !y) { free(d); free(dinv); free(y); return JO_EINVAL; }
    int st = jo_diag(n, rowptr, col, val, d, dinv);
    if (st != JO_OK) { free(d); free(dinv); free(y); return st; }
    double bb = 0.0;
    for (int64_t i = 0; i < n; ++i) bb = bb + b[i] * b[i];
    double bnorm = sqrt(bb);
    int64_t k = 0;
    double rel = 0.0;
    for (;;) {
        double ss, mx;
        jo_sweep(n, rowptr, col, val, d, dinv, b, x, y, NULL, &ss, &mx);
        if (norm_kind == 2) rel = (bnorm > 0.0) ? sqrt(ss) / bnorm : sqrt(ss);
        else rel = mx;
        if (hist) hist[k] = rel;
        if (rel <= tol) { st = JO_OK; break; }
        if (k == maxit) { st = JO_ENOTCONV; break; }
        memcpy(x, y, sizeof(double) * (size_t)n);   /* x^{k+1} becomes current */
        ++k;
    }
    *sweeps = k;
    *relres_out = rel;
    free(d); free(dinv); free(y);
    return st;
}

/*
 * Partitioned sweep: the CPU stand-in for the paper's distributed exchange
 * (Sec. 4.2.2, dependency lists).  Partition p owns the rows
 * rows[part_ptr[p] .. part_ptr[p+1]) and receives exactly the x entries listed
 * in halo[halo_ptr[p] .. halo_ptr[p+1]) from their owners.  Each partition
 * works on a private copy of x in which only its own and its received entries
 * are visible; reading any other entry is reported as JO_EHALO (the
 * dependency list was incomplete).  Partial norms are combined in partition
 * order.  The iterate must equal jo_sweep's bit for bit.
 */
int jo_partitioned_sweep(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                         const double* d, const double* dinv, const double* b, const double* x,
                         int64_t nparts, const int64_t* part_ptr, const int64_t* rows,
                         const int64_t* halo_ptr, const int64_t* halo,
                         double* x_next, double* sumsq, double* maxabs)
{
    double* loc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    unsigned char* vis = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
    if (!loc || !vis) { free(loc); free(vis); return JO_EINVAL; }
    double ss = 0.0, mx = 0.0;
    for (int64_t p = 0; p < nparts; ++p) {
        memset(vis, 0, (size_t)n);
        for (int64_t q = part_ptr[p]; q < part_ptr[p + 1]; ++q) { loc[rows[q]] = x[rows[q]]; vis[rows[q]] = 1; }
        for (int64_t q = halo_ptr[p]; q < halo_ptr[p + 1]; ++q) { loc[halo[q]] = x[halo[q]]; vis[halo[q]] = 1; }
        double pss = 0.0, pmx = 0.0;
        for (int64_t q = part_ptr[p]; q < part_ptr[p + 1]; ++q) {
            int64_t i = rows[q];
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (!vis[col[k]]) { free(loc); free(vis); return JO_EHALO; }
            double xi, ri;
            sweep_row(rowptr, col, val, d, dinv, b, loc, i, &xi, &ri);
            x_next[i] = xi;
            pss = pss + ri * ri;
            double a = fabs(ri);
            if (a > pmx || a != a) pmx = a;
        }
        ss = ss + pss;
        if (pmx > mx || pmx != pmx) mx = pmx;
    }
    *sumsq = ss;
    *maxabs = mx;
    free(loc); free(vis);
    return JO_OK;
}

/*
 * Sparse matrix-vector product y = A x (stored order, no FMA).  Used by the
 * oracle's refinement and adjoint helpers.
 */
void jo_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const double* x, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s = s + val[k] * x[col[k]];
        y[i] = s;
    }
}

/*
 * Multi-right-hand-side sweep for nrhs systems sharing A; x, b are row-major
 * n x nrhs.  Equivalent to nrhs independent jo_sweep calls (each column is
 * processed with exactly the same operations).  sumsq/maxabs have nrhs slots.
 */
int jo_sweep_multi(int64_t n, int64_t nrhs, const int64_t* rowptr, const int32_t* col, const double* val,
                   const double* d, const double* dinv, const double* b, const double* x,
                   double* x_next, double* sumsq, double* maxabs)
{
    for (int64_t c = 0; c < nrhs; ++c) { sumsq[c] = 0.0; maxabs[c] = 0.0; }
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t c = 0; c < nrhs; ++c) {
            double s = 0.0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                int64_t j = col[k];
                if (j == i) continue;
                double p = val[k] * x[j * nrhs + c];
                s = s + p;
            }
            double t = b[i * nrhs + c] - s;
            x_next[i * nrhs + c] = dinv[i] * t;
            double dx = d[i] * x[i * nrhs + c];
            double r = t - dx;
            sumsq[c] = sumsq[c] + r * r;
            double a = fabs(r);
            if (a > maxabs[c] || a != a) maxabs[c] = a;
        }
    }
    return JO_OK;
}

/*
 * Substructuring with the interface block split between subdomains (Sec. 4.3).
 * Subdomain s holds its local matrix A_s over the nodes it knows, assembled
 * from its own elements; summed over subdomains these give A, and on the
 * interface A33 = sum_s A33^(s) (Eq. (4.6)).  The local rows of all
 * subdomains are stacked in subdomain order: rows sub_ptr[s] .. sub_ptr[s+1]
 * belong to subdomain s, row l is global node grow[l], and its entries carry
 * global columns gcol (an entry is on the diagonal when gcol == grow).
 */

/* Assembled diagonal d_g = sum_s (A_s)_gg, subdomains in ascending order, and
 * dinv_g = 1 / d_g, computed once before the iterations (Algorithm 1). */
int jo_split_diag(int64_t nloc, int64_t n, const int64_t* rowptr, const int32_t* gcol, const double* val,
                  const int32_t* grow, double* d, double* dinv)
{
    for (int64_t g = 0; g < n; ++g) d[g] = 0.0;
    for (int64_t l = 0; l < nloc; ++l)
        for (int64_t k = rowptr[l]; k < rowptr[l + 1]; ++k)
            if (gcol[k] == grow[l]) d[grow[l]] = d[grow[l]] + val[k];
    for (int64_t g = 0; g < n; ++g) {
        if (d[g] == 0.0) return JO_ESINGULAR;
        dinv[g] = 1.0 / d[g];
    }
    return JO_OK;
}

/*
 * One sweep in the split form.  Step 1, local products (Sec. 4.3, matrix-vector
 * product): every subdomain forms, for each of its rows, the off-diagonal
 * local sum  s^(s)_l = sum_{j != g} (A_s)_lj x_j  in stored order.  Step 2,
 * assembly at the interface (Algorithms "collect/send" and "receive/update"):
 * q_g = sum_s s^(s)_l over the subdomains holding g, in ascending subdomain
 * order; a node interior to one subdomain gets its single full sum.  Then the
 * Jacobi update of Sec. 3 with the assembled diagonal:
 *   x'_g = dinv_g (b_g - q_g),   r_g = (b_g - q_g) - d_g x_g.
 * Norms of the pre-update residual (Sec. 4.3, dot product): every subdomain
 * weights its interface nodes by 1/mult_g (mult_g = subdomains holding g),
 * adds w_g r_g^2 over its own rows, and the per-subdomain sums are added in
 * subdomain order (the reduction after the exchange); maxabs = max_g |r_g|.
 */
int jo_split_sweep(int64_t nsub, const int64_t* sub_ptr, int64_t n, const int64_t* rowptr,
                   const int32_t* gcol, const double* val, const int32_t* grow, const int32_t* mult,
                   const double* d, const double* dinv, const double* b, const double* x,
                   double* x_next, double* r, double* sumsq, double* maxabs)
{
    double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* rr = r ? r : (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!q || !rr) { free(q); if (!r) free(rr); return JO_EINVAL; }
    for (int64_t g = 0; g < n; ++g) q[g] = 0.0;
    for (int64_t s = 0; s < nsub; ++s)
        for (int64_t l = sub_ptr[s]; l < sub_ptr[s + 1]; ++l) {
            double sl = 0.0;
            for (int64_t k = rowptr[l]; k < rowptr[l + 1]; ++k) {
                if (gcol[k] == grow[l]) continue;
                double p = val[k] * x[gcol[k]];
                sl = sl + p;
            }
            q[grow[l]] = q[grow[l]] + sl;
        }
    double mx = 0.0;
    for (int64_t g = 0; g < n; ++g) {
        double t = b[g] - q[g];
        x_next[g] = dinv[g] * t;
        double dx = d[g] * x[g];
        rr[g] = t - dx;
        double a = fabs(rr[g]);
        if (a > mx || a != a) mx = a;
    }
    double ss = 0.0;
    for (int64_t s = 0; s < nsub; ++s) {
        double ps = 0.0;
        for (int64_t l = sub_ptr[s]; l < sub_ptr[s + 1]; ++l) {
            double rg = rr[grow[l]];
            double w = 1.0 / (double)mult[grow[l]];
            ps = ps + w * (rg * rg);
        }
        ss = ss + ps;
    }
    *sumsq = ss;
    *maxabs = mx;
    free(q);
    if (!r) free(rr);
    return JO_OK;
}
