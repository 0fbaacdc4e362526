/*
 * jacobi.h -- C ABI of the GB300 partitioned synchronous Jacobi solver.
 *
 * The library solves A x = b (paper Sec. 1, Eq. (1.1)) for a real square
 * sparse matrix A given in CSR form (Sec. 4.1) by the synchronous Jacobi
 * iteration x^{k+1} = D^{-1}(b - (L+U) x^k) (Sec. 3, Eqs. (3.4)-(3.5)),
 * fused with the residual norm ||b - A x^k|| of every sweep (Algorithm 1).
 * Rows are distributed by one of the paper's three splittings (Sec. 4):
 * band-row, band-row balanced by non-zeros (the sparsity-pattern splitting
 * with dependency lists), or substructuring with subdomain interiors first and
 * the interface block last (Sec. 4.3, Eq. (4.4)).  On one GPU every partition
 * is worked by a group of CTAs; the iterates do not depend on the splitting.
 *
 * Conventions shared by every entry point:
 *   - Every function returns a jac_status; nothing throws across the ABI.
 *     jac_last_error(ctx) returns a message for the last failure on ctx
 *     (jac_last_error(NULL): the last failure of jac_setup* on this thread).
 *   - Pointers tagged JAC_MEM_HOST are ordinary host memory; JAC_MEM_DEVICE
 *     pointers are device memory on the context's device.  The library
 *     never keeps a caller pointer after the call returns: inputs are
 *     copied, outputs are written before return.
 *   - All device work is issued on the stream given in jac_opts.stream
 *     (NULL = the legacy default stream) and every call that returns results
 *     synchronises that stream before returning.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef JACOBI_GB300_H
#define JACOBI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jac_ctx jac_ctx;   /* opaque; owns all device memory and graphs */

typedef enum {
    JAC_OK = 0,
    JAC_EINVAL = 1,      /* invalid argument (shape, index, option, size) */
    JAC_ENOMEM = 2,      /* device or host allocation failed */
    JAC_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
    JAC_ESINGULAR = 4,   /* a diagonal entry a_ii is missing or zero (D not invertible, Sec. 3) */
    JAC_ENOTCONV = 5,    /* maxit reached before the tolerance; x holds the last iterate */
    JAC_ETIMEOUT = 6,    /* a bounded device wait (grid barrier) gave up; iterate undefined */
    JAC_ENUMERIC = 7     /* a residual became NaN or Inf (divergence, rho(T) >= 1) */
} jac_status;

typedef enum {
    JAC_BANDROW = 0,      /* Sec. 4.2: band p = rows [floor(p n/P), floor((p+1) n/P)) */
    JAC_BANDROW_NNZ = 1,  /* Sec. 4.2.2: contiguous bands balanced by non-zeros:
                             boundary k = min{ r : P * IA(r) >= k * nnz } */
    JAC_SUBSTRUCT = 2     /* Sec. 4.3: geometric boxes, one separator node plane per cut at
                             floor(t g / p); interiors of subdomains 0..S-1, then the interface */
} jac_splitting;

typedef enum { JAC_MEM_HOST = 0, JAC_MEM_DEVICE = 1 } jac_memory;

typedef enum {
    JAC_FP64 = 0,         /* every sweep in FP64 */
    JAC_MIXED = 1         /* FP32 sweeps inside FP64 residual/correction refinement */
} jac_precision;

typedef enum {
    JAC_NORM_REL2 = 2,    /* test ||b - A x^k||_2 / ||b||_2 <= tol (||r||_2 if b == 0) */
    JAC_NORM_INF = 0      /* test ||b - A x^k||_inf <= tol (absolute; Sec. 5.2 criterion
                             ||D(x^{k+1} - x^k)||_inf, which equals it) */
} jac_norm;

/* How the persistent kernel orders consecutive sweeps (jac_opts.sync). */
typedef enum {
    JAC_SYNC_GRID = 0,       /* a grid-wide barrier after every sweep, then the test of that sweep */
    JAC_SYNC_NEIGHBOUR = 1,  /* FP64 sweeps (variant 2, 256 threads): a CTA waits only for the CTAs
                                that own the rows it reads (its dependency list, Sec. 4.2.2) and for
                                the residual sums of the sweep before last; the test of x^k is taken
                                one sweep later and x^k is kept for it, so results and counts are
                                those of JAC_SYNC_GRID */
    JAC_SYNC_ASYNC = 2       /* FP64 (variant 2, 256 threads): asynchronous relaxation, the variant
                                the paper's conclusion points to (Sec. 5.2): every CTA re-sweeps
                                its rows with no barrier, in place, so rows read whichever value of
                                each neighbour is in memory.  Not deterministic.  jac_solve stops
                                when an estimate from the latest per-CTA residual sums passes the
                                test, then takes the exact synchronous test of that iterate (and
                                goes on with synchronous sweeps if it fails): the returned test
                                value is exact; k counts relaxation passes plus synchronous sweeps.
                                jac_sweep runs k passes and returns the estimate. */
} jac_sync;

/* How a solve decides that it has converged (jac_opts.stop). */
typedef enum {
    JAC_STOP_GLOBAL = 0,     /* the test value of the whole residual (jac_opts.norm) <= tol.  With
                                JAC_NORM_INF this is also the paper's "simultaneous local
                                convergence of all the processors" (Sec. 3): every partition's
                                local infinity-norm test passing at once is the global one. */
    JAC_STOP_LOCAL = 1       /* stopping on local convergence, under the reading that the run ends
                                at the first sweep in which one partition is locally converged:
                                partition p holds a set of rows R_p and passes when
                                max_{i in R_p} |r_i| <= tol.  R_p is band p for the band
                                splittings; under substructuring it is the nodes of subdomain p's
                                box of grid cells, i.e. its interior and the interface nodes on
                                its box's boundary (Sec. 4.3), so an interface node is held by
                                2, 4 or 8 subdomains.  The paper's substructuring counts fall as
                                subdomains are added (Sec. 5.2 tables), which no test that needs
                                every partition at once can do.  Needs jac_setup, JAC_FP64,
                                JAC_NORM_INF, JAC_SYNC_GRID, variant 0 or 2 with 256-thread tiles
                                and 1, 2 or 4 lanes per row; jac_stats reports the partition that
                                passed and its local value. */
} jac_stop;

/* Square sparse matrix in CSR form (Sec. 4.1: AA = val, JA = col, IA = rowptr).
 * rowptr has n+1 entries, rowptr[0] == index_base, rowptr[n] == nnz + index_base;
 * col/val have nnz entries; index_base is 0 or 1 (the paper prints 1-based
 * arrays).  Entries of a row may come in any column order: each row's
 * off-diagonal terms are summed in the stored order.  Exactly one entry per
 * row may sit on the diagonal and it must be non-zero.  nnz < 2^31. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    int32_t index_base;   /* 0 or 1 */
    int32_t memory;       /* jac_memory of rowptr/col/val */
} jac_csr;

/* Options.  Fill with jac_opts_default() and change what you need; passing
 * NULL anywhere an opts pointer is accepted means the defaults. */
typedef struct {
    int32_t precision;         /* jac_precision (default JAC_FP64) */
    int32_t norm;              /* jac_norm (default JAC_NORM_REL2) */
    int32_t sweeps_per_graph;  /* sweeps per CUDA-graph launch, 1..4096 (default 64) */
    int32_t inner_sweeps;      /* JAC_MIXED: FP32 sweeps per FP64 refinement step, >= 1 (default 128) */
    int32_t grid[3];           /* node grid (gx, gy, gz); required for JAC_SUBSTRUCT */
    int32_t subdomains[3];     /* boxes per axis (px, py, pz); JAC_SUBSTRUCT only */
    const int64_t* node_of_row;/* host array, n entries: grid node i + gx (j + gy k) of each row;
                                  NULL = row r sits at node r */
    int32_t nrhs;              /* right-hand sides sharing A (1..8, default 1) */
    int32_t transpose;         /* 1 = solve with A^T instead of A (adjoint solves) */
    int32_t variant;           /* 0 = auto (2); 1 = one launch per sweep (row kernel);
                                  2 = persistent grid-synchronised pipelined kernel, x gathered
                                  through L1/L2; 3 = as 2 with each tile's x halo (its dependency list,
                                  Sec. 4.2.2) staged into shared memory */
    int32_t tile_rows;         /* threads of a tile (one row each when lanes_per_row = 1): 0 = auto
                                  (256), 224, 256 or 480 (variant 2); 256 (variant 3) */
    int32_t ctas_per_sm;       /* variant 2 with 256-row tiles: 0 = auto (2), or 3 (3-stage pipeline) */
    int32_t lanes_per_row;     /* variant 2 with 256-thread tiles: lanes summing one row (1, 2, 4, 8);
                                  0 = auto: the smallest count whose tile of 256/L longest rows fits a
                                  pipeline stage.  Each row is summed by L interleaved FMA chains and
                                  a fixed pairwise tree, so iterates are bit-identical across
                                  splittings and tilings for a given L and agree to rounding
                                  across L. */
    int32_t stages;            /* variant 2, 256 threads, 2 CTAs/SM: pipeline stages 0 = auto (4), or 3 / 2
                                  larger stages (36 / 54 KB) that hold whole tiles of long rows */
    int32_t sync;              /* jac_sync (default JAC_SYNC_GRID; the autotuner tries grid and
                                  neighbour; JAC_SYNC_ASYNC only when asked for) */
    int32_t debug;             /* 1: canary bytes in the 16-element padding after every device vector of
                                  jac_setup contexts, checked after each jac_sweep / jac_solve; a
                                  write past the end of a vector returns JAC_ECUDA */
    int32_t autotune;          /* 1: jac_setup / jac_setup_batched time every kernel geometry
                                  (variant, tile_rows, ctas_per_sm, lanes, stages, sync): the median
                                  of three timings of about 2 ms or more each; the cost model's prior
                                  geometry is kept unless another is more than 5 % faster.  jac_setup
                                  then re-cuts the CTA row ranges from the measured per-CTA compute
                                  times while that shortens the sweep.  Needs
                                  variant = tile_rows = ctas_per_sm = 0.  With JAC_AUTOTUNE_LOG=1 in
                                  the environment each candidate's time is printed on stderr. */
    int32_t history;           /* >0: record the relres of every evaluated iterate,
                                  up to this many entries (jac_get_history) */
    void* stream;              /* cudaStream_t for all work; NULL = legacy default stream */
    uint64_t timeout_cycles;   /* bound of every device-side wait, in SM clock cycles
                                  (0 = default, about 2 s) */
    int32_t fault_skip_cta;    /* test hook: this CTA never arrives at the grid barrier,
                                  so the others time out (-1 = off) */
    int32_t device;            /* CUDA device ordinal; -1 = the current device */
    int32_t stop;              /* jac_stop (default JAC_STOP_GLOBAL) */
} jac_opts;

/* Statistics of a context (jac_stats). */
typedef struct {
    int64_t n, nnz;               /* rows and stored entries of A (incl. diagonal; jac_setup_local:
                                     of all local matrices) */
    int64_t nparts;               /* partitions of the splitting (SUBSTRUCT: S interiors + 1) */
    int64_t interface_rows;       /* SUBSTRUCT: rows of the interface block */
    int64_t ntiles, ctas;         /* row tiles and CTAs of the sweep kernel */
    int64_t halo_entries;         /* sum over partitions of received x entries (Sec. 4.2.2);
                                     jac_setup_local: interface partial sums assembled per sweep */
    int64_t max_row;              /* longest row (stored entries) */
    int64_t k;                    /* index of the current iterate x^k */
    int64_t sweeps_total;         /* sweeps evaluated since setup / jac_set_x */
    int64_t outer_iterations;     /* JAC_MIXED refinement steps of the last solve */
    int64_t halo_fallback_tiles;  /* tiles whose x halo is gathered from L2 (staged-halo kernel) */
    int64_t halo_window_elems;    /* x values staged into shared memory per sweep (staged-halo kernel) */
    double last_relres;           /* test value of the last evaluated iterate */
    double last_res2, last_resinf;/* ||r||_2 and ||r||_inf of that iterate */
    double last_ms;               /* device time of the last jac_sweep/jac_solve (CUDA events) */
    double bytes_per_sweep_fp64;  /* algorithmic HBM bytes of one FP64 sweep */
    double bytes_per_sweep_fp32;  /* algorithmic HBM bytes of one FP32 inner sweep */
    int32_t variant, precision, splitting, nrhs;
    int32_t tile_rows, ctas_per_sm;  /* kernel geometry in use (chosen by the autotuner if enabled) */
    int32_t lanes_per_row;           /* lanes per row in use (a tile holds tile_rows / lanes_per_row rows) */
    int32_t sync;                    /* jac_sync in use for FP64 sweeps */
    int32_t stages;                  /* pipeline stages of the persistent kernels */
    int32_t stop;                    /* jac_stop in use */
    int32_t stop_part;               /* JAC_STOP_LOCAL: the partition whose local test ended the last
                                        solve (band index, or subdomain s = sx + px (sy + py sz));
                                        -1 if it did not end on a local test */
    double stop_local;               /* its local test value max_{i in R_p} |r_i| */
} jac_stats_t;

/* Defaults for every option. */
void jac_opts_default(jac_opts* o);

/*
 * jac_setup -- validate A, split and reorder it, upload it, build the graphs.
 *
 * Paper: problem statement Sec. 1 Eq. (1.1) (inputs n, A, b; Algorithm 1's
 * D^{-1} "computed once before the iterations"); splittings Sec. 4.2-4.3.
 *   A       square CSR matrix (see jac_csr), host or device memory.
 *   b       right-hand sides, n*nrhs doubles, row-major (b[i*nrhs + c]),
 *           in A->memory; NULL means b = 0.
 *   s       splitting; nparts = number of bands for the band splittings
 *           (1 <= nparts <= n); ignored for JAC_SUBSTRUCT, whose partitions
 *           are the px*py*pz subdomain interiors plus the interface.
 *   o       options (NULL = defaults).
 *   out     receives the new context; *out = NULL on failure.
 * Initial iterate x^0 = 0.
 * Errors: JAC_EINVAL (n < 1, bad indices, duplicate diagonal, nparts out of
 * range, SUBSTRUCT without grid/subdomains, a grid that does not decouple
 * the subdomain interiors, nnz >= 2^31), JAC_ESINGULAR (zero or missing
 * diagonal), JAC_ENOMEM, JAC_ECUDA.
 */
jac_status jac_setup(const jac_csr* A, const double* b, jac_splitting s, int32_t nparts,
                     const jac_opts* o, jac_ctx** out);

/*
 * jac_setup_batched -- nsys independent systems, solved together.
 *
 * Paper: the same iteration (Sec. 3) applied to a block-diagonal system;
 * every system keeps its own residual norm and convergence test.
 *   A[s], b[s]   system s (n_s rows, b[s] is n_s*nrhs row-major), all in
 *                A[0].memory; systems are band-split with one band each.
 *   nsys         1 <= nsys <= 65536.
 * jac_get_x returns the concatenation of the systems' solutions;
 * jac_get_batch_results the per-system sweeps and residuals.
 * Errors as jac_setup.
 */
jac_status jac_setup_batched(int32_t nsys, const jac_csr* A, const double* const* b,
                             const jac_opts* o, jac_ctx** out);

/* One subdomain's local matrix for jac_setup_local (Sec. 4.3, Eq. (4.5)):
 * the rows and columns of the nodes the subdomain knows, in local numbering,
 * with entries assembled from the subdomain's own elements only, so that
 * A = sum_s P_s^T A_s P_s and on the interface A33 = sum_s A33^(s)
 * (Eq. (4.6)).  0-based: rowptr has n+1 entries, rowptr[0] == 0,
 * rowptr[n] == nnz; col holds local indices 0..n-1; l2g[l] is the global row
 * of local node l (distinct within a subdomain).  A local row holds at most
 * one diagonal entry (col == l); a missing one counts as 0.  Host memory. */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
    const int32_t* l2g;
} jac_local;

/*
 * jac_setup_local -- substructuring with the interface block split between
 * subdomains (Sec. 4.3): the paper's local matrices, its two-step
 * matrix-vector product (local products, then the assembly of the partial
 * interface sums, its collect/send and receive/update algorithms) and its
 * weighted interface dot product.
 *   n      global rows; each row 0..n-1 must belong to at least one subdomain.
 *   nsub   subdomains, 1..65536; sub[s] their local matrices (host memory).
 *   b      n doubles in the original row order, host memory; NULL = 0.
 *   o      options (NULL = defaults).  Supported: FP64, nrhs 1, variant 0 or 2,
 *          tile_rows 0 or 256, sync JAC_SYNC_GRID, ctas_per_sm, lanes_per_row
 *          (1, 2, 4; 0 = auto), stages, autotune, history, debug, norm.
 * A row held by one subdomain is interior to it; a row held by m >= 2
 * subdomains is on the interface (m <= 32 / lanes_per_row).  New row order:
 * the interiors of subdomains 0..nsub-1 (ascending global row within each),
 * then the interface (ascending global row).  The assembled diagonal is
 * d_g = sum_s (A_s)_gg, added in ascending subdomain order, computed once.
 * A sweep, in the y = D x form of jac_sweep: each subdomain sums its local
 * off-diagonal terms of each of its rows with S^(s)_gj = -(A_s)_gj / d_j;
 * an interior row's sum is complete; the partial sums of an interface row
 * are added to b_g in ascending subdomain order.  Every interface row is
 * evaluated once, so the residual norm counts it once, which is what the
 * paper's 1/m weights of the interface dot product achieve.
 * jac_set_x, jac_set_b, jac_sweep, jac_solve, jac_get_x, jac_get_history,
 * jac_get_trace and jac_stats work as for jac_setup contexts; jac_stats
 * reports nnz = stored entries of all local matrices, nparts = nsub + 1 and
 * halo_entries = interface partial sums assembled per sweep.
 * Errors: JAC_EINVAL (sizes, indices, a row in no subdomain, a repeated l2g
 * within a subdomain, two diagonal entries in a local row, too many
 * subdomains on one row for the lane count, an unsupported option),
 * JAC_ESINGULAR (an assembled diagonal entry is 0), JAC_ENOMEM, JAC_ECUDA.
 */
jac_status jac_setup_local(int64_t n, int32_t nsub, const jac_local* sub, const double* b,
                           const jac_opts* o, jac_ctx** out);

/*
 * jac_set_x -- set the current iterate x^0 (warm start / resume; Algorithm 1
 * input u^(0)).  x: n*nrhs doubles row-major in the ORIGINAL row order, in
 * `memory`; NULL = zero.  Resets k and sweeps_total to 0.
 */
jac_status jac_set_x(jac_ctx* ctx, const double* x, int32_t memory);

/*
 * jac_set_b -- replace the right-hand side (same layout as in jac_setup);
 * keeps the current iterate.  NULL = zero.
 */
jac_status jac_set_b(jac_ctx* ctx, const double* b, int32_t memory);

/*
 * jac_sweep -- apply exactly k >= 0 synchronous sweeps, no convergence test.
 *
 * Paper: one pass of Algorithm 1's loop body per sweep (q = A x, r = b - q,
 * ||r||, x += D^{-1} r) in the form of Eq. (3.4), carried in y = D x:
 * y' = b + S y with S = -(L+U) D^{-1}, r = y' - y.  After the call the context
 * holds x^{k0+k}.  relres_out (may be NULL) receives the test value
 * (jac_opts.norm) of the last pre-update iterate x^{k0+k-1}
 * (unchanged if k == 0).  For JAC_MIXED contexts a sweep is one FP64 sweep.
 * Errors: JAC_EINVAL (k < 0), JAC_ETIMEOUT, JAC_ENUMERIC, JAC_ECUDA.
 */
jac_status jac_sweep(jac_ctx* ctx, int32_t k, double* relres_out);

/*
 * jac_solve -- iterate until the test value of the current iterate x^k is
 * <= tol, or k reaches maxit (Algorithm 1's "loop until convergence", the
 * test made before the update).
 *   sweeps_out  (may be NULL) k, the number of updates applied since x^0
 *               (the paper's iteration count is k+1).
 *   relres_out  (may be NULL) the test value of x^k.
 * JAC_FP64: every sweep is FP64.  JAC_MIXED: FP64 residual r = b - A x with
 * the test, then inner_sweeps FP32 Jacobi sweeps on A e = r from e = 0,
 * x += e; the test is made only at refinement steps, so k is a multiple of
 * inner_sweeps.  Returns JAC_OK on convergence, JAC_ENOTCONV when maxit was
 * reached (x valid), JAC_ENUMERIC on NaN/Inf, JAC_ETIMEOUT, JAC_ECUDA.
 * Batched contexts stop every system separately; JAC_OK only if all converged.
 */
jac_status jac_solve(jac_ctx* ctx, double tol, int64_t maxit, int64_t* sweeps_out,
                     double* relres_out);

/* jac_get_x -- copy the current iterate x^k (n*nrhs, row-major, ORIGINAL row
 * order) to `x` in `memory`.  The library carries the iterate as y = D x
 * (D = diag(A)); jac_get_x returns x_i = y_i / a_ii with one IEEE division and
 * jac_set_x stores y_i = a_ii x_i with one rounded multiply, so resuming from
 * a read-back x continues from x^k to within one rounding per row. */
jac_status jac_get_x(jac_ctx* ctx, double* x, int32_t memory);

/* jac_get_history -- relres of the iterates evaluated by the last jac_sweep /
 * jac_solve (first entry: the first iterate that call evaluated), when
 * jac_opts.history > 0.  *count receives the number written (<= max). */
jac_status jac_get_history(jac_ctx* ctx, double* out, int64_t max, int64_t* count);

/* jac_get_batch_results -- per system s and right-hand side c (index s*nrhs+c):
 * sweeps applied and the test value of the final iterate.  Host arrays. */
jac_status jac_get_batch_results(jac_ctx* ctx, int64_t* sweeps, double* relres);

/*
 * jac_adjoint_grad -- gradients of a loss through x = A^{-1} b.
 *
 * Given the adjoint solution lambda = A^{-T} dL/dx (obtained from a context
 * built with opts.transpose = 1) and the solution x, writes
 *   dA[e] = -lambda_i * x_j   for every stored entry e = (i, j) of A, in the
 *                             caller's CSR order (the pattern only), and
 * leaves dL/db = lambda to the caller.  lambda, x: n doubles in the original
 * row order, dA: nnz doubles, all in `memory`.  ctx is the forward context
 * (its stored copy of A's pattern is used).  nrhs must be 1.
 */
jac_status jac_adjoint_grad(jac_ctx* ctx, const double* lambda, const double* x, double* dA,
                            int32_t memory);

/*
 * jac_get_trace -- per-CTA time split of the last jac_sweep / jac_solve of a
 * persistent kernel (variants 2, 3): compute_ms[i] = time CTA i spent in its
 * tiles, wait_ms[i] = time it spent in the grid barrier, summed over sweeps.
 * The GPU counterpart of the paper's communication / total time columns
 * (Sec. 5.2 tables).  Host arrays of `max` entries (may be NULL);
 * *ctas receives the CTA count (0 for the one-launch-per-sweep variant).
 */
jac_status jac_get_trace(jac_ctx* ctx, double* compute_ms, double* wait_ms, int64_t max, int64_t* ctas);

/* jac_stats -- counters of the context (see jac_stats_t). */
jac_status jac_stats(jac_ctx* ctx, jac_stats_t* out);

/*
 * jac_partition_plan -- host-only: the row permutation and partition row
 * ranges jac_setup would use (Sec. 4.2-4.3), without a GPU.
 *   perm      n entries: perm[new] = original row (0-based).
 *   part_ptr  nparts_out+1 entries (caller allocates nparts+2 for SUBSTRUCT
 *             = px*py*pz + 2, else nparts + 1): partition p owns new rows
 *             [part_ptr[p], part_ptr[p+1]).
 *   nparts_out (may be NULL) number of partitions.
 * A must be in host memory.  Errors as jac_setup (without CUDA errors).
 */
jac_status jac_partition_plan(const jac_csr* A, jac_splitting s, int32_t nparts, const jac_opts* o,
                              int64_t* perm, int64_t* part_ptr, int64_t* nparts_out);

/*
 * jac_dependency_lists -- host-only: the receive lists of the sparsity-pattern
 * splitting (Sec. 4.2.2) for the partitions of jac_partition_plan.
 * For partition p, the x entries (original 0-based indices) it receives,
 * grouped by owner q ascending and sorted within a group:
 *   recv_ptr  nparts+1 offsets into recv (partition p: [recv_ptr[p], recv_ptr[p+1]))
 *   recv_from owner partition of each entry
 *   recv      original index of each entry
 * Call with recv == NULL first to get the total in *total (recv_ptr is
 * still filled); then with arrays of that size.  The send lists are the
 * receive lists read the other way round.
 */
jac_status jac_dependency_lists(const jac_csr* A, jac_splitting s, int32_t nparts, const jac_opts* o,
                                int64_t* recv_ptr, int32_t* recv_from, int64_t* recv, int64_t* total);

/*
 * jac_sweep_noalloc -- k synchronous Jacobi sweeps that allocate no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they need a solve -- code running under
 * a memory pool that owns the device, loops that must not stall on the device
 * synchronisation cudaMalloc/cudaFree imply, or host applications that forbid
 * allocation after start-up.  It uses only the caller's buffers and a fixed
 * scratch area compiled into the library (JAC_NOALLOC_SCRATCH_BYTES: a vector
 * of JAC_NOALLOC_MAX_ROWS doubles plus the reduction slots).  Once a call is
 * set up in a CUDA context, it calls no allocator, the CUDA runtime's or any
 * library's, on the device or the host (only a failing call builds an error
 * message on the host).
 *
 * Set-up: the first call in each CUDA context (per device for runtime-API
 * callers; again after cudaDeviceReset, which replaces the context) looks the
 * scratch area's device address up.  Under CUDA's default lazy module loading
 * this look-up is also when the library's device code is loaded into that
 * context and the scratch area's device memory is committed there, once,
 * until the context is destroyed.  Make that first call before any stream
 * capture, and where committing memory later is not acceptable.
 *   n          rows, 1 <= n <= JAC_NOALLOC_MAX_ROWS (larger n: JAC_EINVAL).
 *   rowptr, col, val   0-based CSR of A in device memory, diagonal stored in
 *              every row (a zero or missing diagonal returns JAC_ENUMERIC).
 *   b, x_in    device vectors of n doubles; x_out receives x^k (n doubles,
 *              must not alias x_in).  k >= 0 sweeps (k = 0 copies x_in).
 *   relres_out (host, may be NULL) ||b - A x^{k-1}||_2 / ||b||_2 of the last
 *              pre-update iterate (left unchanged when k = 0).
 *   stream     cudaStream_t (NULL = legacy default stream); the call
 *              synchronises it before returning.
 * Each sweep computes x'_i = (b_i - sum_{j != i} a_ij x_j) / a_ii with one
 * launch, as the one-launch-per-sweep variant does.  All calls share the
 * scratch area, which keeps the last call's contents (each call clears what
 * must start at zero): calls whose work overlaps on the GPU race.
 * Errors: JAC_EINVAL, JAC_ENUMERIC, JAC_ECUDA; jac_last_error(NULL)
 * describes the last failure on this thread.
 */
#define JAC_NOALLOC_MAX_ROWS 4194304
#define JAC_NOALLOC_SCRATCH_BYTES 33947712
jac_status jac_sweep_noalloc(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                             const double* b, const double* x_in, double* x_out, int32_t k,
                             double* relres_out, void* stream);

/* Message of the last failure on ctx (NULL ctx: last jac_setup* failure on
 * this thread).  Never NULL; valid until the next call on ctx. */
const char* jac_last_error(const jac_ctx* ctx);

/* Release the context and everything it owns.  NULL-safe. */
void jac_free(jac_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI_GB300_H */
