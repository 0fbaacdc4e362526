// Host-callable launchers of the kernels in jac_kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include "jac_device.cuh"

namespace jac {

cudaError_t launch_row_sweep(int phase, const DevMat& m, const DevVec& v, JacCtl* ctl, cudaStream_t s);

// Persistent kernel instance for (rows per tile, pipeline stages, mixed cycle);
// nullptr if that combination is not compiled.
// part: 0 for FP64 kernels; mixed kernels come as the two launches of a
// refinement cycle, 1 = its FP64 residual pass, 2 = its FP32 inner sweeps.
const void* persistent_kernel(int threads, int stages, bool mixed, int lanes, int sync, int part = 0);
int persistent_smem_bytes(int rows, int emax, int stages);
int persistent_threads(int rows);
const void* halo_kernel(int stages, bool mixed);
int halo_smem_bytes(int rows, int emax, int xcap, int ntcap, int blkcap, int stages);
cudaError_t launch_persistent(const void* fn, int grid, int threads, int smem, const DevMat& m, const DevVec& v,
                              const DevTiles& t, JacCtl* ctl, int max_sweeps, cudaStream_t s);

// x <-> iterate y = D x conversions (d == nullptr: plain permuted copy)
cudaError_t launch_gather_rows(const long long* perm, const double* src, const double* d, double* dst, int n,
                               int nrhs, cudaStream_t s);
cudaError_t launch_scatter_rows(const long long* perm, const double* src, const double* d, double* dst, int n,
                                int nrhs, cudaStream_t s);
// out[r] = b[perm[r]] (0 where perm[r] < 0), r < nout; ||b||_2 over the nb entries of b.
cudaError_t launch_gather_b(const long long* perm, const double* b, double* out, int nout, int nb, JacCtl* ctl,
                            cudaStream_t s);
cudaError_t launch_arm(JacCtl* ctl, int test, int mixed, int inner, long long k_limit, long long k_delta,
                       double tol, int norm_kind, double* hist, long long hist_cap, long long timeout, int skip,
                       cudaStream_t s);
cudaError_t launch_reset_iterate(JacCtl* ctl, cudaStream_t s);
cudaError_t launch_reset_bar(JacCtl* ctl, cudaStream_t s);
// part: 0 = FP64 solves; 1 / 2 = the FP64 pass / the FP32 sweeps of a mixed cycle
const void* batched_kernel(int nrhs, bool mixed, int rows, int part);
// stages of the FP32-sweep launch of a batched mixed cycle (FP32 data only; with
// its gather buffers they fit in the shared memory of the FP64 launch's four)
constexpr int BATCHED_FP32_STAGES = 4;
int batched_smem_bytes(int rows, int emax, int nrhs, int stages, bool fp32 = false);
int batched_threads(int rows);
cudaError_t launch_batched(const void* fn, int grid, int threads, int smem, const DevMat& m, const DevVec& v,
                           const DevTiles& t, const DevBatch& bt, JacCtl* ctl, int max_sweeps, cudaStream_t s);
cudaError_t launch_batched_scale(double* x, const double* d, long long n, int nrhs, cudaStream_t s);
cudaError_t launch_batched_bnorm(const double* b, const long long* off, int nsys, int nrhs, double* bnorm,
                                 cudaStream_t s);
cudaError_t launch_batched_gather_x(const double* x0, const double* x1, const int* row_sys, const int* mask,
                                    const int* kpar, int cur, long long n, int nrhs, const double* d, double* out,
                                    cudaStream_t s);
cudaError_t launch_batched_reset(const DevBatch& bt, int nrhs, cudaStream_t s);
cudaError_t launch_adjoint_grad(const int* rowptr, const int* col, const double* lam, const double* x,
                                double* dA, int n, cudaStream_t s);

}  // namespace jac
