// Device-side state, helpers and the residual-norm bookkeeping shared by the
// sweep kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jac {

// Status bits written by kernels into JacCtl::status.
// ST_CONFIG: the launch gave a kernel less dynamic shared memory than its
// stage layout needs (it then touches nothing and returns).
enum : int { ST_TIMEOUT = 1, ST_NUMERIC = 2, ST_CONFIG = 4 };

__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}
// JacCtl::done values.
enum : int { DONE_RUNNING = 0, DONE_CONVERGED = 1, DONE_LIMIT = 2, DONE_NUMERIC = 3 };
// Sweep phases, in the diagonally scaled variables y = D x, f = D e (see
// DevMat).  P64: plain FP64 Jacobi sweep.  P64R: FP64 residual pass of the
// mixed refinement (writes r = b - A x in FP32, no update of y).  P32: FP32
// inner sweep f' = r + S f.  P32L: last inner sweep, fused y += f.
enum : int { PH_P64 = 0, PH_P64R = 1, PH_P32 = 2, PH_P32L = 3 };

// Control block in device memory.  Kernels read it at start and the last /
// first CTA writes it back; the host arms it before each call.
struct JacCtl {
    unsigned long long bar;   // grid-barrier arrivals of the current launch
    // neighbour-synchronised sweeps (reset with `bar` before every launch):
    unsigned long long dec_ready;  // sweeps of the launch whose grid-wide residual sums are published
    unsigned int arrive[4];        // CTAs that finished sweep j, slot j mod 4
    unsigned int ticket;      // last-block detection of the per-sweep launch kernel
    int status;               // ST_* bits
    int done;                 // DONE_*
    int test;                 // 1 = convergence test armed
    int mixed;                // 1 = refinement cycle (P64R, P32.., P32L)
    int phase;                // mixed: position in the cycle, 0 = P64R
    int inner;                // mixed: sweeps per cycle m (>= 2)
    int xbuf;                 // which x buffer holds the current iterate
    int norm_kind;            // 2 = relative 2-norm, 0 = absolute inf-norm
    int fault_skip_cta;       // test hook, -1 = off
    long long k;              // index of the current iterate x^k
    long long k_limit;        // sweep mode: stop when k == k_limit; test mode: last iterate to evaluate
    long long evals;          // residual evaluations in the current call
    long long outer;          // mixed: refinement steps in the current call
    long long k_eval;         // iterate whose residual is in relres
    long long timeout;        // clock64 budget of one wait
    double tol;
    double bnorm;             // ||b||_2
    double relres, res2, resinf;
    double* hist;             // optional history (device), hist_cap entries
    long long hist_cap;
    // stopping on local convergence: the row set whose test ended the solve
    // (-1: none) and its value max |r_i| over that set
    int loc_part;
    int loc_pad;
    double loc_val;
};

struct Partial {
    double ss;                // sum of r_i^2
    unsigned long long mx;    // max over rows of abs_key(r_i)
};

// Off-diagonal iteration-matrix data in the new row order (constant during a
// solve).  The kernels iterate on y = D x: the Jacobi step
//   x'_i = (b_i - sum_{j != i} a_ij x_j) / a_ii
// multiplied by a_ii reads y'_i = b_i + sum_{j != i} S_ij y_j with
// S_ij = -a_ij / a_jj, and the residual of the iterate is r_i = y'_i - y_i.
struct DevMat {
    int n;
    const int* rowptr;        // n+1 (+pad)
    const int* col;           // nnz_off (+pad)
    const double* S64;        // nnz_off (+pad): -a_ij / a_jj
    const float* S32;         // nnz_off (+pad), mixed only
    const double* b;          // n (+pad): right-hand side in the new order
    const double* d;          // n (+pad): a_ii (conversions x <-> y only)
    // Split interface block (Sec. 4.3 local matrices): kernel rows at and after
    // n_own are slot rows holding partial sums of interface rows (n_own == n
    // and slot_info == NULL otherwise).  rowptr/col/S64/b then cover the
    // kernel rows; d and the iterate the n rows.
    int n_own;
    const unsigned* slot_info;   // per slot row: (interface index << 6) | group size at a group's first row
    // Stopping on local convergence: the row sets of the partitions' local
    // tests as a CSR over the rows (row r belongs to sets mem_part[mem_ptr[r]
    // .. mem_ptr[r+1])); NULL otherwise.
    const int* mem_ptr;
    const int* mem_part;
    const int* mem_head;      // row: first set | (number of sets << 24), -1 = none
};

struct DevVec {
    double* x[3];             // FP64 iterate y = D x: nbuf buffers used in rotation
    int nbuf;                 // 2 (ping-pong) or 3 (neighbour-synchronised sweeps)
    float* e[2];              // FP32 inner iterate f = D e, ping-pong (mixed)
    float* dlt;               // FP32 residual r of the last P64R pass (mixed)
    Partial* part;            // [2][nslots] per-sweep partial norms
    Partial* dec;             // [4] grid-wide sums of sweep j in slot j mod 4 (neighbour sync)
    int nslots;
    unsigned long long* trace;  // [ctas][4]: compute ns, barrier-wait ns, sweeps, 0 (persistent kernels)
    // stopping on local convergence: [3][nloc] per-set max abs_key(r_i); the
    // residual of iterate k goes to slot k mod 3
    unsigned long long* loc;
    int nloc;
};

struct DevTiles {
    const int* row0;          // ntiles+1: first row of each tile (tile i ends where i+1 starts) ...
    const int* nnz0;          // ntiles+1: first entry of each tile ...
    const int* row1;          // ntiles: ... or, where the tiles skip rows, end row of each tile
    const int* nnz1;          // ntiles: ... and end entry (batched kernel; row0 + 1 / nnz0 + 1 otherwise)
    const int* cta0;          // ctas+1
    const int* cta1;          // ctas+1: a second tile range per CTA (split layouts: slot tiles), or NULL
    const int* blk0;          // ntiles+1 (halo kernel): int4 offset of each tile's run block
    const int* blk;           // run blocks {xlen, own, nruns, flags} + {src, len, dst, 0} x nruns
    const int* lcol;          // nnz_off tile-local columns (halo kernel)
    int ntiles;
    int emax;                 // staged entry cap of a tile
    int xcap;                 // x window capacity (elements)
    int maxruns;              // runs per tile
    int ntcap;                // halo kernel: tile-table capacity per CTA
    int blkcap;               // halo kernel: run-block capacity per CTA (int4)
    const int* dep_ptr;       // ctas+1: each CTA's neighbours (owners of the rows it reads) ...
    const int* dep;           // ... as CTA indices (neighbour-synchronised sweeps)
    unsigned* done;           // ctas x DONE_STRIDE: sweeps each CTA has finished in the current launch
};

// One 128-byte line per CTA progress flag: every flag has its own writer and
// several pollers, which would otherwise contend for a few shared lines.
constexpr int DONE_STRIDE = 32;

// Per-system state of a batched context (systems packed block-diagonally).
struct DevBatch {
    int nsys, npairs;
    const int* tile_sys;        // ntiles: system of each tile
    const int* sys_pair0;       // nsys+1: each system's (CTA, system) partial slots, contiguous
    const int* cta_pair0;       // ctas: first partial slot of each CTA
    const int* cta_sys0;        // ctas: first system of each CTA
    const double* bnorm;        // nsys*nrhs: ||b_s,q||_2
    unsigned* cnt;              // [2][nsys] arrivals of CTAs that finished a system in a sweep
    int* mask;                  // nsys: bit q set = right-hand side q has stopped
    long long* ksys;            // nsys*nrhs: iterate of the last evaluation (the stopping one once stopped)
    int* kpar;                  // nsys*nrhs: x buffer that holds that iterate (FP64 ping-pong)
    double* rel;                // nsys*nrhs: test value of that iterate
    int* sys_status;            // nsys: DONE_*
    unsigned* ndone;            // systems whose right-hand sides have all stopped
    double* pss;                // [2][npairs][nrhs] partial sum of r^2
    unsigned long long* pmx;    // [2][npairs][nrhs] partial max |r| (bits)
};

// Order key of |r|: the IEEE bits of r shifted left by one, which drops the
// sign bit.  For finite r and +-Inf, key(a) < key(b) iff |a| < |b|, and NaN
// keys lie above every finite and infinite one.  Built with integer shifts
// only (a mask of the sign bit would be turned into an FP64 absolute value,
// which takes a slot of the FP64 pipe in every row).
__device__ __forceinline__ unsigned long long abs_key(double r)
{
    return (unsigned long long)__double_as_longlong(r) << 1;
}

__device__ __forceinline__ double abs_from_key(unsigned long long key)
{
    return __longlong_as_double((long long)(key >> 1));
}

constexpr unsigned long long KEY_INF = 0x7ff0000000000000ull << 1;   // key of +-Inf

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

__device__ __forceinline__ double warp_sum(double v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;   // valid in lane 0
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v)
{
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = umax64(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Residual bookkeeping of one row from its update: r = y' - y = (b - A x)_i.
__device__ __forceinline__ void accumulate_residual(double ynew, double yold, double& ss, unsigned long long& mx)
{
    const double r = __dadd_rn(ynew, -yold);
    ss = __fma_rn(r, r, ss);
    mx = umax64(mx, abs_key(r));
}

// As accumulate_residual, also returning the row's order key abs_key(r).
__device__ __forceinline__ unsigned long long accumulate_residual_key(double ynew, double yold, double& ss,
                                                                      unsigned long long& mx)
{
    const double r = __dadd_rn(ynew, -yold);
    ss = __fma_rn(r, r, ss);
    const unsigned long long key = abs_key(r);
    mx = umax64(mx, key);
    return key;
}

// Stopping on local convergence, called by all 32 lanes of a warp: every
// lane with a row (row >= 0; head = its mem_head word, loaded early by the
// caller) raises the maxima of the row sets holding it to the row's key.  A
// warp whose rows all lie in one set and no other (the common case) makes
// one atomic; otherwise the rows' sets are fetched together and, set by set,
// the lanes naming the same set combine their keys (an exact 64-bit max from
// two 32-bit reductions) before one of them makes the atomic.  The maxima
// are integer keys, so the result does not depend on the order.
constexpr int LOC_MAX_SETS = 8;   // sets holding one row (a box corner node: 8)
__device__ __forceinline__ void local_sets_update(unsigned long long* slot, const int* mem_ptr, const int* mem_part,
                                                  int row, int head, unsigned long long key)
{
    const bool has = row >= 0 && head >= 0;
    const int cnt = has ? (int)((unsigned)head >> 24) : 0;
    const int p = has ? (head & 0xffffff) : -1;
    const unsigned act = __ballot_sync(0xffffffffu, has);
    if (!act) return;
    const int src = __ffs(act) - 1;
    const int p0 = __shfl_sync(0xffffffffu, p, src);
    const bool uniform = __all_sync(0xffffffffu, !has || (cnt == 1 && p == p0));
    if (uniform) {
        const unsigned long long wk = warp_max(has ? key : 0ull);
        if ((threadIdx.x & 31) == 0) atomicMax(slot + p0, wk);
        return;
    }
    int ps[LOC_MAX_SETS];
    const int mb = cnt > 1 ? __ldg(mem_ptr + row) : 0;
#pragma unroll
    for (int e = 0; e < LOC_MAX_SETS; ++e) ps[e] = e == 0 ? p : (e < cnt ? __ldg(mem_part + mb + e) : -1);
    const int cmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)cnt);
    const unsigned hi0 = (unsigned)(key >> 32), lo0 = (unsigned)(key & 0xffffffffull);
#pragma unroll
    for (int e = 0; e < LOC_MAX_SETS; ++e) {
        if (e >= cmax) break;
        const int pe = e < cnt ? ps[e] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, pe);
        const unsigned hi = e < cnt ? hi0 : 0u;
        const unsigned mhi = __reduce_max_sync(peers, hi);
        const unsigned lo = (e < cnt && hi == mhi) ? lo0 : 0u;
        const unsigned mlo = __reduce_max_sync(peers, lo);
        if (pe >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
            atomicMax(slot + pe, ((unsigned long long)mhi << 32) | mlo);
    }
}

// The smallest set maximum of a slot and the lowest set index holding it,
// by one warp (all lanes get the result).  Exact integer keys: every CTA
// computing it from the same slot gets the same answer.
__device__ __forceinline__ void local_sets_min(const unsigned long long* slot, int nloc, unsigned long long& kmin,
                                               int& pmin)
{
    const int lane = threadIdx.x & 31;
    unsigned long long k = ~0ull;
    int p = 0x7fffffff;
    for (int i = lane; i < nloc; i += 32) {
        const unsigned long long v = __ldcg(slot + i);
        if (v < k) { k = v; p = i; }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int p2 = __shfl_xor_sync(0xffffffffu, p, o);
        if (k2 < k || (k2 == k && p2 < p)) { k = k2; p = p2; }
    }
    kmin = k;
    pmin = p;
}

// Phase of a sweep: plain FP64 sweeps, or position `pos` in the mixed
// refinement cycle of `inner` sweeps (FP64 residual pass, FP32 inner sweeps,
// last inner sweep fused with y += f).
__device__ __forceinline__ int phase_of(bool mixed, int pos, int inner)
{
    if (!mixed) return PH_P64;
    if (pos == 0) return PH_P64R;
    return pos == inner - 1 ? PH_P32L : PH_P32;
}

// Fixed-order reduction of `cnt` partials by one warp (lane 0 gets the result).
__device__ __forceinline__ void reduce_partials_warp(const Partial* p, int cnt, double& ss,
                                                     unsigned long long& mx)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    unsigned long long m = 0;
    for (int i = lane; i < cnt; i += 32) {
        s += __ldcg(&p[i].ss);
        m = umax64(m, __ldcg(&p[i].mx));
    }
    s = warp_sum(s);
    m = warp_max(m);
    ss = __shfl_sync(0xffffffffu, s, 0);
    mx = __shfl_sync(0xffffffffu, m, 0);
}

// Test value and next state after evaluating the residual of iterate k.
// Pure function of its inputs: every CTA computing it from the same partial
// sums takes the same decision.
struct Decision {
    double relres, res2, resinf;
    int done;         // DONE_*
    bool numeric_bad;
};

__device__ __forceinline__ Decision decide(int test, double tol, long long k_limit, int norm_kind, double bnorm,
                                          double ss, unsigned long long mx, long long k)
{
    Decision d;
    d.res2 = sqrt(ss);
    d.resinf = abs_from_key(mx);
    d.relres = (norm_kind == 2) ? (bnorm > 0.0 ? d.res2 / bnorm : d.res2) : d.resinf;
    d.numeric_bad = !(ss <= 1.7976931348623157e308) || mx >= KEY_INF;
    if (d.numeric_bad) d.done = DONE_NUMERIC;
    else if (test && d.relres <= tol) d.done = DONE_CONVERGED;
    else if (test && k >= k_limit) d.done = DONE_LIMIT;
    else d.done = DONE_RUNNING;
    return d;
}

// ---------------------------------------------------------------- PTX ------

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                         uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Release/acquire fence at GPU scope: with a relaxed atomic after it, the
// release half of a grid barrier (lighter than __threadfence's fence.sc).
__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p)
{
    return *(volatile const int*)p;
}

}  // namespace jac
