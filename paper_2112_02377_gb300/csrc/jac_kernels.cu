// Sweep kernels of the GB300 Jacobi library.
//
// The kernels evaluate the Jacobi step of Sec. 3, Eq. (3.4),
// x' = D^{-1}(b - (L+U) x), in the diagonally scaled iterate y = D x:
//   y'_i = b_i + sum_{j != i} S_ij y_j,   S_ij = -a_ij / a_jj
//   r_i  = y'_i - y_i  = (b - A x)_i      (Algorithm 1's residual of x^k)
// (the same iteration: y' = D x' exactly in real arithmetic; S = D T D^{-1}
// with T = -D^{-1}(L+U)), and fuse the reductions sum r_i^2 and max |r_i|
// (Algorithm 1's norm; the paper's dot products use MPI_ALLREDUCE, Sec. 4.2.2,
// here a grid reduction).  Carrying y instead of x saves the multiply by a_ii
// in the residual and the diagonal's 8 bytes per row in every sweep.
// The off-diagonal terms of a row are accumulated by one thread in the stored
// order with fused multiply-adds, so the iterate depends only on the row and
// never on the splitting, tiling or CTA that computes it.
#include <cuda_runtime.h>

#include "jac_device.cuh"
#include "jac_launch.h"

namespace jac {

constexpr int CHUNK = 8;   // off-diagonal entries whose x loads are issued together

// Load of an iterate entry.  L1 = true: cached in L1 as well (ld.global.ca).
// Only for sweeps that read a buffer nobody writes during the sweep and that
// start after the grid barrier: its release/acquire pair (atomic arrive,
// ld.acquire.gpu and fences by each CTA's thread 0, then a CTA barrier) makes
// the previous sweep's stores visible to these weak loads under the PTX
// memory model, so no L1 line of an older sweep can be returned.  Rows of a
// tile share most of their neighbours' lines (the row's own line, the lines
// one grid line away that the previous tile loaded), which then come from L1
// instead of L2.  Otherwise the load goes to L2 only (ld.global.cg).
template <bool L1, class T>
__device__ __forceinline__ T ld_iter(const T* p)
{
    if constexpr (L1) return __ldca(p);
    else return __ldcg(p);
}

// ------------------------------------------------------------ row math -----

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


// RPT rows of one thread: acc[q] = acc[q] + sum_k T_k x_col(k), entries of each
// row in stored order.  ldx(k) loads x_col(k) (an L2 gather or a read of the
// shared-memory halo); the x loads of a chunk of every row are issued before
// the chunk's FMAs, T is read at the FMA (shared memory, short latency).
// The FMA loop stops at the longest row of the warp (a warp-uniform branch):
// on GB300 the FP64 pipe is the scarce unit, and a predicated-off DFMA costs
// as much of it as a live one.
template <int RPT, bool PREFETCH_T = false, class Real, class LdT, class LdX>
__device__ __forceinline__ void rows_dot(Real (&acc)[RPT], const int (&kb)[RPT], const int (&len)[RPT], LdT ldt,
                                         LdX ldx)
{
    int lmax = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) lmax = len[q] > lmax ? len[q] : lmax;
    lmax = (int)__reduce_max_sync(__activemask(), (unsigned)lmax);
    for (int o = 0; o < lmax; o += CHUNK) {
        Real xv[RPT][CHUNK];
        Real tv[RPT][PREFETCH_T ? CHUNK : 1];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
#pragma unroll
            for (int u = 0; u < CHUNK; ++u) {
                if (o + u < len[q]) {
                    xv[q][u] = ldx(kb[q] + o + u);
                    if constexpr (PREFETCH_T) tv[q][u] = ldt(kb[q] + o + u);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < CHUNK; ++u) {
            if (o + u >= lmax) break;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (o + u < len[q]) {
                    Real tk;
                    if constexpr (PREFETCH_T) tk = tv[q][u];
                    else tk = ldt(kb[q] + o + u);
                    if constexpr (sizeof(Real) == 8) acc[q] = __fma_rn(tk, xv[q][u], acc[q]);
                    else acc[q] = __fmaf_rn(tk, xv[q][u], acc[q]);
                }
            }
        }
    }
}

// A row summed by a group of L consecutive lanes (long rows): lane q of the
// group runs one FMA chain over the row's entries q, q+L, q+2L, ... in stored
// order, starting from `acc` (the caller passes b_i to lane 0 and 0 to the
// others); group_sum then adds the L chains with a fixed xor-shuffle tree.  The
// result depends only on the row and L, never on the tiling or the splitting.
// The loop stops at the warp's longest per-lane count (a warp-uniform bound).
template <int L, class Real, class LdT, class LdX>
__device__ __forceinline__ Real lanes_dot(Real acc, int kb, int len, int q, LdT ldt, LdX ldx)
{
    const int my = len > q ? (len - q + L - 1) / L : 0;
    const int lmax = (int)__reduce_max_sync(__activemask(), (unsigned)my);
    // FP32 sweeps (the inner sweeps of a mixed cycle) also load a chunk's S
    // values together, before its FMAs: the chain then waits on no shared-memory
    // load (mixed 160^3 solve to 1e-8 5 % faster, FE-27 to 1e-10 4.7 %).  For
    // FP64 the eight extra registers cost more than they save (FE-27 sweep
    // 142 against 128 us).
    constexpr bool PRE_T = sizeof(Real) == 4;
    for (int o = 0; o < lmax; o += CHUNK) {
        Real xv[CHUNK];
        [[maybe_unused]] Real tv[CHUNK];
#pragma unroll
        for (int u = 0; u < CHUNK; ++u)
            if (o + u < my) xv[u] = ldx(kb + q + (o + u) * L);
        if constexpr (PRE_T) {
#pragma unroll
            for (int u = 0; u < CHUNK; ++u)
                if (o + u < my) tv[u] = ldt(kb + q + (o + u) * L);
        }
#pragma unroll
        for (int u = 0; u < CHUNK; ++u) {
            if (o + u >= lmax) break;
            if (o + u < my) {
                const Real t = PRE_T ? tv[u] : ldt(kb + q + (o + u) * L);
                if constexpr (sizeof(Real) == 8) acc = __fma_rn(t, xv[u], acc);
                else acc = __fmaf_rn(t, xv[u], acc);
            }
        }
    }
    return acc;
}

// Sum over the L lanes of a group (all lanes of the warp must call it); every
// lane of the group gets the same value (the adds are commutative pairwise).
template <int L, class Real>
__device__ __forceinline__ Real group_sum(Real v)
{
#pragma unroll
    for (int off = L / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// A row of an oversized tile (its S and col were not staged), summed by L
// lanes straight from global memory; kept out of line so that the staged
// loop's register allocation does not carry it.  The loads of GCH entries
// go out together (values and columns, then the gathers) before their FMAs,
// which still run in stored order: a long row costs a few round trips per
// GCH entries instead of one per entry.
constexpr int GCH = 4;
template <int L, class Real>
__device__ __noinline__ Real lanes_global(const Real* S, const int* col, const Real* src, int kb, int len, int q,
                                          Real acc)
{
    int e = kb + q;
    const int end = kb + len;
    for (; e + (GCH - 1) * L < end; e += GCH * L) {
        int c[GCH];
        Real s[GCH], x[GCH];
#pragma unroll
        for (int u = 0; u < GCH; ++u) {
            c[u] = __ldg(col + e + u * L);
            s[u] = __ldg(S + e + u * L);
        }
#pragma unroll
        for (int u = 0; u < GCH; ++u) x[u] = __ldcg(src + c[u]);
#pragma unroll
        for (int u = 0; u < GCH; ++u) {
            if constexpr (sizeof(Real) == 8) acc = __fma_rn(s[u], x[u], acc);
            else acc = __fmaf_rn(s[u], x[u], acc);
        }
    }
    for (; e < end; e += L) {
        if constexpr (sizeof(Real) == 8) acc = __fma_rn(__ldg(S + e), __ldcg(src + __ldg(col + e)), acc);
        else acc = __fmaf_rn(__ldg(S + e), __ldcg(src + __ldg(col + e)), acc);
    }
    return acc;
}

// Interface rows of a split interface block (Sec. 4.3, the two-step product):
// a warp's slot rows hold whole groups, one group per interface row g, its
// rows consecutive in ascending subdomain order, each the partial sum of one
// subdomain's local row; the first row's sum started from b_g.  The lane of
// that first row (info = (interface index << 6) | group size, 0 elsewhere)
// adds the other rows' sums in order -- the receive/update step -- stores y'_g
// and returns (y'_g, y_g); other lanes return zeros.  All 32 lanes call it
// (the acc of a row is the same on its L lanes after group_sum).
template <int L>
__device__ __noinline__ double2 split_assemble(double acc, unsigned info, int n_own, const double* xs, double* xd)
{
    const int lane = threadIdx.x & 31;
    const int g = (int)(info & 63u);
    const int gmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)g);
    double y = acc;
    for (int q = 1; q < gmax; ++q) {
        const int src = lane + q * L;
        const double v = __shfl_sync(0xffffffffu, acc, src < 32 ? src : 31);
        if (q < g) y = __dadd_rn(y, v);
    }
    double2 out = make_double2(0.0, 0.0);
    if (g) {
        const int gi = n_own + (int)(info >> 6);
        out.x = y;
        out.y = __ldcg(xs + gi);
        __stcg(xd + gi, y);
    }
    return out;
}

// Entries prefetched per row by the pipelined persistent kernel (a 7-point row
// has 6 off-diagonal entries); longer rows finish in row_tail.
constexpr int PF = 6;

// Rest of a row beyond the prefetched entries (T and col staged in shared
// memory, x gathered from L2), continuing the same FMA chain in stored order.
template <class Real>
__device__ __noinline__ Real row_tail(const Real* sv, const int* scol, const Real* src, int kb, int len, Real acc)
{
    for (int e = kb; e < kb + len; ++e) {
        if constexpr (sizeof(Real) == 8) acc = __fma_rn(sv[e], __ldcg(src + scol[e]), acc);
        else acc = __fmaf_rn(sv[e], __ldcg(src + scol[e]), acc);
    }
    return acc;
}

// A row of an oversized tile (its T and col were not staged): all from global.
template <class Real>
__device__ __noinline__ Real row_global(const Real* T, const int* col, const Real* src, int kb, int len, Real acc)
{
    for (int e = kb; e < kb + len; ++e) {
        if constexpr (sizeof(Real) == 8) acc = __fma_rn(__ldg(T + e), __ldcg(src + __ldg(col + e)), acc);
        else acc = __fmaf_rn(__ldg(T + e), __ldcg(src + __ldg(col + e)), acc);
    }
    return acc;
}

// =========================================================================
// Variant 1: one launch per sweep, one thread per row, last-block finalize.
// =========================================================================

template <int PH>
__global__ void __launch_bounds__(256) k_row_sweep(DevMat m, DevVec v, JacCtl* ctl)
{
    __shared__ int s_go, s_xb, s_phase, s_inner;
    __shared__ double s_wss[8];
    __shared__ unsigned long long s_wmx[8];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const volatile JacCtl* c = ctl;
        int go = (c->done == DONE_RUNNING) && (c->status == 0);
        if (go && !c->test && c->k >= c->k_limit) go = 0;
        s_go = go;
        s_xb = c->xbuf;
        s_phase = c->phase;
        s_inner = c->inner;
    }
    __syncthreads();
    if (!s_go) return;
    const int i = blockIdx.x * 256 + tid;
    const int xb = s_xb;
    double ss = 0.0;
    unsigned long long mx = 0;
    if (i < m.n) {
        const int kb = __ldg(m.rowptr + i), ke = __ldg(m.rowptr + i + 1);
        auto ldc = [&](int k) { return __ldg(m.col + k); };
        if (PH == PH_P64 || PH == PH_P64R) {
            const double* xs = v.x[xb];
            const double xi = __ldcg(xs + i);
            double acc1[1] = {__ldg(m.b + i)};
            const int kb1[1] = {kb}, len1[1] = {ke - kb};
            rows_dot<1>(acc1, kb1, len1, [&](int k) { return __ldg(m.S64 + k); },
                        [&](int k) { return __ldcg(xs + ldc(k)); });
            const double acc = acc1[0];
            if (PH == PH_P64) {
                v.x[xb ^ 1][i] = acc;
            } else {
                const float dl = (float)__dadd_rn(acc, -xi);
                v.dlt[i] = dl;
                v.e[1][i] = dl;
            }
            accumulate_residual(acc, xi, ss, mx);
        } else {
            const int j = s_phase;   // inner step: e_j -> e_{j+1}
            const float* es = v.e[j & 1];
            float acc1[1] = {__ldcg(v.dlt + i)};
            const int kb1[1] = {kb}, len1[1] = {ke - kb};
            rows_dot<1>(acc1, kb1, len1, [&](int k) { return __ldg(m.S32 + k); },
                        [&](int k) { return __ldcg(es + ldc(k)); });
            const float acc = acc1[0];
            if (PH == PH_P32) v.e[(j + 1) & 1][i] = acc;
            else v.x[xb][i] = __dadd_rn(v.x[xb][i], (double)acc);
        }
    }
    if (PH == PH_P64 || PH == PH_P64R) {
        const double ws = warp_sum(ss);
        const unsigned long long wm = warp_max(mx);
        if ((tid & 31) == 0) { s_wss[tid >> 5] = ws; s_wmx[tid >> 5] = wm; }
        __syncthreads();
        if (tid == 0) {
            double b = 0.0;
            unsigned long long bm = 0;
            for (int w = 0; w < 8; ++w) { b += s_wss[w]; bm = umax64(bm, s_wmx[w]); }
            v.part[blockIdx.x].ss = b;
            v.part[blockIdx.x].mx = bm;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < 32) {
        double tss = 0.0;
        unsigned long long tmx = 0;
        if (PH == PH_P64 || PH == PH_P64R) reduce_partials_warp(v.part, gridDim.x, tss, tmx);
        if (tid == 0) {
            JacCtl* c = ctl;
            c->ticket = 0;
            if (PH == PH_P64 || PH == PH_P64R) {
                const long long k = c->k;
                const Decision d = decide(c->test, c->tol, c->k_limit, c->norm_kind, c->bnorm, tss, tmx, k);
                c->relres = d.relres;
                c->res2 = d.res2;
                c->resinf = d.resinf;
                c->k_eval = k;
                if (c->hist && c->evals < c->hist_cap) c->hist[c->evals] = d.relres;
                c->evals += 1;
                if (d.numeric_bad) c->status |= ST_NUMERIC;
                if (d.done != DONE_RUNNING) c->done = d.done;
                else if (PH == PH_P64) { c->k = k + 1; c->xbuf = xb ^ 1; }
                else c->phase = 1;
            } else if (PH == PH_P32) {
                c->phase = s_phase + 1;
            } else {
                c->phase = 0;
                c->k += s_inner;
                c->outer += 1;
            }
            __threadfence();
        }
    }
}

// =========================================================================
// Variant 2: persistent, grid-synchronised, warp-specialised pipeline.
//
// One CTA = 256 consumer threads (8 warps) + one producer warp.  A tile holds
// 256*RPT consecutive rows; consumer thread t owns rows r0 + t + 256 q,
// q < RPT.  The CTA owns a contiguous range of tiles; for every (sweep, tile)
// job the producer's lane 0 streams the tile's constant data (T, col, IA, c,
// d) into one of STAGES shared-memory stages with cp.async.bulk (completion on
// the stage's `full` mbarrier) as soon as all 8 consumer warps have released
// the stage (its `empty` mbarrier) -- across sweep boundaries, so the matrix
// for the next sweep is in flight while the grid waits at the barrier.
// Consumer warps progress independently between sweep boundaries, which
// overlaps one warp's L2 gathers of x with another warp's FP64 arithmetic.
// Sweeps under the grid barrier gather x through L1 (ld_iter<true>: the
// barrier's acquire orders every read after the stores of the sweep before);
// the other forms gather with ld.global.cg.
// After each sweep the CTAs publish partial norms, pass a bounded grid barrier
// and each reduces all partials in the same fixed order, so every CTA takes
// the same convergence decision.
// =========================================================================

struct StageLayout {
    int o_val, o_col, o_rp, o_c, bytes;   // o_c: the tile's b (FP64 phases)
};

// Regions start on 16-byte boundaries (what cp.async.bulk needs), not on
// 128-byte lines: with 256-row tiles of 7-point rows three CTAs' stages then
// fit the 196 KB shared-memory configuration instead of 228 KB, which leaves
// the SM 60 KB of L1 for the iterate gathers instead of 28 KB.
__host__ __device__ inline StageLayout stage_layout(int rows, int emax)
{
    auto up = [](int v) { return (v + 15) & ~15; };
    StageLayout L;
    L.o_val = 16;                                   // 16-byte header (r0, r1, p0, p1)
    L.o_col = L.o_val + up((emax + 4) * 8);
    L.o_rp = L.o_col + up((emax + 8) * 4);
    L.o_c = L.o_rp + up((rows + 12) * 4);
    L.bytes = L.o_c + up((rows + 4) * 8);
    return L;
}

int persistent_smem_bytes(int rows, int emax, int stages)
{
    return stages * stage_layout(rows, emax).bytes + 2 * stages * 8 + 64;
}


__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int NTHREADS>
__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NTHREADS) : "memory");
}

// Register budget: each SM sub-partition holds 16K registers and a CTA's warps
// are dealt round-robin to the 4 sub-partitions, so (math warps + producer)
// in multiples of 4 per SM leave 128 registers a thread; 2 x 9 warps leave 96.
// LPR = lanes per row: a tile holds 256/LPR rows, each summed by LPR lanes.
//
// SYNC orders consecutive sweeps: 0 = grid barrier, 1 = neighbour flags, 2 =
// none (asynchronous relaxation, see below), 3 = grid barrier over a split
// interface layout (rows from n_own on are slot rows, see split_assemble).
//
// SYNC = 1, neighbour-synchronised FP64 sweeps.  Instead of a grid barrier after
// every sweep, a CTA starts sweep j once (a) the CTAs that own the rows it
// reads (its dependency list, Sec. 4.2.2) have finished sweep j-1, and (b)
// the grid-wide residual sums of sweep j-2 are published.  The last CTA to
// finish a sweep reduces the partial sums once and publishes them; every
// CTA then takes the same convergence decision for sweep j-2 at its gate of
// sweep j.  The iterate rotates through three buffers, so when the test of
// x^k passes, x^k is still intact although sweeps k and k+1 may have run.
// (b) also orders the overwrite of x^{k-2} after every read of it.
//
// SYNC = 2, asynchronous relaxation (the asynchronous variant the paper points
// to for many processes, Sec. 5.2 conclusion): each CTA re-sweeps its rows
// with no barrier, reading and writing one iterate buffer in place, so a row
// uses whichever value of each neighbour is in memory.  After every pass a
// CTA publishes its latest residual sums; CTA 0 adds them into an estimate
// of the test value and stops the launch when it passes.  The estimate mixes
// passes, so jac_solve certifies the result with a synchronous evaluation.
//
// PART splits a mixed refinement cycle into two launches: 1 = its FP64
// residual pass, 2 = its FP32 inner sweeps (0 = every phase).  Each part then
// holds only its own phase's code and registers.
template <int RPT, int STAGES, bool MIXED, int NWM, int LPR, int SYNC, int PART = 0>
__global__ void __maxnreg__(NWM == 8 ? (STAGES == 3 ? 72 : 96) : 128)   // STAGES 3 with 8 math warps: 3 CTAs/SM
k_persistent(DevMat m, DevVec v, DevTiles t, JacCtl* ctl, int max_sweeps)
{
    static_assert(PART == 0 || (MIXED && SYNC == 0), "only the mixed cycle is split");
    constexpr bool NS = (SYNC == 1);      // neighbour-synchronised sweeps
    constexpr bool ASYNC = (SYNC == 2);   // asynchronous (chaotic) relaxation
    constexpr bool SPLIT = (SYNC == 3);   // grid barrier; rows from n_own on are slot rows of a split interface
    constexpr bool LOC = (SYNC == 4);     // grid barrier; the test also ends on one partition's local test
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CT = NWM * 32, NW = NWM, ROWS = CT * RPT / LPR;
    // 7 or 15 math warps have 128 registers: software-pipeline the x gathers of
    // the next tile (pays off when latency, not the FP64 pipe, bounds the sweep:
    // the FP32 inner sweeps); 8 math warps (96 registers) use the plain loop.
    constexpr bool PIPE = (NWM != 8);
    static_assert(!PIPE || LPR == 1, "the pipelined loop sums a row in one lane");
    static_assert(!NS || (!MIXED && !PIPE), "neighbour sync is built for the plain FP64 loop");
    static_assert(!ASYNC || (!MIXED && !PIPE), "asynchronous relaxation is built for the plain FP64 loop");
    static_assert(!SPLIT || (!MIXED && !PIPE), "the split interface block is built for the plain FP64 loop");
    static_assert(!LOC || (!MIXED && !PIPE), "local stopping is built for the plain FP64 loop");
    // Two lanes per row, FP64 sweeps under the grid barrier: consecutive tiles
    // are paired, so that the add of a row's two chains and its residual serve
    // 32 rows per warp instruction instead of 16 (see pair_finish).
    constexpr bool PAIR2 = (LPR == 2 && !PIPE && !SPLIT && !MIXED && (SYNC == 0 || SYNC == 4));
    // gathers of the iterate through L1 (see ld_iter): sweeps under the grid barrier
    constexpr bool GL1 = (SYNC == 0 || SYNC == 3 || SYNC == 4);
    const StageLayout L = stage_layout(ROWS, t.emax);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L.bytes);
    uint64_t* empty = full + STAGES;
    __shared__ double s_wss[NW];
    __shared__ unsigned long long s_wmx[NW];
    __shared__ long long s_k, s_klim, s_evals, s_outer, s_timeout, s_keval;
    __shared__ int s_xb, s_phase, s_inner, s_test, s_done, s_start, s_skip, s_fail, s_dec_done, s_last, s_stopj;
    __shared__ volatile int s_stop;
    __shared__ double s_relres, s_res2, s_resinf;
    __shared__ int s_locpart;
    __shared__ double s_locval;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        const volatile JacCtl* c = ctl;
        s_k = c->k;
        s_klim = c->k_limit;
        s_evals = c->evals;
        s_outer = c->outer;
        s_timeout = c->timeout;
        s_xb = c->xbuf;
        s_phase = c->phase;
        s_inner = c->inner < 2 ? 2 : c->inner;
        s_test = c->test;
        s_done = c->done;
        s_skip = c->fault_skip_cta;
        // the stages and their barriers must fit the dynamic shared memory of the
        // launch, and a split interface layout needs the kernel form built for it
        const bool fits = (unsigned long long)STAGES * L.bytes + 2ull * STAGES * 8 <= dynamic_smem_bytes() &&
                          (m.slot_info != nullptr) == SPLIT;
        if (!fits) atomicOr(&ctl->status, ST_CONFIG);
        s_start = fits && (c->done == DONE_RUNNING) && (c->status == 0);
        s_relres = c->relres;
        s_res2 = c->res2;
        s_resinf = c->resinf;
        s_keval = c->k_eval;
        s_locpart = -1;
        s_locval = 0.0;
        s_stop = 0;
        s_fail = 0;
        if (fits) {
            for (int s = 0; s < STAGES; ++s) {
                mbar_init(&full[s], 1);
                mbar_init(&empty[s], NW);
            }
            fence_mbar_init();
        }
    }
    __syncthreads();
    if (!s_start) return;

    const int tb = t.cta0[blockIdx.x], nt1 = t.cta0[blockIdx.x + 1] - tb;
    // a split interface layout gives every CTA a second range: its share of the slot tiles
    int tb2 = 0, nt2 = 0;
    if constexpr (SPLIT) {
        if (t.cta1) {
            tb2 = t.cta1[blockIdx.x];
            nt2 = t.cta1[blockIdx.x + 1] - tb2;
        }
    }
    const int nt = nt1 + nt2;
    int ksw = max_sweeps;
    if (!MIXED && !s_test) {
        const long long rem = s_klim - s_k;
        ksw = (int)(rem < (long long)ksw ? (rem > 0 ? rem : 0) : ksw);
    }
    // a split-cycle launch runs exactly its phases from the cycle position
    if constexpr (PART == 1) ksw = (s_phase == 0) ? (ksw < 1 ? ksw : 1) : 0;
    if constexpr (PART == 2) {
        const int left = s_phase >= 1 ? s_inner - s_phase : 0;
        ksw = ksw < left ? ksw : left;
    }
    const long long njobs = (long long)ksw * nt;
    const int inner = s_inner;
    const int phase0 = s_phase;
    const int emax = t.emax;
    const long long budget = s_timeout;

    // ================================================= producer warp
    if (warp == NW) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            long long issued = 0;
            for (long long j = 0; j < njobs; ++j) {
                const int sidx = (int)(j % STAGES);
                if (j >= STAGES) {
                    const unsigned par = (unsigned)(((j / STAGES) - 1) & 1);
                    bool ok = mbar_try_wait(&empty[sidx], par);
                    if (!ok) {
                        const long long t0 = clock64();
                        while (!(ok = mbar_try_wait(&empty[sidx], par))) {
                            if (s_stop) break;
                            if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
                        }
                    }
                    if (!ok) break;
                }
                // ---- issue job j
                const int sw = (int)(j / nt);
                const int tj = (int)(j - (long long)sw * nt);
                const int ti = tj < nt1 ? tb + tj : tb2 + (tj - nt1);
                const int ph = phase_of(MIXED, MIXED ? (phase0 + sw) % inner : 0, inner);
                const bool fp64 = PART == 1 ? true : PART == 2 ? false : (ph == PH_P64 || ph == PH_P64R);
                unsigned char* st = smem + sidx * L.bytes;
                const int r0 = __ldg(t.row0 + ti), r1 = __ldg(t.row0 + ti + 1);
                const int p0 = __ldg(t.nnz0 + ti), p1 = __ldg(t.nnz0 + ti + 1);
                int* hdr = reinterpret_cast<int*>(st);
                hdr[0] = r0; hdr[1] = r1; hdr[2] = p0; hdr[3] = p1;
                const bool over = (p1 - p0) > emax;
                unsigned bytes = 0;
                int vb = 0, ve = 0, cb = 0, ce = 0;
                if (!over) {
                    if (fp64) { vb = p0 & ~1; ve = (p1 + 1) & ~1; bytes += (unsigned)(ve - vb) * 8u; }
                    else { vb = p0 & ~3; ve = (p1 + 3) & ~3; bytes += (unsigned)(ve - vb) * 4u; }
                    cb = p0 & ~3; ce = (p1 + 3) & ~3;
                    bytes += (unsigned)(ce - cb) * 4u;
                }
                const int rb = r0 & ~3, re = (r1 + 1 + 3) & ~3;
                bytes += (unsigned)(re - rb) * 4u;
                const int hb = r0 & ~1, he = (r1 + 1) & ~1;
                if (fp64) bytes += (unsigned)(he - hb) * 8u;
                uint64_t* bar = &full[sidx];
                mbar_expect_tx(bar, bytes);
                if (!over) {
                    if (ve > vb) {
                        if (fp64) bulk_g2s(st + L.o_val, m.S64 + vb, (unsigned)(ve - vb) * 8u, bar, pol);
                        else bulk_g2s(st + L.o_val, m.S32 + vb, (unsigned)(ve - vb) * 4u, bar, pol);
                    }
                    if (ce > cb) bulk_g2s(st + L.o_col, m.col + cb, (unsigned)(ce - cb) * 4u, bar, pol);
                }
                bulk_g2s(st + L.o_rp, m.rowptr + rb, (unsigned)(re - rb) * 4u, bar, pol);
                if (fp64 && he > hb) bulk_g2s(st + L.o_c, m.b + hb, (unsigned)(he - hb) * 8u, bar, pol);
                issued = j + 1;
            }
            // Drain: the last min(STAGES, issued) jobs occupy distinct stages;
            // wait until their copies have landed before the CTA may exit.
            const long long t0 = clock64();
            for (long long j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j) {
                const unsigned par = (unsigned)((j / STAGES) & 1);
                while (!mbar_try_wait(&full[(int)(j % STAGES)], par)) {
                    if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
                }
            }
        }
        return;
    }

    // ================================================= consumer warps
    long long k = s_k;
    int xb = s_xb, pos = phase0;
    long long evals = s_evals, outer = s_outer;
    long long jc = 0;
    int nbar = 0;
    unsigned long long tr_comp = 0, tr_wait = 0, tr_mark = (tid == 0) ? global_ns() : 0;
    const long long k0 = k;
    const int xb0 = xb;
    auto next_buf = [&](int b) { return b + 1 == v.nbuf ? 0 : b + 1; };
    // Neighbour sync: convergence decision of sweep j from the published sums
    // (warp 0, lane 0; it has acquired dec_ready > j).  Returns DONE_*.
    auto ns_decide = [&](int j) -> int {
        const Partial* ds = v.dec + (j & 3);
        const double tss = __ldcg(&ds->ss);
        const unsigned long long tmx = __ldcg(&ds->mx);
        const Decision d = decide(s_test, ctl->tol, s_klim, ctl->norm_kind, ctl->bnorm, tss, tmx, k0 + j);
        s_relres = d.relres;
        s_res2 = d.res2;
        s_resinf = d.resinf;
        s_keval = k0 + j;
        if (d.numeric_bad && blockIdx.x == 0) atomicOr(&ctl->status, ST_NUMERIC);
        if (blockIdx.x == 0 && ctl->hist && evals < ctl->hist_cap) ctl->hist[evals] = d.relres;
        evals += 1;
        return d.done;
    };
    // Bounded spin until *p >= target (acquire); false on timeout.
    auto spin_u64 = [&](const unsigned long long* p, unsigned long long target) -> bool {
        const long long t0 = clock64();
        while (ld_acquire_u64(p) < target) {
            if (ld_volatile_i32(&ctl->status) & ST_TIMEOUT) return false;
            if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); return false; }
            __nanosleep(32);
        }
        return true;
    };
    if (tid == 0) s_stopj = -1;
    consumer_sync<CT>();
    for (int sw = 0; sw < ksw; ++sw) {
        if constexpr (ASYNC) {
            // another CTA (CTA 0) may have stopped the relaxation
            if (sw > 0) {
                if (tid == 0 && ld_volatile_i32(&ctl->done) != DONE_RUNNING) s_stopj = sw;
                consumer_sync<CT>();
                if (s_stopj >= 0) break;
            }
        }
        if constexpr (NS) {
            // ---- gate of sweep sw
            if (sw > 0) {
                if (warp == 0) {
                    bool ok = true;
                    const int d0 = __ldg(t.dep_ptr + blockIdx.x), nd = __ldg(t.dep_ptr + blockIdx.x + 1) - d0;
                    if (nd <= 32) {
                        if (lane < nd) {
                            const unsigned* f = t.done + DONE_STRIDE * __ldg(t.dep + d0 + lane);
                            const long long t0 = clock64();
                            while (ld_acquire_u32(f) < (unsigned)sw) {
                                if (ld_volatile_i32(&ctl->status) & ST_TIMEOUT) { ok = false; break; }
                                if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); ok = false; break; }
                                __nanosleep(64);
                            }
                        }
                    } else if (lane == 0) {
                        // many neighbours: wait for the whole grid instead
                        ok = spin_u64(&ctl->dec_ready, (unsigned long long)sw);
                    }
                    if (sw >= 2 && lane == 0 && ok) ok = spin_u64(&ctl->dec_ready, (unsigned long long)(sw - 1));
                    __threadfence();
                    ok = __all_sync(0xffffffffu, ok);
                    if (lane == 0) {
                        // every stop state is written before the barrier below,
                        // so all math threads leave the loop together
                        if (!ok) {
                            s_fail = 1;
                        } else if (sw >= 2) {
                            const int dn = ns_decide(sw - 2);
                            if (dn != DONE_RUNNING) { s_done = dn; s_stopj = sw - 2; }
                        }
                        const unsigned long long tc_ = global_ns();
                        tr_wait += tc_ - tr_mark;
                        tr_mark = tc_;
                    }
                }
                consumer_sync<CT>();
                if (s_fail || s_stopj >= 0) break;
            }
        }
        const int ph = phase_of(MIXED, pos, inner);
        const bool norm_ph = PART == 1 ? true : PART == 2 ? false : (ph == PH_P64 || ph == PH_P64R);
        double ss = 0.0;
        unsigned long long mx = 0;
        // local sets: iterate k's maxima go to slot k mod 3; CTA 0 clears slot
        // (k+1) mod 3 now -- every CTA read it (as slot k-2) before arriving at
        // the barrier of sweep k-1, and it is written after the barrier of
        // sweep k, which CTA 0 reaches after these stores
        unsigned long long* lslot = nullptr;
        if constexpr (LOC) {
            lslot = v.loc + (size_t)(k % 3) * v.nloc;
            if (blockIdx.x == 0 && warp == 0) {
                unsigned long long* nx = v.loc + (size_t)((k + 1) % 3) * v.nloc;
                for (int i = lane; i < v.nloc; i += 32) __stcg(nx + i, 0ull);
                __threadfence();
            }
        }
        const double* xs = v.x[xb];
        double* xd = ASYNC ? v.x[xb] : v.x[next_buf(xb)];   // asynchronous: in place
        const float* es = v.e[pos & 1];
        float* ed = v.e[(pos + 1) & 1];
        // Software pipeline over the sweep's tiles: the x gathers (first chunk of
        // the row and the row's own x) of tile i+1 are issued before the FMA
        // chain of tile i, so L2 latency overlaps FP64 work.  Each row is still
        // one FMA chain in stored order, bit-identical to the other kernels.
        auto wait_full = [&](long long j) -> bool {
            uint64_t* bar = &full[(int)(j % STAGES)];
            const unsigned par = (unsigned)((j / STAGES) & 1);
            if (mbar_try_wait(bar, par)) return true;
            if (s_fail) return false;
            const long long t0 = clock64();
            while (!mbar_try_wait(bar, par)) {
                if (s_fail) return false;
                if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; return false; }
            }
            return true;
        };
        auto run_tiles = [&](auto tag) {
            using Real = decltype(tag);
            constexpr bool F64 = sizeof(Real) == 8;
            const Real* src = F64 ? reinterpret_cast<const Real*>(xs) : reinterpret_cast<const Real*>(es);
            struct Job {
                int sidx, r0, p0, kb, len;
                bool ok, in, over;
                Real xi;
                Real xv[PF];
            };
            auto fetch = [&](long long j, Job& J) {
                J.ok = wait_full(j);
                J.sidx = (int)(j % STAGES);
                if (!J.ok) return;
                const unsigned char* st = smem + J.sidx * L.bytes;
                const int* hdr = reinterpret_cast<const int*>(st);
                J.r0 = hdr[0];
                J.p0 = hdr[2];
                J.over = (hdr[3] - J.p0) > emax;
                const int r = J.r0 + tid;
                J.in = r < hdr[1];
                const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (J.r0 & ~3);
                J.kb = J.in ? srp[r] : 0;
                J.len = J.in ? srp[r + 1] - J.kb : 0;
                if (F64) J.xi = J.in ? __ldcg(reinterpret_cast<const Real*>(xs) + r) : Real(0);
                if (!J.over) {
                    const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (J.p0 & ~3);
#pragma unroll
                    for (int u = 0; u < PF; ++u)
                        if (u < J.len) J.xv[u] = __ldcg(src + scol[J.kb + u]);
                }
            };
            Job cur, nxt;
            bool have = false;
            for (int i = 0; i < nt; ++i, ++jc) {
                if (have) cur = nxt;
                else fetch(jc, cur);
                have = false;
                if (i + 1 < nt && cur.ok) {
                    fetch(jc + 1, nxt);
                    have = nxt.ok;
                }
                if (cur.ok) {
                    const unsigned char* st = smem + cur.sidx * L.bytes;
                    const int r = cur.r0 + tid;
                    const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (cur.p0 & ~3);
                    const Real* sv = reinterpret_cast<const Real*>(st + L.o_val) - (cur.p0 & (F64 ? ~1 : ~3));
                    Real acc;
                    if (F64) acc = cur.in ? Real(reinterpret_cast<const double*>(st + L.o_c)[r - (cur.r0 & ~1)]) : Real(0);
                    else acc = cur.in ? Real(__ldcg(v.dlt + r)) : Real(0);
                    if (!cur.over) {
                        const int lmax = (int)__reduce_max_sync(__activemask(), (unsigned)cur.len);
#pragma unroll
                        for (int u = 0; u < PF; ++u) {
                            if (u >= lmax) break;
                            if (u < cur.len) {
                                if constexpr (F64) acc = __fma_rn(sv[cur.kb + u], cur.xv[u], acc);
                                else acc = __fmaf_rn(sv[cur.kb + u], cur.xv[u], acc);
                            }
                        }
                        if (lmax > PF && cur.len > PF) acc = row_tail(sv, scol, src, cur.kb + PF, cur.len - PF, acc);
                    } else if (cur.in) {
                        acc = row_global(F64 ? reinterpret_cast<const Real*>(m.S64) : reinterpret_cast<const Real*>(m.S32),
                                         m.col, src, cur.kb, cur.len, acc);
                    }
                    if (cur.in) {
                        if constexpr (F64) {
                            if (ph == PH_P64) {
                                __stcg(xd + r, (double)acc);
                            } else {
                                const float dl = (float)__dadd_rn((double)acc, -(double)cur.xi);
                                __stcg(v.dlt + r, dl);
                                __stcg(v.e[1] + r, dl);
                            }
                            accumulate_residual((double)acc, (double)cur.xi, ss, mx);
                        } else {
                            if (ph == PH_P32) __stcg(ed + r, (float)acc);
                            else __stcg(v.x[xb] + r, __dadd_rn(__ldcg(v.x[xb] + r), (double)acc));
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[cur.sidx]);
            }
        };
        if constexpr (PIPE) {
            if (norm_ph) run_tiles(double(0));
            else run_tiles(float(0));
        } else {
            // Tile pairs (PAIR2): after tile t (even position) each lane keeps its
            // chain of its row; after tile t+1 one shuffle gives lane 2p both
            // chains of row p of tile t and lane 2p+1 both chains of row p of
            // tile t+1.  Each adds its two (the same operands as group_sum's
            // tree, so the same bits), then stores y' and takes the residual: one
            // DADD and the residual's DADD and DFMA per 32 rows.
            [[maybe_unused]] double pr_acc = 0.0, pr_xi = 0.0;
            [[maybe_unused]] int pr_r = 0, pr_head = -1;
            [[maybe_unused]] bool pr_in = false;
            [[maybe_unused]] auto pair_finish = [&](double bacc, double bxi, int br, bool bin, int bhead) {
                const bool q0 = (tid & 1) == 0;
                const double recv = __shfl_xor_sync(0xffffffffu, q0 ? bacc : pr_acc, 1);
                const double y = q0 ? pr_acc + recv : bacc + recv;
                const double xv = q0 ? pr_xi : bxi;
                const int row = q0 ? pr_r : br;
                const bool has = q0 ? pr_in : bin;
                [[maybe_unused]] const int head = q0 ? pr_head : bhead;
                [[maybe_unused]] unsigned long long key = 0;
                if (has) {
                    __stcg(xd + row, y);
                    if constexpr (LOC) key = accumulate_residual_key(y, xv, ss, mx);
                    else accumulate_residual(y, xv, ss, mx);
                }
                if constexpr (LOC) local_sets_update(lslot, m.mem_ptr, m.mem_part, has ? row : -1, head, key);
            };
            for (int i = 0; i < nt; ++i, ++jc) {
                const int sidx = (int)(jc % STAGES);
                bool ok = wait_full(jc);
                // the tile body shuffles across the warp (row groups, interface
                // groups): after a timeout every lane must skip it together
                if constexpr (SPLIT || LPR > 1 || LOC) ok = __all_sync(0xffffffffu, ok);
                if (ok) {
                    const unsigned char* st = smem + sidx * L.bytes;
                    const int* hdr = reinterpret_cast<const int*>(st);
                    const int r0 = hdr[0], r1 = hdr[1], p0 = hdr[2], p1 = hdr[3];
                    const bool over = (p1 - p0) > emax;
                    const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (r0 & ~3);
                    const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (p0 & ~3);
                    const int q = tid % LPR;              // lane within the row's group
                    const int r = r0 + tid / LPR;
                    const bool in = r < r1;
                    const bool lead = in && q == 0;       // the lane that owns the row's result
                    const bool own = !SPLIT || r < m.n_own;   // else a slot row of a split interface block
                    const int kb = in ? srp[r] : 0;
                    const int len = in ? srp[r + 1] - kb : 0;
                    if (PAIR2 && norm_ph) {
                        const double* sv = reinterpret_cast<const double*>(st + L.o_val) - (p0 & ~1);
                        const double* sc = reinterpret_cast<const double*>(st + L.o_c) - (r0 & ~1);
                        // y_i of this tile's row, read by the lane that will own the row
                        const bool odd = (i & 1) != 0;
                        const bool owner = in && q == (odd ? 1 : 0);
                        const double xt = owner ? ld_iter<GL1>(xs + r) : 0.0;
                        // the row's set word, fetched while the row is summed
                        [[maybe_unused]] int hd = -1;
                        if constexpr (LOC) hd = owner ? __ldg(m.mem_head + r) : -1;
                        double acc = lead ? sc[r] : 0.0;
                        if (!over)
                            acc = lanes_dot<LPR>(acc, kb, len, q, [&](int e) { return sv[e]; },
                                                 [&](int e) { return ld_iter<GL1>(xs + scol[e]); });
                        else if (in)
                            acc = lanes_global<LPR>(m.S64, m.col, xs, kb, len, q, acc);
                        if (!odd) {
                            pr_acc = acc;
                            pr_xi = xt;
                            pr_r = r;
                            pr_in = in;
                            pr_head = hd;
                            if (i + 1 == nt) pair_finish(0.0, 0.0, 0, false, -1);   // a last tile without a partner
                        } else {
                            pair_finish(acc, xt, r, in, hd);
                        }
                    } else if (norm_ph) {
                        const double* sv = reinterpret_cast<const double*>(st + L.o_val) - (p0 & ~1);
                        const double* sc = reinterpret_cast<const double*>(st + L.o_c) - (r0 & ~1);
                        const double xi = (lead && own) ? ld_iter<GL1>(xs + r) : 0.0;
                        // the row's set word, fetched while the row is summed
                        [[maybe_unused]] int hd = -1;
                        if constexpr (LOC) hd = (lead && own) ? __ldg(m.mem_head + r) : -1;
                        double acc = lead ? sc[r] : 0.0;
                        if (!over)
                            acc = lanes_dot<LPR>(acc, kb, len, q, [&](int e) { return sv[e]; },
                                                 [&](int e) { return ld_iter<GL1>(xs + scol[e]); });
                        else if (in)
                            acc = lanes_global<LPR>(m.S64, m.col, xs, kb, len, q, acc);
                        acc = group_sum<LPR>(acc);
                        [[maybe_unused]] unsigned long long lkey = 0;
                        if (lead && own) {
                            if (ph == PH_P64) {
                                __stcg(xd + r, acc);
                            } else {
                                const float dl = (float)__dadd_rn(acc, -xi);
                                __stcg(v.dlt + r, dl);
                                __stcg(v.e[1] + r, dl);
                            }
                            if constexpr (LOC) lkey = accumulate_residual_key(acc, xi, ss, mx);
                            else accumulate_residual(acc, xi, ss, mx);
                        }
                        if constexpr (LOC)
                            local_sets_update(lslot, m.mem_ptr, m.mem_part, (lead && own) ? r : -1, hd, lkey);
                        if constexpr (SPLIT) {
                            if (r0 >= m.n_own) {          // a tile of slot rows (tiles never mix the two)
                                const unsigned info = lead ? __ldg(m.slot_info + (r - m.n_own)) : 0u;
                                const double2 yy = split_assemble<LPR>(acc, info, m.n_own, xs, xd);
                                if (info) accumulate_residual(yy.x, yy.y, ss, mx);
                            }
                        }
                    } else {
                        const float* sv = reinterpret_cast<const float*>(st + L.o_val) - (p0 & ~3);
                        float acc = lead ? __ldcg(v.dlt + r) : 0.f;
                        if (!over)
                            acc = lanes_dot<LPR>(acc, kb, len, q, [&](int e) { return sv[e]; },
                                                 [&](int e) { return ld_iter<GL1>(es + scol[e]); });
                        else if (in)
                            acc = lanes_global<LPR>(m.S32, m.col, es, kb, len, q, acc);
                        acc = group_sum<LPR>(acc);
                        if (lead) {
                            if (ph == PH_P32) __stcg(ed + r, acc);
                            else __stcg(v.x[xb] + r, __dadd_rn(__ldcg(v.x[xb] + r), (double)acc));
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[sidx]);
            }
        }
        // ---- publish partial norms, grid barrier
        if (norm_ph) {
            const double ws = warp_sum(ss);
            const unsigned long long wm = warp_max(mx);
            if (lane == 0) { s_wss[warp] = ws; s_wmx[warp] = wm; }
        }
        if constexpr (ASYNC) {
            // ---- publish this CTA's latest residual sums; CTA 0 tests their total
            consumer_sync<CT>();
            if (tid == 0) {
                const unsigned long long tb_ = global_ns();
                tr_comp += tb_ - tr_mark;
                tr_mark = tb_;
                double b = 0.0;
                unsigned long long bm = 0;
                for (int w = 0; w < NW; ++w) { b += s_wss[w]; bm = umax64(bm, s_wmx[w]); }
                Partial* slot = v.part + blockIdx.x;
                __stcg(&slot->ss, b);
                __stcg(&slot->mx, bm);
                __threadfence();
            }
            if (blockIdx.x == 0) {
                consumer_sync<CT>();
                if (warp == 0) {
                    __threadfence();
                    double tss;
                    unsigned long long tmx;
                    reduce_partials_warp(v.part, gridDim.x, tss, tmx);
                    if (lane == 0) {
                        // the passes done so far count as sweeps
                        const Decision d = decide(s_test, ctl->tol, s_klim, ctl->norm_kind, ctl->bnorm, tss, tmx,
                                                  k0 + sw + 1);
                        s_relres = d.relres;
                        s_res2 = d.res2;
                        s_resinf = d.resinf;
                        s_keval = k0 + sw + 1;
                        if (d.done != DONE_RUNNING) {
                            s_done = d.done;
                            if (d.numeric_bad) atomicOr(&ctl->status, ST_NUMERIC);
                            atomicExch(&ctl->done, d.done);
                        }
                    }
                }
            }
            ++nbar;
            continue;
        }
        if constexpr (NS) {
            // ---- publish: partial sums, this CTA's progress flag, and (last
            // CTA of the sweep) the grid-wide sums of sweep sw
            consumer_sync<CT>();
            if (tid == 0) {
                const unsigned long long tb_ = global_ns();
                tr_comp += tb_ - tr_mark;
                tr_mark = tb_;
                double b = 0.0;
                unsigned long long bm = 0;
                for (int w = 0; w < NW; ++w) { b += s_wss[w]; bm = umax64(bm, s_wmx[w]); }
                Partial* slot = v.part + (sw & 1) * v.nslots + blockIdx.x;
                __stcg(&slot->ss, b);
                __stcg(&slot->mx, bm);
                __threadfence();
                s_last = 0;
                if (!(s_skip == (int)blockIdx.x)) {
                    st_release_u32(t.done + DONE_STRIDE * blockIdx.x, (unsigned)(sw + 1));
                    s_last = atomicAdd(&ctl->arrive[sw & 3], 1u) == gridDim.x - 1;
                }
            }
            consumer_sync<CT>();
            if (s_last && warp == 0) {
                __threadfence();
                double tss;
                unsigned long long tmx;
                reduce_partials_warp(v.part + (sw & 1) * v.nslots, gridDim.x, tss, tmx);
                if (lane == 0) {
                    Partial* ds = v.dec + (sw & 3);
                    __stcg(&ds->ss, tss);
                    __stcg(&ds->mx, tmx);
                    ctl->arrive[sw & 3] = 0;            // reused by sweep sw + 4
                    __threadfence();
                    atomicMax(&ctl->dec_ready, (unsigned long long)(sw + 1));
                }
            }
            ++nbar;
            xb = next_buf(xb);
            continue;
        }
        consumer_sync<CT>();
        if (tid == 0) {
            const unsigned long long tb_ = global_ns();
            tr_comp += tb_ - tr_mark;
            tr_mark = tb_;
            if (norm_ph) {
                double b = 0.0;
                unsigned long long bm = 0;
                for (int w = 0; w < NW; ++w) { b += s_wss[w]; bm = umax64(bm, s_wmx[w]); }
                Partial* slot = v.part + (sw & 1) * v.nslots + blockIdx.x;
                __stcg(&slot->ss, b);
                __stcg(&slot->mx, bm);
            }
            // release: this CTA's stores (ordered before by the CTA barrier) and
            // its partial sums; acquire: the polling load that sees the last
            // arrival, which the CTA barrier below extends to every thread
            fence_acq_rel_gpu();
            if (!(s_skip == (int)blockIdx.x)) atomicAdd(&ctl->bar, 1ull);
            const unsigned long long target = (unsigned long long)(nbar + 1) * gridDim.x;
            const long long t0 = clock64();
            while (ld_acquire_u64(&ctl->bar) < target) {
                if (ld_volatile_i32(&ctl->status) & ST_TIMEOUT) { s_fail = 1; break; }
                if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; break; }
                __nanosleep(32);
            }
            {
                const unsigned long long tc_ = global_ns();
                tr_wait += tc_ - tr_mark;
                tr_mark = tc_;
            }
        }
        ++nbar;
        consumer_sync<CT>();
        if (s_fail) break;
        // ---- convergence decision (identical in every CTA)
        if (norm_ph) {
            if (warp == 0) {
                double tss;
                unsigned long long tmx;
                reduce_partials_warp(v.part + (sw & 1) * v.nslots, gridDim.x, tss, tmx);
                unsigned long long lk = ~0ull;
                int lp = -1;
                if constexpr (LOC) local_sets_min(lslot, v.nloc, lk, lp);
                if (lane == 0) {
                    const Decision d = decide(s_test, ctl->tol, s_klim, ctl->norm_kind, ctl->bnorm, tss, tmx, k);
                    s_relres = d.relres;
                    s_res2 = d.res2;
                    s_resinf = d.resinf;
                    s_keval = k;
                    s_dec_done = d.done;
                    if constexpr (LOC) {
                        // one partition's local test ends the solve (the global
                        // test passing implies it; NaN keys never pass)
                        if (s_test && !d.numeric_bad && lp >= 0 && lk <= KEY_INF && abs_from_key(lk) <= ctl->tol) {
                            s_dec_done = DONE_CONVERGED;
                            s_locpart = lp;
                            s_locval = abs_from_key(lk);
                        }
                    }
                    if (d.numeric_bad && blockIdx.x == 0) atomicOr(&ctl->status, ST_NUMERIC);
                    if (blockIdx.x == 0 && ctl->hist && evals < ctl->hist_cap) ctl->hist[evals] = d.relres;
                }
            }
            consumer_sync<CT>();
            evals += 1;
            if (s_dec_done != DONE_RUNNING) { s_done = s_dec_done; break; }
            if (ph == PH_P64) { k += 1; xb = next_buf(xb); }
            else pos = 1;
        } else if (ph == PH_P32) {
            pos += 1;
        } else {   // PH_P32L
            pos = 0;
            k += inner;
            outer += 1;
        }
        if (!MIXED && !s_test && k >= s_klim) break;
    }
    if constexpr (ASYNC) {
        k = k0 + nbar;       // passes of this CTA; the iterate stays in its buffer
        xb = xb0;
        evals += nbar;
    }
    if constexpr (NS) {
        // ---- end of the launch: the decisions of the last two sweeps, in order
        if (!s_fail && s_stopj < 0) {
            if (tid == 0) {
                if (nbar > 0 && !spin_u64(&ctl->dec_ready, (unsigned long long)nbar)) s_fail = 1;
                else
                    for (int j = nbar >= 2 ? nbar - 2 : 0; j < nbar; ++j) {
                        const int dn = ns_decide(j);
                        if (dn != DONE_RUNNING) { s_done = dn; s_stopj = j; break; }
                    }
            }
            consumer_sync<CT>();
        }
        // the launch ends at x^{k0+j} (stopped at j) or after its nbar sweeps
        const int jend = s_stopj >= 0 ? s_stopj : nbar;
        k = k0 + jend;
        xb = xb0;
        for (int j = 0; j < jend; ++j) xb = next_buf(xb);
    }
    // tell the producer to stop issuing; it drains its copies before exiting
    if (tid == 0 && v.trace) {
        atomicAdd(v.trace + 4 * blockIdx.x + 0, tr_comp);
        atomicAdd(v.trace + 4 * blockIdx.x + 1, tr_wait);
        atomicAdd(v.trace + 4 * blockIdx.x + 2, (unsigned long long)nbar);
    }
    if (tid == 0) s_stop = 1;
    if (blockIdx.x == 0 && tid == 0) {
        ctl->k = k;
        ctl->xbuf = xb;
        ctl->phase = pos;
        ctl->evals = evals;
        ctl->outer = outer;
        ctl->done = s_done;
        ctl->relres = s_relres;
        ctl->res2 = s_res2;
        ctl->resinf = s_resinf;
        ctl->k_eval = s_keval;
        if constexpr (LOC) {
            ctl->loc_part = s_locpart;
            ctl->loc_val = s_locval;
        }
        __threadfence();
    }
}

// =========================================================================
// Variant 3: persistent kernel with staged x halos (the default).
//
// As variant 2, but each tile also stages its x halo -- the few contiguous
// runs of x its rows read (the tile's dependency list, Sec. 4.2.2), built at
// setup with tile-local column numbers -- into shared memory with
// cp.async.bulk.  The producer warp streams the constant tile data (T, local
// col, IA, c, d, run list) for up to STAGES tiles ahead, across sweep
// boundaries; the x runs of a tile are copied once the grid barrier that
// completes the previous sweep has passed.  The 8 math warps then read only
// shared memory, which keeps the FP64 pipe (GB300's scarce unit for this
// sweep) fed.  Tiles whose halo does not fit (scattered columns) fall back to
// L2 gathers with global column numbers.
// =========================================================================

struct HaloLayout {
    int o_val, o_col, o_rp, o_c, o_x, bytes;
};

__host__ __device__ inline HaloLayout halo_layout(int rows, int emax, int xcap)
{
    auto up = [](int v) { return (v + 127) & ~127; };
    HaloLayout L;
    L.o_val = 128;                                  // header (r0, r1, p0, p1) in the first line
    L.o_col = L.o_val + up((emax + 4) * 8);
    L.o_rp = L.o_col + up((emax + 8) * 4);
    L.o_c = L.o_rp + up((rows + 12) * 4);
    L.o_x = L.o_c + up((rows + 4) * 8);
    L.bytes = L.o_x + up((xcap + 8) * 8);
    return L;
}

// Shared memory of the halo kernel: STAGES stages, then the CTA's tile table
// (row0, nnz0, run-block offsets: ntcap+1 ints each; run blocks: blkcap int4),
// then the mbarriers.
__host__ __device__ inline int halo_table_offset(int rows, int emax, int xcap, int stages)
{
    return stages * halo_layout(rows, emax, xcap).bytes;
}

int halo_smem_bytes(int rows, int emax, int xcap, int ntcap, int blkcap, int stages)
{
    const int tab = ((3 * (ntcap + 1) * 4 + 15) & ~15) + blkcap * 16;
    return halo_table_offset(rows, emax, xcap, stages) + tab + 3 * stages * 8 + 64;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int STAGES, bool MIXED>
__global__ void __maxnreg__(96)
k_halo(DevMat m, DevVec v, DevTiles t, JacCtl* ctl, int max_sweeps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CT = 256, NW = 8;
    const HaloLayout L = halo_layout(CT, t.emax, t.xcap);
    int* s_row0 = reinterpret_cast<int*>(smem + halo_table_offset(CT, t.emax, t.xcap, STAGES));
    int* s_nnz0 = s_row0 + (t.ntcap + 1);
    int* s_boff = s_nnz0 + (t.ntcap + 1);
    int4* s_blk = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(s_row0) +
                                          ((3 * (t.ntcap + 1) * 4 + 15) & ~15));
    uint64_t* fmat = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(s_blk) + t.blkcap * 16);
    uint64_t* fx = fmat + STAGES;
    uint64_t* empty = fx + STAGES;
    // the stages, the tile table and the barriers must fit the launch's dynamic shared memory
    const bool halo_fits =
        (unsigned long long)(reinterpret_cast<unsigned char*>(empty + STAGES) - smem) <= dynamic_smem_bytes();
    __shared__ double s_wss[NW];
    __shared__ unsigned long long s_wmx[NW];
    __shared__ long long s_k, s_klim, s_evals, s_outer, s_timeout, s_keval;
    __shared__ int s_xb, s_phase, s_inner, s_test, s_done, s_start, s_skip, s_fail, s_dec_done;
    __shared__ volatile int s_stop, s_epoch;
    __shared__ double s_relres, s_res2, s_resinf;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tb = t.cta0[blockIdx.x], te = t.cta0[blockIdx.x + 1], nt = te - tb;
    if (tid == 0) {
        const volatile JacCtl* c = ctl;
        s_k = c->k;
        s_klim = c->k_limit;
        s_evals = c->evals;
        s_outer = c->outer;
        s_timeout = c->timeout;
        s_xb = c->xbuf;
        s_phase = c->phase;
        s_inner = c->inner < 2 ? 2 : c->inner;
        s_test = c->test;
        s_done = c->done;
        s_skip = c->fault_skip_cta;
        if (!halo_fits) atomicOr(&ctl->status, ST_CONFIG);
        s_start = halo_fits && (c->done == DONE_RUNNING) && (c->status == 0) && nt <= t.ntcap;
        s_relres = c->relres;
        s_res2 = c->res2;
        s_resinf = c->resinf;
        s_keval = c->k_eval;
        s_stop = 0;
        s_epoch = 0;
        s_fail = 0;
        if (halo_fits) {
            for (int q = 0; q < STAGES; ++q) {
                mbar_init(&fmat[q], 1);
                mbar_init(&fx[q], 1);
                mbar_init(&empty[q], NW);
            }
            fence_mbar_init();
        }
    }
    // the CTA's tile table (constant for the launch)
    if (halo_fits && nt <= t.ntcap) {
        const int bbase = __ldg(t.blk0 + tb);
        for (int i = tid; i <= nt; i += blockDim.x) {
            s_row0[i] = __ldg(t.row0 + tb + i);
            s_nnz0[i] = __ldg(t.nnz0 + tb + i);
            s_boff[i] = __ldg(t.blk0 + tb + i) - bbase;
        }
        const int nblk = __ldg(t.blk0 + te) - bbase;
        const int4* gb = reinterpret_cast<const int4*>(t.blk) + bbase;
        for (int i = tid; i < nblk && i < t.blkcap; i += blockDim.x) s_blk[i] = __ldg(gb + i);
    }
    __syncthreads();
    if (!s_start) {
        if (tid == 0 && nt > t.ntcap) atomicOr(&ctl->status, ST_TIMEOUT);
        return;
    }

    int ksw = max_sweeps;
    if (!MIXED && !s_test) {
        const long long rem = s_klim - s_k;
        ksw = (int)(rem < (long long)ksw ? (rem > 0 ? rem : 0) : ksw);
    }
    const long long njobs = (long long)ksw * nt;
    const int inner = s_inner;
    const int phase0 = s_phase;
    const int xb0 = s_xb;
    const int emax = t.emax;
    const long long budget = s_timeout;

    // ================================================= producer warp
    if (warp == NW) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            long long jm = 0, jx = 0;
            int fenced_sweep = 0;     // x of sweep 0 was written before this launch
            long long t_last = clock64();
            while (jx < njobs) {
                bool prog = false;
                // (A) constant tile data, as far ahead as the stages allow
                if (jm < njobs) {
                    const int sidx = (int)(jm % STAGES);
                    const bool freed = jm < STAGES ||
                                       mbar_try_wait(&empty[sidx], (unsigned)(((jm / STAGES) - 1) & 1));
                    if (freed) {
                        const int sw = (int)(jm / nt);
                        const int i = (int)(jm - (long long)sw * nt);
                        const int ph = phase_of(MIXED, MIXED ? (phase0 + sw) % inner : 0, inner);
                        const bool fp64 = (ph == PH_P64 || ph == PH_P64R);
                        unsigned char* st = smem + sidx * L.bytes;
                        const int r0 = s_row0[i], r1 = s_row0[i + 1];
                        const int p0 = s_nnz0[i], p1 = s_nnz0[i + 1];
                        int* hdr = reinterpret_cast<int*>(st);
                        hdr[0] = r0; hdr[1] = r1; hdr[2] = p0; hdr[3] = p1;
                        const int4 h = s_blk[s_boff[i]];
                        const bool over = (p1 - p0) > emax;
                        unsigned bytes = 0;
                        int vb = 0, ve = 0, cb = 0, ce = 0;
                        if (!over) {
                            if (fp64) { vb = p0 & ~1; ve = (p1 + 1) & ~1; bytes += (unsigned)(ve - vb) * 8u; }
                            else { vb = p0 & ~3; ve = (p1 + 3) & ~3; bytes += (unsigned)(ve - vb) * 4u; }
                            cb = p0 & ~3; ce = (p1 + 3) & ~3;
                            bytes += (unsigned)(ce - cb) * 4u;
                        }
                        const int rb = r0 & ~3, re = (r1 + 1 + 3) & ~3;
                        bytes += (unsigned)(re - rb) * 4u;
                        const int hb = r0 & ~1, he = (r1 + 1) & ~1;
                        if (fp64) bytes += (unsigned)(he - hb) * 8u;
                        uint64_t* bar = &fmat[sidx];
                        mbar_expect_tx(bar, bytes);
                        // windowed tiles read tile-local columns, fallback tiles global ones
                        const int* colsrc = (h.w & 1) ? m.col : t.lcol;
                        if (!over) {
                            if (ve > vb) {
                                if (fp64) bulk_g2s(st + L.o_val, m.S64 + vb, (unsigned)(ve - vb) * 8u, bar, pol);
                                else bulk_g2s(st + L.o_val, m.S32 + vb, (unsigned)(ve - vb) * 4u, bar, pol);
                            }
                            if (ce > cb) bulk_g2s(st + L.o_col, colsrc + cb, (unsigned)(ce - cb) * 4u, bar, pol);
                        }
                        bulk_g2s(st + L.o_rp, m.rowptr + rb, (unsigned)(re - rb) * 4u, bar, pol);
                        if (fp64 && he > hb) bulk_g2s(st + L.o_c, m.b + hb, (unsigned)(he - hb) * 8u, bar, pol);
                        ++jm;
                        prog = true;
                    }
                }
                // (B) x halo of the oldest claimed job whose sweep's x is complete
                if (jx < jm) {
                    const int sw = (int)(jx / nt);
                    if (s_epoch >= sw) {
                        if (sw > fenced_sweep) {
                            // x of this sweep was written by other CTAs (generic proxy) before the
                            // grid barrier; order those writes before our bulk (async-proxy) reads
                            __threadfence();
                            fence_proxy_async_global();
                            fenced_sweep = sw;
                        }
                        const int sidx = (int)(jx % STAGES);
                        const int i = (int)(jx - (long long)sw * nt);
                        const int pos = MIXED ? (phase0 + sw) % inner : 0;
                        const int ph = phase_of(MIXED, pos, inner);
                        unsigned char* st = smem + sidx * L.bytes;
                        const int4* blk = s_blk + s_boff[i];
                        const int4 h = blk[0];
                        uint64_t* bar = &fx[sidx];
                        if (ph == PH_P64 || ph == PH_P64R) {
                            const double* xsrc = MIXED ? v.x[xb0] : v.x[(xb0 + sw) & 1];
                            mbar_expect_tx(bar, (unsigned)h.x * 8u);
                            for (int q = 1; q <= h.z; ++q) {
                                const int4 rn = blk[q];
                                bulk_g2s(st + L.o_x + rn.z * 8, xsrc + rn.x, (unsigned)rn.y * 8u, bar, 0);
                            }
                        } else {
                            const float* esrc = v.e[pos & 1];
                            mbar_expect_tx(bar, (unsigned)h.x * 4u);
                            for (int q = 1; q <= h.z; ++q) {
                                const int4 rn = blk[q];
                                bulk_g2s(st + L.o_x + rn.z * 4, esrc + rn.x, (unsigned)rn.y * 4u, bar, 0);
                            }
                        }
                        ++jx;
                        prog = true;
                    }
                }
                if (prog) {
                    t_last = clock64();
                } else {
                    if (s_stop) break;
                    if (clock64() - t_last > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
                }
            }
            // Drain: the copies of the last jobs must land before the CTA exits.
            const long long t0 = clock64();
            for (long long j = (jm > STAGES ? jm - STAGES : 0); j < jm; ++j) {
                const unsigned par = (unsigned)((j / STAGES) & 1);
                while (!mbar_try_wait(&fmat[(int)(j % STAGES)], par))
                    if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
                if (j < jx)
                    while (!mbar_try_wait(&fx[(int)(j % STAGES)], par))
                        if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
            }
        }
        return;
    }

    // ================================================= math warps
    long long k = s_k;
    int xb = xb0, pos = phase0;
    long long evals = s_evals, outer = s_outer;
    long long jc = 0;
    int nbar = 0;
    unsigned long long tr_comp = 0, tr_wait = 0, tr_mark = (tid == 0) ? global_ns() : 0;
    for (int sw = 0; sw < ksw; ++sw) {
        const int ph = phase_of(MIXED, pos, inner);
        const bool norm_ph = (ph == PH_P64 || ph == PH_P64R);
        double ss = 0.0;
        unsigned long long mx = 0;
        const double* xs = v.x[xb];
        double* xd = v.x[xb ^ 1];
        const float* es = v.e[pos & 1];
        float* ed = v.e[(pos + 1) & 1];
        for (int i = 0; i < nt; ++i, ++jc) {
            const int sidx = (int)(jc % STAGES);
            const unsigned par = (unsigned)((jc / STAGES) & 1);
            bool ok = true;
            for (int w = 0; w < 2 && ok; ++w) {
                uint64_t* bar = w == 0 ? &fmat[sidx] : &fx[sidx];
                if (!mbar_try_wait(bar, par)) {
                    if (s_fail) { ok = false; break; }
                    const long long t0 = clock64();
                    while (!mbar_try_wait(bar, par)) {
                        if (s_fail || clock64() - t0 > budget) {
                            if (!s_fail) atomicOr(&ctl->status, ST_TIMEOUT);
                            s_fail = 1;
                            ok = false;
                            break;
                        }
                    }
                }
            }
            if (ok) {
                const unsigned char* st = smem + sidx * L.bytes;
                const int r0 = s_row0[i], r1 = s_row0[i + 1], p0 = s_nnz0[i], p1 = s_nnz0[i + 1];
                const int4 h = s_blk[s_boff[i]];
                const bool over = (p1 - p0) > emax;
                const bool win = !(h.w & 1);
                const int r = r0 + tid;
                const bool in = r < r1;
                const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (r0 & ~3);
                const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (p0 & ~3);
                const int kb = in ? srp[r] : 0, ke = in ? srp[r + 1] : 0;
                if (norm_ph) {
                    const double* sv = reinterpret_cast<const double*>(st + L.o_val) - (p0 & ~1);
                    const double* sc = reinterpret_cast<const double*>(st + L.o_c) - (r0 & ~1);
                    const double* sx = reinterpret_cast<const double*>(st + L.o_x);
                    double acc = in ? sc[r] : 0.0;
                    double xi = 0.0;
                    double a1[1] = {acc};
                    const int kb1[1] = {kb}, len1[1] = {ke - kb};
                    if (win) {
                        xi = in ? sx[h.y + tid] : 0.0;
                        rows_dot<1>(a1, kb1, len1, [&](int e) { return sv[e]; }, [&](int e) { return sx[scol[e]]; });
                    } else {
                        xi = in ? __ldcg(xs + r) : 0.0;
                        if (!over)
                            rows_dot<1>(a1, kb1, len1, [&](int e) { return sv[e]; },
                                        [&](int e) { return __ldcg(xs + scol[e]); });
                        else
                            rows_dot<1>(a1, kb1, len1, [&](int e) { return __ldg(m.S64 + e); },
                                        [&](int e) { return __ldcg(xs + __ldg(m.col + e)); });
                    }
                    acc = a1[0];
                    if (in) {
                        if (ph == PH_P64) {
                            __stcg(xd + r, acc);
                        } else {
                            const float dl = (float)__dadd_rn(acc, -xi);
                            __stcg(v.dlt + r, dl);
                            __stcg(v.e[1] + r, dl);
                        }
                        accumulate_residual(acc, xi, ss, mx);
                    }
                } else {
                    const float* sv = reinterpret_cast<const float*>(st + L.o_val) - (p0 & ~3);
                    const float* sx = reinterpret_cast<const float*>(st + L.o_x);
                    float acc = in ? __ldcg(v.dlt + r) : 0.f;
                    float a1[1] = {acc};
                    const int kb1[1] = {kb}, len1[1] = {ke - kb};
                    if (win)
                        rows_dot<1>(a1, kb1, len1, [&](int e) { return sv[e]; }, [&](int e) { return sx[scol[e]]; });
                    else if (!over)
                        rows_dot<1>(a1, kb1, len1, [&](int e) { return sv[e]; },
                                    [&](int e) { return __ldcg(es + scol[e]); });
                    else
                        rows_dot<1>(a1, kb1, len1, [&](int e) { return __ldg(m.S32 + e); },
                                    [&](int e) { return __ldcg(es + __ldg(m.col + e)); });
                    acc = a1[0];
                    if (in) {
                        if (ph == PH_P32) __stcg(ed + r, acc);
                        else __stcg(v.x[xb] + r, __dadd_rn(__ldcg(v.x[xb] + r), (double)acc));
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[sidx]);
        }
        // ---- publish partial norms, grid barrier
        if (norm_ph) {
            const double ws = warp_sum(ss);
            const unsigned long long wm = warp_max(mx);
            if (lane == 0) { s_wss[warp] = ws; s_wmx[warp] = wm; }
        }
        consumer_sync<CT>();
        if (tid == 0) {
            const unsigned long long tb_ = global_ns();
            tr_comp += tb_ - tr_mark;
            tr_mark = tb_;
            if (norm_ph) {
                double b = 0.0;
                unsigned long long bm = 0;
                for (int w = 0; w < NW; ++w) { b += s_wss[w]; bm = umax64(bm, s_wmx[w]); }
                Partial* slot = v.part + (sw & 1) * v.nslots + blockIdx.x;
                __stcg(&slot->ss, b);
                __stcg(&slot->mx, bm);
            }
            __threadfence();
            if (!(s_skip == (int)blockIdx.x)) atomicAdd(&ctl->bar, 1ull);
            const unsigned long long target = (unsigned long long)(nbar + 1) * gridDim.x;
            const long long t0 = clock64();
            while (ld_acquire_u64(&ctl->bar) < target) {
                if (ld_volatile_i32(&ctl->status) & ST_TIMEOUT) { s_fail = 1; break; }
                if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; break; }
                __nanosleep(32);
            }
            {
                const unsigned long long tc_ = global_ns();
                tr_wait += tc_ - tr_mark;
                tr_mark = tc_;
            }
            __threadfence();
            if (!s_fail) s_epoch = nbar + 1;      // x of sweep nbar+1 is complete: the producer may copy it
        }
        ++nbar;
        consumer_sync<CT>();
        if (s_fail) break;
        // ---- convergence decision (identical in every CTA)
        if (norm_ph) {
            if (warp == 0) {
                double tss;
                unsigned long long tmx;
                reduce_partials_warp(v.part + (sw & 1) * v.nslots, gridDim.x, tss, tmx);
                if (lane == 0) {
                    const Decision d = decide(s_test, ctl->tol, s_klim, ctl->norm_kind, ctl->bnorm, tss, tmx, k);
                    s_relres = d.relres;
                    s_res2 = d.res2;
                    s_resinf = d.resinf;
                    s_keval = k;
                    s_dec_done = d.done;
                    if (d.numeric_bad && blockIdx.x == 0) atomicOr(&ctl->status, ST_NUMERIC);
                    if (blockIdx.x == 0 && ctl->hist && evals < ctl->hist_cap) ctl->hist[evals] = d.relres;
                }
            }
            consumer_sync<CT>();
            evals += 1;
            if (s_dec_done != DONE_RUNNING) { s_done = s_dec_done; break; }
            if (ph == PH_P64) { k += 1; xb ^= 1; }
            else pos = 1;
        } else if (ph == PH_P32) {
            pos += 1;
        } else {   // PH_P32L
            pos = 0;
            k += inner;
            outer += 1;
        }
        if (!MIXED && !s_test && k >= s_klim) break;
    }
    if (tid == 0 && v.trace) {
        atomicAdd(v.trace + 4 * blockIdx.x + 0, tr_comp);
        atomicAdd(v.trace + 4 * blockIdx.x + 1, tr_wait);
        atomicAdd(v.trace + 4 * blockIdx.x + 2, (unsigned long long)nbar);
    }
    if (tid == 0) s_stop = 1;
    if (blockIdx.x == 0 && tid == 0) {
        ctl->k = k;
        ctl->xbuf = xb;
        ctl->phase = pos;
        ctl->evals = evals;
        ctl->outer = outer;
        ctl->done = s_done;
        ctl->relres = s_relres;
        ctl->res2 = s_res2;
        ctl->resinf = s_resinf;
        ctl->k_eval = s_keval;
        __threadfence();
    }
}

template <int STAGES, bool MIXED>
static const void* halo_fn()
{
    return reinterpret_cast<const void*>(&k_halo<STAGES, MIXED>);
}

const void* halo_kernel(int stages, bool mixed)
{
    if (stages == 3) return mixed ? halo_fn<3, true>() : halo_fn<3, false>();
    if (stages == 4) return mixed ? halo_fn<4, true>() : halo_fn<4, false>();
    return nullptr;
}

// =========================================================================
// Small kernels: permutation in/out, right-hand side, control block, adjoint.
// =========================================================================

// dst[r*nrhs + c] = src[perm[r]*nrhs + c] (src may be NULL = zero)
// x (caller's row order) -> iterate y_r = a_rr x_perm(r) in the new order
// (d == nullptr: no scaling; src == nullptr: zero).
__global__ void k_gather_rows(const long long* __restrict__ perm, const double* __restrict__ src,
                              const double* __restrict__ d, double* __restrict__ dst, int n, int nrhs)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nrhs) return;
    const int r = (int)(idx / nrhs), c = (int)(idx - (long long)r * nrhs);
    const double v = src ? src[perm[r] * nrhs + c] : 0.0;
    dst[idx] = d ? __dmul_rn(d[r], v) : v;
}

// iterate y (new order) -> x_perm(r) = y_r / a_rr in the caller's order
// (IEEE division; d == nullptr: no scaling).
__global__ void k_scatter_rows(const long long* __restrict__ perm, const double* __restrict__ src,
                               const double* __restrict__ d, double* __restrict__ dst, int n, int nrhs)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nrhs) return;
    const int r = (int)(idx / nrhs), c = (int)(idx - (long long)r * nrhs);
    dst[perm[r] * nrhs + c] = d ? __ddiv_rn(src[idx], d[r]) : src[idx];
}

// The right-hand side in the new row order: b'_r = b_perm(r) (zero if b is NULL).
__global__ void k_gather_b(const long long* __restrict__ perm, const double* __restrict__ b, double* __restrict__ out,
                           int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const long long i = perm[r];
    out[r] = (b && i >= 0) ? b[i] : 0.0;
}

// ||b||_2 with a fixed reduction order (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_bnorm(const double* __restrict__ b, long long n, JacCtl* ctl)
{
    __shared__ double s[32];
    double acc = 0.0;
    if (b)
        for (long long i = threadIdx.x; i < n; i += 1024) acc = __fma_rn(b[i], b[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += s[w];
        ctl->bnorm = sqrt(t);
    }
}

__global__ void k_arm(JacCtl* ctl, int test, int mixed, int inner, long long k_limit, long long k_delta,
                      double tol, int norm_kind, double* hist, long long hist_cap, long long timeout, int skip)
{
    JacCtl* c = ctl;
    c->inner = inner < 2 ? 2 : inner;
    c->bar = 0;
    c->ticket = 0;
    c->status = 0;
    c->done = DONE_RUNNING;
    c->test = test;
    c->mixed = mixed;
    c->phase = 0;
    c->k_limit = (k_delta >= 0) ? c->k + k_delta : k_limit;
    c->evals = 0;
    c->outer = 0;
    c->tol = tol;
    c->norm_kind = norm_kind;
    c->hist = hist;
    c->hist_cap = hist_cap;
    c->timeout = timeout;
    c->fault_skip_cta = skip;
    c->loc_part = -1;
    c->loc_val = 0.0;
}

__global__ void k_reset_iterate(JacCtl* ctl)
{
    ctl->k = 0;
    ctl->xbuf = 0;
    ctl->phase = 0;
    ctl->k_eval = -1;
    ctl->relres = 0.0;
    ctl->res2 = 0.0;
    ctl->resinf = 0.0;
}

// dA[e] = -lambda_i x_j over the stored pattern of A (original order).
__global__ void k_adjoint_grad(const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ lam, const double* __restrict__ x,
                               double* __restrict__ dA, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double li = lam[i];
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) dA[e] = -(li * x[col[e]]);
}

// --------------------------------------------------------------- launchers

cudaError_t launch_row_sweep(int ph, const DevMat& m, const DevVec& v, JacCtl* ctl, cudaStream_t s)
{
    const int blocks = (m.n + 255) / 256;
    switch (ph) {
    case PH_P64: k_row_sweep<PH_P64><<<blocks, 256, 0, s>>>(m, v, ctl); break;
    case PH_P64R: k_row_sweep<PH_P64R><<<blocks, 256, 0, s>>>(m, v, ctl); break;
    case PH_P32: k_row_sweep<PH_P32><<<blocks, 256, 0, s>>>(m, v, ctl); break;
    default: k_row_sweep<PH_P32L><<<blocks, 256, 0, s>>>(m, v, ctl); break;
    }
    return cudaGetLastError();
}

template <int RPT, int STAGES, bool MIXED, int NWM, int LPR = 1, int SYNC = 0, int PART = 0>
static const void* persistent_fn()
{
    return reinterpret_cast<const void*>(&k_persistent<RPT, STAGES, MIXED, NWM, LPR, SYNC, PART>);
}

template <int STAGES, bool MIXED, int SYNC, int PART = 0>
static const void* persistent_fn_lanes(int lanes)
{
    switch (lanes) {
    case 1: return persistent_fn<1, STAGES, MIXED, 8, 1, SYNC, PART>();
    case 2: return persistent_fn<1, STAGES, MIXED, 8, 2, SYNC, PART>();
    case 4: return persistent_fn<1, STAGES, MIXED, 8, 4, SYNC, PART>();
    case 8:
        if constexpr (SYNC >= 3) return nullptr;   // split layouts and local stopping use 1, 2 or 4 lanes
        else return persistent_fn<1, STAGES, MIXED, 8, 8, SYNC, PART>();
    default: return nullptr;
    }
}

// The two launches of a mixed cycle (part 1: FP64 pass, 2: FP32 sweeps).
template <int STAGES>
static const void* mixed_fn_lanes(int lanes, int part)
{
    return part == 1 ? persistent_fn_lanes<STAGES, true, 0, 1>(lanes)
                     : part == 2 ? persistent_fn_lanes<STAGES, true, 0, 2>(lanes) : nullptr;
}

// threads = 32 x math warps: 224 -> 7 (2 CTAs/SM, 128 regs),
// 256 -> 8 (2 CTAs/SM, 96 regs; or 3 stages, 72 regs, 3 CTAs/SM),
// 480 -> 15 (1 CTA/SM, 128 regs).  lanes = lanes per row (256 threads only);
// a tile then holds threads / lanes rows.  sync = 0 grid barrier, 1 neighbour
// flags, 2 asynchronous relaxation (1 and 2: 256 threads, FP64 only), 3 grid
// barrier over a split interface layout (256 threads, FP64, lanes 1, 2, 4),
// 4 grid barrier with the local stopping tests (256 threads, FP64, lanes 1, 2, 4).
const void* persistent_kernel(int threads, int stages, bool mixed, int lanes, int sync, int part)
{
    if (mixed != (part != 0)) return nullptr;   // mixed solves run as split cycles
    if (sync == 3) {
        // grid barrier with a split interface block: FP64, 256 threads, 1/2/4 lanes
        if (mixed || threads != 256 || (lanes != 1 && lanes != 2 && lanes != 4)) return nullptr;
        switch (stages) {
        case 2: return persistent_fn_lanes<2, false, 3>(lanes);
        case 3: return persistent_fn_lanes<3, false, 3>(lanes);
        case 4: return persistent_fn_lanes<4, false, 3>(lanes);
        default: return nullptr;
        }
    }
    if (sync == 4) {
        // grid barrier with local stopping tests: FP64, 256 threads, 1/2/4 lanes
        if (mixed || threads != 256 || (lanes != 1 && lanes != 2 && lanes != 4)) return nullptr;
        switch (stages) {
        case 2: return persistent_fn_lanes<2, false, 4>(lanes);
        case 3: return persistent_fn_lanes<3, false, 4>(lanes);
        case 4: return persistent_fn_lanes<4, false, 4>(lanes);
        default: return nullptr;
        }
    }
    if (sync == 1 || sync == 2) {
        if (mixed || threads != 256) return nullptr;
        // every stage count gets its own instantiation: the kernel's stage
        // layout must match the shared memory the launch provides
        switch (stages * 4 + sync) {
        case 2 * 4 + 1: return persistent_fn_lanes<2, false, 1>(lanes);
        case 3 * 4 + 1: return persistent_fn_lanes<3, false, 1>(lanes);
        case 4 * 4 + 1: return persistent_fn_lanes<4, false, 1>(lanes);
        case 2 * 4 + 2: return persistent_fn_lanes<2, false, 2>(lanes);
        case 3 * 4 + 2: return persistent_fn_lanes<3, false, 2>(lanes);
        case 4 * 4 + 2: return persistent_fn_lanes<4, false, 2>(lanes);
        default: return nullptr;
        }
    }
    if (sync != 0) return nullptr;
    if (threads == 256 && stages == 3)
        return mixed ? mixed_fn_lanes<3>(lanes, part) : persistent_fn_lanes<3, false, 0>(lanes);
    if (threads == 256 && stages == 2)
        return mixed ? mixed_fn_lanes<2>(lanes, part) : persistent_fn_lanes<2, false, 0>(lanes);
    if (stages != 4) return nullptr;
    if (threads == 256)
        return mixed ? mixed_fn_lanes<4>(lanes, part) : persistent_fn_lanes<4, false, 0>(lanes);
    if (lanes != 1) return nullptr;
    if (threads == 224)
        return mixed ? (part == 1 ? persistent_fn<1, 4, true, 7, 1, 0, 1>() : persistent_fn<1, 4, true, 7, 1, 0, 2>())
                     : persistent_fn<1, 4, false, 7>();
    if (threads == 480)
        return mixed ? (part == 1 ? persistent_fn<1, 4, true, 15, 1, 0, 1>() : persistent_fn<1, 4, true, 15, 1, 0, 2>())
                     : persistent_fn<1, 4, false, 15>();
    return nullptr;
}

int persistent_threads(int rows) { return rows + 32; }

cudaError_t launch_persistent(const void* fn, int grid, int threads, int smem, const DevMat& m, const DevVec& v,
                              const DevTiles& t, JacCtl* ctl, int max_sweeps, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {(void*)&m, (void*)&v, (void*)&t, (void*)&ctl, (void*)&max_sweeps};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t launch_gather_rows(const long long* perm, const double* src, const double* d, double* dst, int n,
                               int nrhs, cudaStream_t s)
{
    const long long tot = (long long)n * nrhs;
    k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(perm, src, d, dst, n, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows(const long long* perm, const double* src, const double* d, double* dst, int n,
                                int nrhs, cudaStream_t s)
{
    const long long tot = (long long)n * nrhs;
    k_scatter_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(perm, src, d, dst, n, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_gather_b(const long long* perm, const double* b, double* out, int nout, int nb, JacCtl* ctl,
                            cudaStream_t s)
{
    k_gather_b<<<(nout + 255) / 256, 256, 0, s>>>(perm, b, out, nout);
    k_bnorm<<<1, 1024, 0, s>>>(b, nb, ctl);
    return cudaGetLastError();
}

cudaError_t launch_arm(JacCtl* ctl, int test, int mixed, int inner, long long k_limit, long long k_delta,
                       double tol, int norm_kind, double* hist, long long hist_cap, long long timeout, int skip,
                       cudaStream_t s)
{
    k_arm<<<1, 1, 0, s>>>(ctl, test, mixed, inner, k_limit, k_delta, tol, norm_kind, hist, hist_cap, timeout, skip);
    return cudaGetLastError();
}

cudaError_t launch_reset_iterate(JacCtl* ctl, cudaStream_t s)
{
    k_reset_iterate<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

cudaError_t launch_reset_bar(JacCtl* ctl, cudaStream_t s)
{
    // bar, dec_ready and arrive[] are contiguous
    return cudaMemsetAsync(&ctl->bar, 0, offsetof(JacCtl, ticket) - offsetof(JacCtl, bar), s);
}

cudaError_t launch_adjoint_grad(const int* rowptr, const int* col, const double* lam, const double* x,
                                double* dA, int n, cudaStream_t s)
{
    k_adjoint_grad<<<(n + 255) / 256, 256, 0, s>>>(rowptr, col, lam, x, dA, n);
    return cudaGetLastError();
}

}  // namespace jac
