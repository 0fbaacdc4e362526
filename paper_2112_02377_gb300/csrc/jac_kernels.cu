// Sweep kernels of the GB300 Jacobi library.
//
// Both kernels evaluate, for every row i of the (reordered) matrix,
//   x'_i = c_i + sum_{j != i} T_ij x_j          (Sec. 3, Eq. (3.4) with
//                                                 T = -D^{-1}(L+U), c = D^{-1} b)
//   r_i  = a_ii (x'_i - x_i)  = (b - A x)_i      (Algorithm 1's residual of x^k)
// and fuse the reductions sum r_i^2 and max |r_i| (Algorithm 1's norm; the
// paper's dot products use MPI_ALLREDUCE, Sec. 4.2.2, here a grid reduction).
// The off-diagonal terms of a row are accumulated by one thread in the stored
// order with fused multiply-adds, so the iterate depends only on the row and
// never on the splitting, tiling or CTA that computes it.
#include <cuda_runtime.h>

#include "jac_device.cuh"
#include "jac_launch.h"

namespace jac {

constexpr int CHUNK = 8;   // off-diagonal entries whose x loads are issued together

// ------------------------------------------------------------ row math -----

// FP64 row: acc = c + sum T x (stored order).  tv/cv read through `ldt`/`ldc`.
template <class LdT, class LdC>
__device__ __forceinline__ double row_dot64(double acc, int kb, int ke, const double* __restrict__ xs,
                                            LdT ldt, LdC ldc)
{
    for (int kk = kb; kk < ke; kk += CHUNK) {
        double tv[CHUNK], xv[CHUNK];
#pragma unroll
        for (int u = 0; u < CHUNK; ++u) {
            if (kk + u < ke) {
                tv[u] = ldt(kk + u);
                xv[u] = __ldcg(xs + ldc(kk + u));
            }
        }
#pragma unroll
        for (int u = 0; u < CHUNK; ++u)
            if (kk + u < ke) acc = __fma_rn(tv[u], xv[u], acc);
    }
    return acc;
}

template <class LdT, class LdC>
__device__ __forceinline__ float row_dot32(float acc, int kb, int ke, const float* __restrict__ es, LdT ldt,
                                           LdC ldc)
{
    for (int kk = kb; kk < ke; kk += CHUNK) {
        float tv[CHUNK], ev[CHUNK];
#pragma unroll
        for (int u = 0; u < CHUNK; ++u) {
            if (kk + u < ke) {
                tv[u] = ldt(kk + u);
                ev[u] = __ldcg(es + ldc(kk + u));
            }
        }
#pragma unroll
        for (int u = 0; u < CHUNK; ++u)
            if (kk + u < ke) acc = __fmaf_rn(tv[u], ev[u], acc);
    }
    return acc;
}

// Residual bookkeeping of one row from its update.
__device__ __forceinline__ void accumulate_residual(double xnew, double xold, double di, double& ss,
                                                    unsigned long long& mx)
{
    const double dl = __dadd_rn(xnew, -xold);
    const double r = __dmul_rn(di, dl);
    ss = __fma_rn(r, r, ss);
    mx = umax64(mx, abs_bits(r));
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
            const double acc = row_dot64(__ldg(m.c + i), kb, ke, xs, [&](int k) { return __ldg(m.T64 + k); }, ldc);
            if (PH == PH_P64) {
                v.x[xb ^ 1][i] = acc;
            } else {
                const float dl = (float)__dadd_rn(acc, -xi);
                v.dlt[i] = dl;
                v.e[1][i] = dl;
            }
            accumulate_residual(acc, xi, __ldg(m.d + i), ss, mx);
        } else {
            const int j = s_phase;   // inner step: e_j -> e_{j+1}
            const float* es = v.e[j & 1];
            const float acc = row_dot32(__ldcg(v.dlt + i), kb, ke, es, [&](int k) { return __ldg(m.T32 + k); }, ldc);
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
// x is gathered with ld.global.cg (it changes every sweep; L1 is not coherent).
// After each sweep the CTAs publish partial norms, pass a bounded grid barrier
// and each reduces all partials in the same fixed order, so every CTA takes
// the same convergence decision.
// =========================================================================

struct StageLayout {
    int o_val, o_col, o_rp, o_c, o_d, bytes;
};

__host__ __device__ inline StageLayout stage_layout(int rows, int emax)
{
    auto up = [](int v) { return (v + 127) & ~127; };
    StageLayout L;
    L.o_val = 128;                                  // 16-byte header (r0, r1, p0, p1) in the first line
    L.o_col = L.o_val + up((emax + 4) * 8);
    L.o_rp = L.o_col + up((emax + 8) * 4);
    L.o_c = L.o_rp + up((rows + 12) * 4);
    L.o_d = L.o_c + up((rows + 4) * 8);
    L.bytes = L.o_d + up((rows + 4) * 8);
    return L;
}

int persistent_smem_bytes(int rows, int emax, int stages)
{
    return stages * stage_layout(rows, emax).bytes + 2 * stages * 8 + 64;
}

__device__ __forceinline__ int phase_of(bool mixed, int pos, int inner)
{
    if (!mixed) return PH_P64;
    if (pos == 0) return PH_P64R;
    return pos == inner - 1 ? PH_P32L : PH_P32;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

// RPT rows of one thread: acc[q] = acc[q] + sum_k T_k x_col(k), entries of each
// row in stored order.  The L2 gathers of a chunk of every row are issued
// before the chunk's FMAs; T is read at the FMA (shared memory, short latency).
template <int RPT, class Real, class LdT, class LdC>
__device__ __forceinline__ void rows_dot(Real (&acc)[RPT], const int (&kb)[RPT], const int (&len)[RPT],
                                         const Real* __restrict__ xs, LdT ldt, LdC ldc)
{
    int lmax = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) lmax = len[q] > lmax ? len[q] : lmax;
    for (int o = 0; o < lmax; o += CHUNK) {
        Real xv[RPT][CHUNK];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
#pragma unroll
            for (int u = 0; u < CHUNK; ++u)
                if (o + u < len[q]) xv[q][u] = __ldcg(xs + ldc(kb[q] + o + u));
        }
#pragma unroll
        for (int u = 0; u < CHUNK; ++u) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                if (o + u < len[q]) {
                    if constexpr (sizeof(Real) == 8) acc[q] = __fma_rn(ldt(kb[q] + o + u), xv[q][u], acc[q]);
                    else acc[q] = __fmaf_rn(ldt(kb[q] + o + u), xv[q][u], acc[q]);
                }
            }
        }
    }
}

template <int RPT, int STAGES, bool MIXED>
__global__ void __launch_bounds__(288) __maxnreg__(RPT == 1 ? 96 : 168)
k_persistent(DevMat m, DevVec v, DevTiles t, JacCtl* ctl, int max_sweeps)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CT = 256, NW = 8, ROWS = CT * RPT;
    const StageLayout L = stage_layout(ROWS, t.emax);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L.bytes);
    uint64_t* empty = full + STAGES;
    __shared__ double s_wss[NW];
    __shared__ unsigned long long s_wmx[NW];
    __shared__ long long s_k, s_klim, s_evals, s_outer, s_timeout, s_keval;
    __shared__ int s_xb, s_phase, s_inner, s_test, s_done, s_start, s_skip, s_fail, s_dec_done;
    __shared__ volatile int s_stop;
    __shared__ double s_relres, s_res2, s_resinf;

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
        s_start = (c->done == DONE_RUNNING) && (c->status == 0);
        s_relres = c->relres;
        s_res2 = c->res2;
        s_resinf = c->resinf;
        s_keval = c->k_eval;
        s_stop = 0;
        s_fail = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (!s_start) return;

    const int tb = t.cta0[blockIdx.x], te = t.cta0[blockIdx.x + 1], nt = te - tb;
    int ksw = max_sweeps;
    if (!MIXED && !s_test) {
        const long long rem = s_klim - s_k;
        ksw = (int)(rem < (long long)ksw ? (rem > 0 ? rem : 0) : ksw);
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
                const int ti = tb + (int)(j - (long long)sw * nt);
                const int ph = phase_of(MIXED, MIXED ? (phase0 + sw) % inner : 0, inner);
                const bool fp64 = (ph == PH_P64 || ph == PH_P64R);
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
                if (fp64) bytes += 2u * (unsigned)(he - hb) * 8u;
                uint64_t* bar = &full[sidx];
                mbar_expect_tx(bar, bytes);
                if (!over) {
                    if (ve > vb) {
                        if (fp64) bulk_g2s(st + L.o_val, m.T64 + vb, (unsigned)(ve - vb) * 8u, bar, pol);
                        else bulk_g2s(st + L.o_val, m.T32 + vb, (unsigned)(ve - vb) * 4u, bar, pol);
                    }
                    if (ce > cb) bulk_g2s(st + L.o_col, m.col + cb, (unsigned)(ce - cb) * 4u, bar, pol);
                }
                bulk_g2s(st + L.o_rp, m.rowptr + rb, (unsigned)(re - rb) * 4u, bar, pol);
                if (fp64 && he > hb) {
                    bulk_g2s(st + L.o_c, m.c + hb, (unsigned)(he - hb) * 8u, bar, pol);
                    bulk_g2s(st + L.o_d, m.d + hb, (unsigned)(he - hb) * 8u, bar, pol);
                }
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
            uint64_t* bar = &full[sidx];
            const unsigned par = (unsigned)((jc / STAGES) & 1);
            bool ok = mbar_try_wait(bar, par);
            if (!ok && !s_fail) {
                const long long t0 = clock64();
                while (!(ok = mbar_try_wait(bar, par))) {
                    if (s_fail) break;
                    if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; break; }
                }
            }
            if (ok) {
                const unsigned char* st = smem + sidx * L.bytes;
                const int* hdr = reinterpret_cast<const int*>(st);
                const int r0 = hdr[0], r1 = hdr[1], p0 = hdr[2], p1 = hdr[3];
                const bool over = (p1 - p0) > emax;
                const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (r0 & ~3);
                const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (p0 & ~3);
                int r[RPT], kb[RPT], len[RPT];
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    r[q] = r0 + tid + CT * q;
                    const bool in = r[q] < r1;
                    kb[q] = in ? srp[r[q]] : 0;
                    len[q] = in ? srp[r[q] + 1] - kb[q] : 0;
                }
                if (norm_ph) {
                    const double* sv = reinterpret_cast<const double*>(st + L.o_val) - (p0 & ~1);
                    const double* sc = reinterpret_cast<const double*>(st + L.o_c) - (r0 & ~1);
                    const double* sd = reinterpret_cast<const double*>(st + L.o_d) - (r0 & ~1);
                    double xi[RPT], acc[RPT];
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        const bool in = r[q] < r1;
                        xi[q] = in ? __ldcg(xs + r[q]) : 0.0;
                        acc[q] = in ? sc[r[q]] : 0.0;
                    }
                    if (!over)
                        rows_dot<RPT>(acc, kb, len, xs, [&](int e) { return sv[e]; }, [&](int e) { return scol[e]; });
                    else
                        rows_dot<RPT>(acc, kb, len, xs, [&](int e) { return __ldg(m.T64 + e); },
                                      [&](int e) { return __ldg(m.col + e); });
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        if (r[q] < r1) {
                            if (ph == PH_P64) {
                                __stcg(xd + r[q], acc[q]);
                            } else {
                                const float dl = (float)__dadd_rn(acc[q], -xi[q]);
                                __stcg(v.dlt + r[q], dl);
                                __stcg(v.e[1] + r[q], dl);
                            }
                            accumulate_residual(acc[q], xi[q], sd[r[q]], ss, mx);
                        }
                    }
                } else {
                    const float* sv = reinterpret_cast<const float*>(st + L.o_val) - (p0 & ~3);
                    float acc[RPT];
#pragma unroll
                    for (int q = 0; q < RPT; ++q) acc[q] = r[q] < r1 ? __ldcg(v.dlt + r[q]) : 0.f;
                    if (!over)
                        rows_dot<RPT>(acc, kb, len, es, [&](int e) { return sv[e]; }, [&](int e) { return scol[e]; });
                    else
                        rows_dot<RPT>(acc, kb, len, es, [&](int e) { return __ldg(m.T32 + e); },
                                      [&](int e) { return __ldg(m.col + e); });
#pragma unroll
                    for (int q = 0; q < RPT; ++q) {
                        if (r[q] < r1) {
                            if (ph == PH_P32) __stcg(ed + r[q], acc[q]);
                            else __stcg(v.x[xb] + r[q], __dadd_rn(__ldcg(v.x[xb] + r[q]), (double)acc[q]));
                        }
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
        consumer_sync();
        if (tid == 0) {
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
            __threadfence();
        }
        ++nbar;
        consumer_sync();
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
            consumer_sync();
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
    // tell the producer to stop issuing; it drains its copies before exiting
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

// =========================================================================
// Small kernels: permutation in/out, right-hand side, control block, adjoint.
// =========================================================================

// dst[r*nrhs + c] = src[perm[r]*nrhs + c] (src may be NULL = zero)
__global__ void k_gather_rows(const long long* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst, int n, int nrhs)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nrhs) return;
    const int r = (int)(idx / nrhs), c = (int)(idx - (long long)r * nrhs);
    dst[idx] = src ? src[perm[r] * nrhs + c] : 0.0;
}

__global__ void k_scatter_rows(const long long* __restrict__ perm, const double* __restrict__ src,
                               double* __restrict__ dst, int n, int nrhs)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nrhs) return;
    const int r = (int)(idx / nrhs), c = (int)(idx - (long long)r * nrhs);
    dst[perm[r] * nrhs + c] = src[idx];
}

// c_r = b_perm(r) / a_rr  (IEEE division, as Algorithm 1's D^{-1} "computed once").
__global__ void k_make_c(const long long* __restrict__ perm, const double* __restrict__ b,
                         const double* __restrict__ d, double* __restrict__ c, int n)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    c[r] = b ? __ddiv_rn(b[perm[r]], d[r]) : 0.0;
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

template <int RPT, int STAGES, bool MIXED>
static const void* persistent_fn()
{
    return reinterpret_cast<const void*>(&k_persistent<RPT, STAGES, MIXED>);
}

const void* persistent_kernel(int rows, int stages, bool mixed)
{
    if (rows == 256 && stages == 4) return mixed ? persistent_fn<1, 4, true>() : persistent_fn<1, 4, false>();
    if (rows == 512 && stages == 4) return mixed ? persistent_fn<2, 4, true>() : persistent_fn<2, 4, false>();
    if (rows == 512 && stages == 3) return mixed ? persistent_fn<2, 3, true>() : persistent_fn<2, 3, false>();
    return nullptr;
}

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

cudaError_t launch_gather_rows(const long long* perm, const double* src, double* dst, int n, int nrhs,
                               cudaStream_t s)
{
    const long long tot = (long long)n * nrhs;
    k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(perm, src, dst, n, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows(const long long* perm, const double* src, double* dst, int n, int nrhs,
                                cudaStream_t s)
{
    const long long tot = (long long)n * nrhs;
    k_scatter_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(perm, src, dst, n, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_make_c(const long long* perm, const double* b, const double* d, double* c, int n,
                          JacCtl* ctl, cudaStream_t s)
{
    k_make_c<<<(n + 255) / 256, 256, 0, s>>>(perm, b, d, c, n);
    k_bnorm<<<1, 1024, 0, s>>>(b, n, ctl);
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
    return cudaMemsetAsync(&ctl->bar, 0, sizeof(unsigned long long), s);
}

cudaError_t launch_adjoint_grad(const int* rowptr, const int* col, const double* lam, const double* x,
                                double* dA, int n, cudaStream_t s)
{
    k_adjoint_grad<<<(n + 255) / 256, 256, 0, s>>>(rowptr, col, lam, x, dA, n);
    return cudaGetLastError();
}

}  // namespace jac
