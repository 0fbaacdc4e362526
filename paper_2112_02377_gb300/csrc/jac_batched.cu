// Batched solves: many independent systems, each with NRHS right-hand sides,
// in one persistent launch.
//
// The systems are packed as one block-diagonal matrix (rows of system s are
// [off_s, off_{s+1})); row tiles never cross a system.  Every sweep is the
// synchronous Jacobi sweep of Sec. 3 applied to all right-hand sides of every
// active system at once, so each matrix entry read from HBM serves NRHS
// updates.  Each system, and each of its right-hand sides, keeps its own
// residual norm and stopping test (Algorithm 1): a right-hand side stops at
// its first iterate whose test value is <= tol (that iterate is kept), and a
// system whose right-hand sides have all stopped is skipped from then on.
//
// Norms: every CTA reduces the rows it owns of a system into a per-(CTA,
// system) partial; the last CTA to finish a system in a sweep (an atomic
// arrival count) reduces that system's partials in CTA order -- a fixed
// order -- and takes the system's decisions, which the grid barrier at the
// end of the sweep publishes.
#include <cuda_runtime.h>

#include "jac_device.cuh"
#include "jac_launch.h"

namespace jac {

// Entries per row whose NRHS-wide x gathers are issued together: 3 in the
// FP64 sweeps (bound by the FP64 pipe; more would spill at 128 registers),
// 6 in the FP32 inner sweeps, which are bound by L2 gather latency and run in
// a kernel of their own (a 7-point row's gathers in one round trip).
template <class Real>
constexpr int bchunk() { return sizeof(Real) == 4 ? 6 : 3; }

__device__ __forceinline__ void b_consumer_sync(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive_b(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Gathered entries per row the FP32 launch copies ahead (a 7-point row has 6).
constexpr int GMAXE = 6;

// Shared memory of the FP32 launch's two gather buffers (4 right-hand sides).
__host__ __device__ constexpr int batched_gather_bytes(int rows, int nrhs, int part)
{
    return (part == 2 && nrhs == 4) ? 2 * GMAXE * rows * 16 : 0;
}

struct BStageLayout {
    int o_val, o_col, o_rp, o_c, bytes;   // o_c: the tile's b, NRHS per row (FP64 phases)
};

// fp32: the stages of the FP32-sweep launch of a mixed cycle (4-byte values,
// no right-hand side)
__host__ __device__ inline BStageLayout bstage_layout(int rows, int emax, int nrhs, bool fp32 = false)
{
    auto up = [](int v) { return (v + 127) & ~127; };
    BStageLayout L;
    L.o_val = 128;
    L.o_col = L.o_val + up((emax + 4) * (fp32 ? 4 : 8));
    L.o_rp = L.o_col + up((emax + 8) * 4);
    L.o_c = L.o_rp + up((rows + 12) * 4);
    L.bytes = L.o_c + (fp32 ? 0 : up((rows + 4) * nrhs * 8));
    return L;
}

int batched_smem_bytes(int rows, int emax, int nrhs, int stages, bool fp32)
{
    return stages * bstage_layout(rows, emax, nrhs, fp32).bytes + batched_gather_bytes(rows, nrhs, fp32 ? 2 : 0) +
           2 * stages * 8 + 64;
}

// Loads of a row's NRHS values.  L1 = false: L2 only (ld.global.cg).  L1 =
// true, for the iterate gathers of a sweep: cached in L1 too (ld.global.ca).
// A sweep reads an iterate buffer that nobody writes during the sweep, after
// the grid barrier whose release/acquire pair (atomic arrive, ld.acquire.gpu
// and fences by each CTA's thread 0, then a CTA barrier) makes the previous
// sweep's stores visible to these weak loads under the PTX memory model.
template <bool L1, class T>
__device__ __forceinline__ T ld_b(const T* p)
{
    if constexpr (L1) return __ldca(p);
    else return __ldcg(p);
}

template <int NRHS, bool L1 = false>
__device__ __forceinline__ void load_rhs(const double* p, double (&v)[NRHS])
{
    if constexpr (NRHS % 2 == 0) {
#pragma unroll
        for (int q = 0; q < NRHS; q += 2) {
            const double2 t = ld_b<L1>(reinterpret_cast<const double2*>(p) + q / 2);
            v[q] = t.x;
            v[q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) v[q] = ld_b<L1>(p + q);
    }
}

template <int NRHS, bool L1 = false>
__device__ __forceinline__ void load_rhs(const float* p, float (&v)[NRHS])
{
    if constexpr (NRHS == 4) {
        const float4 t = ld_b<L1>(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (NRHS == 2) {
        const float2 t = ld_b<L1>(reinterpret_cast<const float2*>(p));
        v[0] = t.x; v[1] = t.y;
    } else {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) v[q] = ld_b<L1>(p + q);
    }
}

// 16-byte asynchronous copy global -> shared, cached in L2 only, and its group
// operations.  (Through L1 as well, cp.async.ca, the FP32 sweeps of a mixed
// batched solve took 8 % longer: the gathers land in shared memory anyway.)
__device__ __forceinline__ void cp_async16_cg(void* dst_smem, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NRHS>
__device__ __forceinline__ void store_rhs(float* p, const float (&v)[NRHS])
{
    if constexpr (NRHS == 4) {
        __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    } else if constexpr (NRHS == 2) {
        __stcg(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    } else {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) __stcg(p + q, v[q]);
    }
}

template <int NRHS>
__device__ __forceinline__ void store_rhs(double* p, const double (&v)[NRHS])
{
    if constexpr (NRHS % 2 == 0) {
#pragma unroll
        for (int q = 0; q < NRHS; q += 2) __stcg(reinterpret_cast<double2*>(p) + q / 2, make_double2(v[q], v[q + 1]));
    } else {
#pragma unroll
        for (int q = 0; q < NRHS; ++q) __stcg(p + q, v[q]);
    }
}

// acc[q] += sum_k T_k x[col_k][q] for the row's entries in stored order.
template <int NRHS, class Real, class LdT, class LdC>
__device__ __forceinline__ void brow_dot(Real (&acc)[NRHS], int kb, int len, const Real* __restrict__ xs, LdT ldt,
                                         LdC ldc)
{
    constexpr int BCHUNK = bchunk<Real>();
    int lmax = (int)__reduce_max_sync(__activemask(), (unsigned)len);
    for (int o = 0; o < lmax; o += BCHUNK) {
        Real xv[BCHUNK][NRHS];
#pragma unroll
        for (int u = 0; u < BCHUNK; ++u)
            if (o + u < len) load_rhs<NRHS, true>(xs + (size_t)ldc(kb + o + u) * NRHS, xv[u]);
#pragma unroll
        for (int u = 0; u < BCHUNK; ++u) {
            if (o + u >= lmax) break;
            if (o + u < len) {
                const Real t = ldt(kb + o + u);
#pragma unroll
                for (int q = 0; q < NRHS; ++q) {
                    if constexpr (sizeof(Real) == 8) acc[q] = __fma_rn(t, xv[u][q], acc[q]);
                    else acc[q] = __fmaf_rn(t, xv[u][q], acc[q]);
                }
            }
        }
    }
}

// PART: 0 = every phase of the launch's sweeps; for the mixed cycle, 1 = its
// FP64 residual pass only, 2 = its FP32 inner sweeps only.  A mixed graph step
// alternates a PART 1 and a PART 2 launch per cycle, so the FP32 sweeps run in
// a kernel without the FP64 code and its registers.  The FP32 sweeps are bound
// by the latency of the iterate gathers (the iterates outgrow L2) and the
// registers that hold them cap the loads in flight.  With 4 right-hand sides
// (16-byte iterate rows) PART 2 therefore gathers through shared memory: each
// thread starts the cp.async copies of its row's entries in tile i+1 before it
// sums its row of tile i, twice the loads in flight at the same occupancy and
// without registers held; its stages hold FP32 data only.
template <int NRHS, int STAGES, bool MIXED, int NWM, int PART = 0>
__global__ void __maxnreg__(128)
k_batched(DevMat m, DevVec v, DevTiles t, DevBatch bt, JacCtl* ctl, int max_sweeps)
{
    static_assert(PART == 0 || MIXED, "the split cycle is for mixed solves");
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CT = NWM * 32, NW = NWM, ROWS = CT;
    const BStageLayout L = bstage_layout(ROWS, t.emax, NRHS, PART == 2);
    // the FP32 launch with 4 right-hand sides: two gather buffers after the stages
    constexpr int GBYTES = batched_gather_bytes(ROWS, NRHS, PART);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * L.bytes + GBYTES);
    uint64_t* empty = full + STAGES;
    __shared__ double s_wss[NW][NRHS];
    __shared__ unsigned long long s_wmx[NW][NRHS];
    __shared__ long long s_k, s_klim, s_evals, s_outer, s_timeout;
    __shared__ int s_xb, s_phase, s_inner, s_test, s_start, s_fail, s_stop_all, s_norm, s_blast;
    __shared__ double s_tol;
    __shared__ volatile int s_stop;

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
        s_tol = c->tol;
        s_norm = c->norm_kind;
        // the stages and their barriers must fit the dynamic shared memory of the launch
        const bool fits = (unsigned long long)STAGES * L.bytes + GBYTES + 2ull * STAGES * 8 <= dynamic_smem_bytes();
        if (!fits) atomicOr(&ctl->status, ST_CONFIG);
        s_start = fits && (c->done == DONE_RUNNING) && (c->status == 0);
        s_stop = 0;
        s_fail = 0;
        s_stop_all = 0;
        if (fits) {
            for (int q = 0; q < STAGES; ++q) {
                mbar_init(&full[q], 1);
                mbar_init(&empty[q], NW);
            }
            fence_mbar_init();
        }
    }
    __syncthreads();
    if (!s_start) return;

    const int tb = t.cta0[blockIdx.x], te = t.cta0[blockIdx.x + 1], nt = te - tb;
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
    const int inner = s_inner, phase0 = s_phase, emax = t.emax;
    const long long budget = s_timeout;
    constexpr int ALL = (1 << NRHS) - 1;

    // ================================================= producer warp
    if (warp == NW) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            int cached_sys = -1, cached_mask = 0;
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
                const int sw = (int)(j / nt);
                const int ti = tb + (int)(j - (long long)sw * nt);
                const int sys = __ldg(bt.tile_sys + ti);
                if (sys != cached_sys || (j % nt) == 0) {   // refresh at system changes and sweep starts
                    cached_sys = sys;
                    cached_mask = ld_volatile_i32(bt.mask + sys);
                }
                uint64_t* bar = &full[sidx];
                if (cached_mask == ALL) {        // retired system: an empty job
                    mbar_expect_tx(bar, 0);
                    issued = j + 1;
                    continue;
                }
                const int ph = phase_of(MIXED, MIXED ? (phase0 + sw) % inner : 0, inner);
                const bool fp64 = (ph == PH_P64 || ph == PH_P64R);
                unsigned char* st = smem + sidx * L.bytes;
                const int r0 = __ldg(t.row0 + ti), r1 = __ldg(t.row1 + ti);
                const int p0 = __ldg(t.nnz0 + ti), p1 = __ldg(t.nnz1 + ti);
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
                if (fp64) bytes += (unsigned)(he - hb) * 8u * NRHS;
                mbar_expect_tx(bar, bytes);
                if (!over) {
                    if (ve > vb) {
                        if (fp64) bulk_g2s(st + L.o_val, m.S64 + vb, (unsigned)(ve - vb) * 8u, bar, pol);
                        else bulk_g2s(st + L.o_val, m.S32 + vb, (unsigned)(ve - vb) * 4u, bar, pol);
                    }
                    if (ce > cb) bulk_g2s(st + L.o_col, m.col + cb, (unsigned)(ce - cb) * 4u, bar, pol);
                }
                bulk_g2s(st + L.o_rp, m.rowptr + rb, (unsigned)(re - rb) * 4u, bar, pol);
                if (fp64 && he > hb)
                    bulk_g2s(st + L.o_c, m.b + (size_t)hb * NRHS, (unsigned)(he - hb) * 8u * NRHS, bar, pol);
                issued = j + 1;
            }
            const long long t0 = clock64();
            for (long long j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j) {
                const unsigned par = (unsigned)((j / STAGES) & 1);
                while (!mbar_try_wait(&full[(int)(j % STAGES)], par))
                    if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); break; }
            }
        }
        return;
    }

    // ================================================= math warps
    long long k = s_k;
    int xb = s_xb, pos = phase0;
    long long evals = s_evals, outer = s_outer;
    long long jc = 0;
    int nbar = 0;
    const int my_pair0 = PART == 2 ? 0 : bt.cta_pair0[blockIdx.x];   // FP32 sweeps keep no norms
    for (int sw = 0; sw < ksw; ++sw) {
        const int ph = phase_of(MIXED, pos, inner);
        const bool norm_ph = (ph == PH_P64 || ph == PH_P64R);
        const double* xs = v.x[xb];
        double* xd = v.x[xb ^ 1];
        const float* es = v.e[pos & 1];
        float* ed = v.e[(pos + 1) & 1];
        // One tile loop per phase type (FP64 sweeps with the norms, FP32 inner
        // sweeps without): the FP32 loop then carries no norm accumulators.
        auto run_tiles = [&](auto tag) {
        using Real = decltype(tag);
        constexpr bool F64 = sizeof(Real) == 8;
        double ss[F64 ? NRHS : 1];
        unsigned long long mx[F64 ? NRHS : 1];
        int cur = -1, msk = ALL;
        int pidx = -1;   // the CTA's partial slot of the current system: systems met so far - 1
        // per-(CTA, system) partials: block reduction, then the last CTA of the system decides
        auto finish = [&](int sys) {
#pragma unroll
            for (int q = 0; q < NRHS; ++q) {
                const double a = warp_sum(ss[q]);
                const unsigned long long b2 = warp_max(mx[q]);
                if (lane == 0) { s_wss[warp][q] = a; s_wmx[warp][q] = b2; }
            }
            b_consumer_sync(CT);
            if (tid == 0) {
                const int slot = my_pair0 + pidx;
                const int par = sw & 1;
                for (int q = 0; q < NRHS; ++q) {
                    double a = 0.0;
                    unsigned long long b2 = 0;
                    for (int w = 0; w < NW; ++w) { a += s_wss[w][q]; b2 = umax64(b2, s_wmx[w][q]); }
                    __stcg(bt.pss + ((size_t)par * bt.npairs + slot) * NRHS + q, a);
                    __stcg(bt.pmx + ((size_t)par * bt.npairs + slot) * NRHS + q, b2);
                }
                __threadfence();
                const unsigned arrived = atomicAdd(bt.cnt + par * bt.nsys + sys, 1u);
                s_blast = arrived == (unsigned)(__ldg(bt.sys_pair0 + sys + 1) - __ldg(bt.sys_pair0 + sys)) - 1;
            }
            b_consumer_sync(CT);
            // the last CTA of the system: warp 0 adds the system's (CTA, system)
            // partials, lane-strided then a fixed shuffle tree
            if (s_blast && warp == 0) {
                __threadfence();
                const int pb = __ldg(bt.sys_pair0 + sys), pe = __ldg(bt.sys_pair0 + sys + 1);
                const int par = sw & 1;
                double ta[NRHS];
                unsigned long long tm[NRHS];
#pragma unroll
                for (int q = 0; q < NRHS; ++q) {
                    double a = 0.0;
                    unsigned long long b2 = 0;
                    for (int pp = pb + lane; pp < pe; pp += 32) {
                        a += __ldcg(bt.pss + ((size_t)par * bt.npairs + pp) * NRHS + q);
                        b2 = umax64(b2, __ldcg(bt.pmx + ((size_t)par * bt.npairs + pp) * NRHS + q));
                    }
                    ta[q] = warp_sum(a);
                    tm[q] = warp_max(b2);
                }
                if (lane == 0) {
                    bt.cnt[par * bt.nsys + sys] = 0;
                    int mk = ld_volatile_i32(bt.mask + sys);
                    for (int q = 0; q < NRHS; ++q) {
                        if (mk & (1 << q)) continue;
                        const double a = ta[q];
                        const unsigned long long b2 = tm[q];
                        const double bn = bt.bnorm[sys * NRHS + q];
                        const Decision d = decide(s_test, s_tol, s_klim, s_norm, bn, a, b2, k);
                        bt.rel[sys * NRHS + q] = d.relres;
                        bt.ksys[sys * NRHS + q] = k;
                        bt.kpar[sys * NRHS + q] = xb;
                        if (d.done != DONE_RUNNING) {
                            mk |= 1 << q;
                            if (d.done == DONE_NUMERIC) atomicOr(&ctl->status, ST_NUMERIC);
                            if (d.done == DONE_LIMIT) bt.sys_status[sys] = DONE_LIMIT;
                            if (d.done == DONE_NUMERIC) bt.sys_status[sys] = DONE_NUMERIC;
                        }
                    }
                    if (mk != ld_volatile_i32(bt.mask + sys)) {
                        bt.mask[sys] = mk;
                        if (mk == ALL) {
                            if (bt.sys_status[sys] == DONE_RUNNING) bt.sys_status[sys] = DONE_CONVERGED;
                            atomicAdd(bt.ndone, 1u);
                        }
                    }
                    __threadfence();
                }
            }
            b_consumer_sync(CT);
        };
        if constexpr (!F64 && PART == 2 && NRHS == 4) {
            // FP32 inner sweeps with 4 right-hand sides (16-byte iterate rows):
            // the gathers of tile i+1 are in flight, as cp.async copies into
            // shared memory, while tile i is summed (see the kernel's comment).
            // Thread t's gathered row u sits at slot u * ROWS + t of its buffer,
            // so each thread reads only what it copied itself and lanes read
            // consecutive 16-byte slots.  Rows longer than GMAXE entries gather
            // the rest when they are summed.
            float4* gbuf = reinterpret_cast<float4*>(smem + STAGES * L.bytes);
            auto wait_stage = [&](long long j) -> bool {
                uint64_t* bar = &full[(int)(j % STAGES)];
                const unsigned par = (unsigned)((j / STAGES) & 1);
                bool ok = mbar_try_wait(bar, par);
                if (!ok && !s_fail) {
                    const long long t0 = clock64();
                    while (!(ok = mbar_try_wait(bar, par))) {
                        if (s_fail) break;
                        if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; break; }
                    }
                }
                return ok;
            };
            struct Pend {
                int sidx, r, kb, len, p0, mk;
                bool act, in, over;
                float4 dl;
            };
            // wait for tile i's stage and start its gathers into buffer (i & 1)
            auto issue = [&](int i, Pend& P) {
                const int ti = tb + i;
                const long long j = jc + i;
                P.sidx = (int)(j % STAGES);
                P.act = false;
                P.in = false;
                P.len = 0;
                const int sys = __ldg(bt.tile_sys + ti);
                if (sys != cur) {
                    cur = sys;
                    msk = ld_volatile_i32(bt.mask + sys);
                }
                P.mk = msk;
                if (wait_stage(j) && msk != ALL) {
                    P.act = true;
                    const unsigned char* st = smem + P.sidx * L.bytes;
                    const int r0 = __ldg(t.row0 + ti), r1 = __ldg(t.row1 + ti);
                    P.p0 = __ldg(t.nnz0 + ti);
                    P.over = (__ldg(t.nnz1 + ti) - P.p0) > emax;
                    const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (r0 & ~3);
                    const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (P.p0 & ~3);
                    P.r = r0 + tid;
                    P.in = P.r < r1;
                    P.kb = P.in ? srp[P.r] : 0;
                    P.len = P.in ? srp[P.r + 1] - P.kb : 0;
                    if (P.in) P.dl = __ldcg(reinterpret_cast<const float4*>(v.dlt) + P.r);
                    if (!P.over) {
                        float4* dst = gbuf + (size_t)(i & 1) * GMAXE * ROWS + tid;
#pragma unroll
                        for (int u = 0; u < GMAXE; ++u)
                            if (u < P.len) cp_async16_cg(dst + u * ROWS, reinterpret_cast<const float4*>(es) + scol[P.kb + u]);
                    }
                }
                cp_async_commit();
            };
            Pend c, nx;
            if (nt > 0) issue(0, c);
            for (int i = 0; i < nt; ++i) {
                if (i + 1 < nt) {
                    issue(i + 1, nx);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                if (c.act && c.in) {
                    const unsigned char* st = smem + c.sidx * L.bytes;
                    float acc[4] = {c.dl.x, c.dl.y, c.dl.z, c.dl.w};
                    if (!c.over) {
                        const float* sv = reinterpret_cast<const float*>(st + L.o_val) - (c.p0 & ~3);
                        const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (c.p0 & ~3);
                        const float4* src = gbuf + (size_t)(i & 1) * GMAXE * ROWS + tid;
#pragma unroll
                        for (int u = 0; u < GMAXE; ++u) {
                            if (u < c.len) {
                                const float tv = sv[c.kb + u];
                                const float4 xv = src[u * ROWS];
                                acc[0] = __fmaf_rn(tv, xv.x, acc[0]);
                                acc[1] = __fmaf_rn(tv, xv.y, acc[1]);
                                acc[2] = __fmaf_rn(tv, xv.z, acc[2]);
                                acc[3] = __fmaf_rn(tv, xv.w, acc[3]);
                            }
                        }
                        for (int u = GMAXE; u < c.len; ++u) {   // the rest of a long row, in order
                            const float tv = sv[c.kb + u];
                            const float4 xv = __ldcg(reinterpret_cast<const float4*>(es) + scol[c.kb + u]);
                            acc[0] = __fmaf_rn(tv, xv.x, acc[0]);
                            acc[1] = __fmaf_rn(tv, xv.y, acc[1]);
                            acc[2] = __fmaf_rn(tv, xv.z, acc[2]);
                            acc[3] = __fmaf_rn(tv, xv.w, acc[3]);
                        }
                    } else {
                        for (int u = 0; u < c.len; ++u) {       // a tile larger than a stage: from global memory
                            const float tv = __ldg(m.S32 + c.kb + u);
                            const float4 xv = __ldcg(reinterpret_cast<const float4*>(es) + __ldg(m.col + c.kb + u));
                            acc[0] = __fmaf_rn(tv, xv.x, acc[0]);
                            acc[1] = __fmaf_rn(tv, xv.y, acc[1]);
                            acc[2] = __fmaf_rn(tv, xv.z, acc[2]);
                            acc[3] = __fmaf_rn(tv, xv.w, acc[3]);
                        }
                    }
                    if (ph == PH_P32) {
                        store_rhs<4>(ed + (size_t)c.r * 4, acc);
                    } else {
                        // y += f; a stopped right-hand side keeps its iterate
                        double y[4];
                        load_rhs<4>(v.x[xb] + (size_t)c.r * 4, y);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (!(c.mk & (1 << q))) y[q] = __dadd_rn(y[q], (double)acc[q]);
                        store_rhs<4>(v.x[xb] + (size_t)c.r * 4, y);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive_b(&empty[c.sidx]);
                c = nx;
            }
            jc += nt;
        } else {
        for (int i = 0; i < nt; ++i, ++jc) {
            const int ti = tb + i;
            const int sys = __ldg(bt.tile_sys + ti);
            if (sys != cur) {
                if constexpr (F64) {
                    if (cur >= 0 && msk != ALL) finish(cur);
                }
                cur = sys;
                ++pidx;
                msk = ld_volatile_i32(bt.mask + sys);
                if constexpr (F64) {
#pragma unroll
                    for (int q = 0; q < NRHS; ++q) { ss[q] = 0.0; mx[q] = 0; }
                }
            }
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
            if (ok && msk != ALL) {
                const unsigned char* st = smem + sidx * L.bytes;
                const int r0 = __ldg(t.row0 + ti), r1 = __ldg(t.row1 + ti);
                const int p0 = __ldg(t.nnz0 + ti), p1 = __ldg(t.nnz1 + ti);
                const bool over = (p1 - p0) > emax;
                const int* srp = reinterpret_cast<const int*>(st + L.o_rp) - (r0 & ~3);
                const int* scol = reinterpret_cast<const int*>(st + L.o_col) - (p0 & ~3);
                const int r = r0 + tid;
                const bool in = r < r1;
                const int kb = in ? srp[r] : 0, len = in ? srp[r + 1] - kb : 0;
                if constexpr (F64) {
                    const double* sv = reinterpret_cast<const double*>(st + L.o_val) - (p0 & ~1);
                    const double* sc = reinterpret_cast<const double*>(st + L.o_c) - (size_t)(r0 & ~1) * NRHS;
                    double acc[NRHS], xi[NRHS];
#pragma unroll
                    for (int q = 0; q < NRHS; ++q) { acc[q] = in ? sc[(size_t)r * NRHS + q] : 0.0; xi[q] = 0.0; }
                    if (in) load_rhs<NRHS>(xs + (size_t)r * NRHS, xi);
                    if (!over)
                        brow_dot<NRHS>(acc, kb, len, xs, [&](int e) { return sv[e]; }, [&](int e) { return scol[e]; });
                    else
                        brow_dot<NRHS>(acc, kb, len, xs, [&](int e) { return __ldg(m.S64 + e); },
                                       [&](int e) { return __ldg(m.col + e); });
                    if (in) {
#pragma unroll
                        for (int q = 0; q < NRHS; ++q) {
                            if (msk & (1 << q)) continue;        // stopped: its iterate stays where it is
                            if (ph == PH_P64) {
                                __stcg(xd + (size_t)r * NRHS + q, acc[q]);
                            } else {
                                const float dl = (float)__dadd_rn(acc[q], -xi[q]);
                                __stcg(v.dlt + (size_t)r * NRHS + q, dl);
                                __stcg(v.e[1] + (size_t)r * NRHS + q, dl);
                            }
                            accumulate_residual(acc[q], xi[q], ss[q], mx[q]);
                        }
                    }
                } else {
                    const float* sv = reinterpret_cast<const float*>(st + L.o_val) - (p0 & ~3);
                    float acc[NRHS];
#pragma unroll
                    for (int q = 0; q < NRHS; ++q) acc[q] = 0.f;
                    if (in) load_rhs<NRHS>(v.dlt + (size_t)r * NRHS, acc);
                    if (!over)
                        brow_dot<NRHS>(acc, kb, len, es, [&](int e) { return sv[e]; }, [&](int e) { return scol[e]; });
                    else
                        brow_dot<NRHS>(acc, kb, len, es, [&](int e) { return __ldg(m.S32 + e); },
                                       [&](int e) { return __ldg(m.col + e); });
                    if (in) {
                        if (ph == PH_P32) {
                            store_rhs<NRHS>(ed + (size_t)r * NRHS, acc);
                        } else {
                            // y += f; a stopped right-hand side keeps its iterate
                            double y[NRHS];
                            load_rhs<NRHS>(v.x[xb] + (size_t)r * NRHS, y);
#pragma unroll
                            for (int q = 0; q < NRHS; ++q)
                                if (!(msk & (1 << q))) y[q] = __dadd_rn(y[q], (double)acc[q]);
                            store_rhs<NRHS>(v.x[xb] + (size_t)r * NRHS, y);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive_b(&empty[sidx]);
        }
        }
        if constexpr (F64) {
            if (cur >= 0 && msk != ALL) finish(cur);
        }
        };
        if constexpr (PART == 1) run_tiles(double(0));
        else if constexpr (PART == 2) run_tiles(float(0));
        else if (norm_ph) run_tiles(double(0));
        else run_tiles(float(0));
        // ---- grid barrier
        b_consumer_sync(CT);
        if (tid == 0) {
            fence_acq_rel_gpu();       // release half of the barrier (see k_persistent)
            atomicAdd(&ctl->bar, 1ull);
            const unsigned long long target = (unsigned long long)(nbar + 1) * gridDim.x;
            const long long t0 = clock64();
            while (ld_acquire_u64(&ctl->bar) < target) {
                if (ld_volatile_i32(&ctl->status) & ST_TIMEOUT) { s_fail = 1; break; }
                if (clock64() - t0 > budget) { atomicOr(&ctl->status, ST_TIMEOUT); s_fail = 1; break; }
                __nanosleep(32);
            }
            s_stop_all = (int)(*(volatile unsigned*)bt.ndone >= (unsigned)bt.nsys);
        }
        ++nbar;
        b_consumer_sync(CT);
        if (s_fail) break;
        if (norm_ph) {
            evals += 1;
            if (s_test && s_stop_all) break;
            if (ph == PH_P64) { k += 1; xb ^= 1; }
            else pos = 1;
        } else if (ph == PH_P32) {
            pos += 1;
        } else {
            pos = 0;
            k += inner;
            outer += 1;
        }
        if (!MIXED && !s_test && k >= s_klim) break;
    }
    if (tid == 0) s_stop = 1;
    if (blockIdx.x == 0 && tid == 0) {
        ctl->k = k;
        ctl->xbuf = xb;
        ctl->phase = pos;
        ctl->evals = evals;
        ctl->outer = outer;
        ctl->done = (s_test && s_stop_all) ? DONE_CONVERGED : DONE_RUNNING;
        __threadfence();
    }
}

template <int NRHS, bool MIXED, int NWM, int PART = 0>
static const void* batched_fn()
{
    // the FP32-sweep launch: more, smaller stages of FP32 data
    return reinterpret_cast<const void*>(&k_batched<NRHS, PART == 2 ? BATCHED_FP32_STAGES : 4, MIXED, NWM, PART>);
}

template <int NRHS, int NWM>
static const void* batched_fn_part(bool mixed, int part)
{
    if (!mixed) return part == 0 ? batched_fn<NRHS, false, NWM>() : nullptr;
    switch (part) {
    case 1: return batched_fn<NRHS, true, NWM, 1>();
    case 2: return batched_fn<NRHS, true, NWM, 2>();
    default: return nullptr;
    }
}

// Geometries: 224-row tiles (7 math warps + producer, 2 CTAs/SM) or 96-row
// tiles (3 + 1 warps, 4 CTAs/SM: finer tiles for small systems).  Both leave
// 128 registers a thread (16 warps per SM).  part: 0 = FP64 solves; 1 / 2 =
// the FP64 pass / the FP32 sweeps of a mixed refinement cycle (part 2:
// BATCHED_FP32_STAGES stages of FP32 data; with 4 right-hand sides, gathers
// through shared memory one tile ahead).
const void* batched_kernel(int nrhs, bool mixed, int rows, int part)
{
    if (rows == 224) {
        switch (nrhs) {
        case 1: return batched_fn_part<1, 7>(mixed, part);
        case 2: return batched_fn_part<2, 7>(mixed, part);
        case 4: return batched_fn_part<4, 7>(mixed, part);
        default: return nullptr;
        }
    }
    if (rows == 96) {
        switch (nrhs) {
        case 1: return batched_fn_part<1, 3>(mixed, part);
        case 2: return batched_fn_part<2, 3>(mixed, part);
        case 4: return batched_fn_part<4, 3>(mixed, part);
        default: return nullptr;
        }
    }
    return nullptr;
}

int batched_threads(int rows) { return rows + 32; }

cudaError_t launch_batched(const void* fn, int grid, int threads, int smem, const DevMat& m, const DevVec& v,
                           const DevTiles& t, const DevBatch& bt, JacCtl* ctl, int max_sweeps, cudaStream_t s)
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
    void* args[] = {(void*)&m, (void*)&v, (void*)&t, (void*)&bt, (void*)&ctl, (void*)&max_sweeps};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

// ----------------------------------------------------------- helpers

// x -> iterate y[r][q] = a_rr x[r][q] in place (packed systems, identity order).
__global__ void k_batched_scale(double* __restrict__ x, const double* __restrict__ d, long long n, int nrhs)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    x[i] = __dmul_rn(d[i / nrhs], x[i]);
}

// ||b_s,q||_2 for every system (one CTA per system, fixed order).
__global__ void __launch_bounds__(256) k_batched_bnorm(const double* __restrict__ b, const long long* __restrict__ off,
                                                       int nrhs, double* __restrict__ bnorm)
{
    __shared__ double sh[8];
    const int s = blockIdx.x;
    const long long r0 = off[s], r1 = off[s + 1];
    for (int q = 0; q < nrhs; ++q) {
        double a = 0.0;
        for (long long r = r0 + threadIdx.x; r < r1; r += 256) a = __fma_rn(b[r * nrhs + q], b[r * nrhs + q], a);
        a = warp_sum(a);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += sh[w];
            bnorm[s * nrhs + q] = sqrt(t);
        }
        __syncthreads();
    }
}

// Result read-back: each (row, right-hand side) from the buffer that holds its
// reported iterate, converted back from y to x = y / a_rr (IEEE division;
// d == nullptr: y itself).
__global__ void k_batched_gather_x(const double* __restrict__ x0, const double* __restrict__ x1,
                                   const int* __restrict__ row_sys, const int* __restrict__ mask,
                                   const int* __restrict__ kpar, int cur, long long n, int nrhs,
                                   const double* __restrict__ d, double* __restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nrhs) return;
    const long long r = i / nrhs;
    const int q = (int)(i - r * nrhs);
    const int s = row_sys[r];
    const int p = (mask[s] >> q) & 1 ? kpar[s * nrhs + q] : cur;
    const double y = (p & 1) ? x1[i] : x0[i];
    out[i] = d ? __ddiv_rn(y, d[r]) : y;
}

__global__ void k_batched_reset(int* mask, long long* ksys, double* rel, int* kpar, int* sys_status, unsigned* cnt,
                                unsigned* ndone, int nsys, int nrhs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsys) {
        mask[i] = 0;
        sys_status[i] = DONE_RUNNING;
        cnt[i] = 0;
        cnt[nsys + i] = 0;
    }
    if (i < nsys * nrhs) {
        ksys[i] = -1;
        rel[i] = 0.0;
        kpar[i] = 0;
    }
    if (i == 0) *ndone = 0;
}

cudaError_t launch_batched_scale(double* x, const double* d, long long n, int nrhs, cudaStream_t s)
{
    const long long tot = n * nrhs;
    k_batched_scale<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x, d, n, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_batched_bnorm(const double* b, const long long* off, int nsys, int nrhs, double* bnorm,
                                 cudaStream_t s)
{
    k_batched_bnorm<<<nsys, 256, 0, s>>>(b, off, nrhs, bnorm);
    return cudaGetLastError();
}

cudaError_t launch_batched_gather_x(const double* x0, const double* x1, const int* row_sys, const int* mask,
                                    const int* kpar, int cur, long long n, int nrhs, const double* d, double* out,
                                    cudaStream_t s)
{
    const long long tot = n * nrhs;
    k_batched_gather_x<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(x0, x1, row_sys, mask, kpar, cur, n, nrhs, d,
                                                                        out);
    return cudaGetLastError();
}

cudaError_t launch_batched_reset(const DevBatch& bt, int nrhs, cudaStream_t s)
{
    const int tot = bt.nsys * nrhs;
    k_batched_reset<<<(tot + 255) / 256, 256, 0, s>>>(bt.mask, bt.ksys, bt.rel, bt.kpar, bt.sys_status, bt.cnt,
                                                      bt.ndone, bt.nsys, nrhs);
    return cudaGetLastError();
}

}  // namespace jac
