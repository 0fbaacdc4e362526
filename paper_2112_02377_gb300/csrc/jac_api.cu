// C ABI of the GB300 Jacobi library: context life cycle, uploads, CUDA graphs
// and the host loops around the sweep kernels.  See include/jacobi.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <numeric>
#include <string>
#include <vector>

#include "jac_device.cuh"
#include "jac_internal.h"
#include "jac_launch.h"

using namespace jac;

static thread_local std::string g_setup_error = "no error";

namespace jac {
// Message for jac_last_error(NULL) from calls that have no context.
void record_thread_error(const std::string& msg) { g_setup_error = msg; }
}  // namespace jac

struct jac_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    jac_opts o{};
    std::string err = "no error";
    int64_t n = 0, nnz = 0, nnz_off = 0, max_row = 0, max_off = 0, halo_entries = 0, interface_rows = 0;
    int64_t rows = 0;              // kernel rows (n, or more with a split interface block)
    // split interface block (jac_setup_local): rows at and after n_own are slot rows
    bool split = false;
    int64_t n_own = 0;
    long long* d_bmap = nullptr;   // rows: original row whose b starts each kernel row's sum, -1 = none
    unsigned* d_slot_info = nullptr;
    int nrhs = 1;
    int splitting = 0, precision = 0, variant = 2;
    int64_t nparts = 0;
    // device data (new row order)
    int* d_rowptr = nullptr;
    int* d_col = nullptr;
    double* d_S64 = nullptr;
    float* d_S32 = nullptr;
    double* d_b = nullptr;         // b in the new row order (FP64 sweep input)
    double* d_d = nullptr;
    double* d_x[3] = {nullptr, nullptr, nullptr};
    int nbuf = 2;                  // iterate buffers in rotation (3 with neighbour sync)
    bool ns = false;               // neighbour-synchronised FP64 sweeps
    int sync = JAC_SYNC_GRID;      // jac_sync of the FP64 kernel
    bool certify = false;          // asynchronous contexts: run the grid-synchronised kernel
    const void* pfn64grid = nullptr;
    int* d_dep_ptr = nullptr;      // ctas+1 / neighbour CTAs of each CTA
    int* d_dep = nullptr;
    unsigned* d_done = nullptr;    // ctas: sweeps finished in the current launch
    int64_t dep_edges = 0;
    float* d_e[2] = {nullptr, nullptr};
    float* d_dlt = nullptr;
    Partial* d_part = nullptr;
    int nslots = 0;
    unsigned long long* d_trace = nullptr;
    std::vector<int32_t> h_cta_row0;      // ctas+1: first row of each CTA (persistent variants)
    std::vector<int32_t> h_cta_row1;      // ctas+1: first row of each CTA's second range (split layouts)
    std::vector<double> h_row_cost;       // per-row cost estimates the CTA ranges were cut with
    JacCtl* d_ctl = nullptr;
    JacCtl* h_ctl = nullptr;     // pinned mirrors [2]
    double* d_hist = nullptr;
    int64_t hist_cap = 0;
    long long* d_perm = nullptr;
    double* d_stage = nullptr;   // n*nrhs staging (original order)
    double* d_stage2 = nullptr;  // second staging buffer (adjoint)
    double* d_grad = nullptr;    // nnz (adjoint)
    int* d_orow = nullptr;       // original pattern (adjoint)
    int* d_ocol = nullptr;
    // tiling / launch
    int* d_row0 = nullptr;
    int* d_nnz0 = nullptr;
    int* d_row1 = nullptr;         // batched: tile end rows / entries (tiles of active systems only)
    int* d_nnz1 = nullptr;
    int* d_cta0 = nullptr;
    int* d_cta1 = nullptr;         // split layouts: each CTA's range of slot tiles
    int* d_blk0 = nullptr;
    int* d_blk = nullptr;
    int* d_lcol = nullptr;
    int xcap = 0, maxruns = 0, ntcap = 0, blkcap = 0;
    int64_t fallback_tiles = 0, window_elems = 0;
    int sms = 1;
    int ntiles = 0, emax = 0, rows_per_tile = 256, stages = 4, grid = 0, threads = 0, smem = 0;
    int lanes = 1;                        // lanes per row (persistent variant, 256 threads)
    // stopping on local convergence (JAC_STOP_LOCAL)
    int stop = JAC_STOP_GLOBAL;
    int* d_mem_ptr = nullptr;             // rows+1: each row's local sets ...
    int* d_mem_part = nullptr;            // ... as dense set numbers
    int* d_mem_head = nullptr;            // rows: first set | (number of sets << 24)
    unsigned long long* d_loc = nullptr;  // [3][nloc] per-set maxima of |r| (order keys)
    int nloc = 0;
    std::vector<int32_t> h_set_id;        // partition number of each dense set
    const void* pfn64 = nullptr;
    const void* pfnmix = nullptr;
    const void* pfnmix32 = nullptr;    // batched mixed: the FP32 sweeps of a cycle (pfnmix: its FP64 pass)
    int K = 64;
    cudaGraphExec_t g64 = nullptr, gmix = nullptr, gcert = nullptr;
    bool no_graph = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // batched contexts
    bool batched = false;
    int nsys = 0, npairs = 0;
    const void* bfn = nullptr;
    int* d_tile_sys = nullptr;
    int* d_sys_pair0 = nullptr;
    int* d_cta_pair0 = nullptr;
    int* d_cta_sys0 = nullptr;
    double* d_bnorm = nullptr;
    unsigned* d_cnt = nullptr;
    int* d_mask = nullptr;
    long long* d_ksys = nullptr;
    int* d_kpar = nullptr;
    double* d_rel = nullptr;
    int* d_sys_status = nullptr;
    unsigned* d_ndone = nullptr;
    double* d_pss = nullptr;
    unsigned long long* d_pmx = nullptr;
    int* d_row_sys = nullptr;
    long long* d_sys_off = nullptr;
    double* d_bstage = nullptr;      // n*nrhs staging for batched rhs / x
    std::vector<long long> h_sys_off;
    std::vector<int32_t> h_rowptr;   // batched: off-diagonal row pointers (tile cuts on re-tiling)
    int tile_cap = 0, pair_cap = 0;  // batched: capacity of the tile and pair arrays
    int64_t tiled_rows = 0;          // batched: rows covered by the current tiles
    bool retiled = false;            // batched: tiles cover a subset of the systems
    // opts.debug: canary bytes in the padding after device vectors
    struct Canary {
        const char* name;
        unsigned char* at;
        size_t bytes;
    };
    std::vector<Canary> canaries;
    // host-side bookkeeping
    int64_t sweeps_total = 0, outer_last = 0;
    double last_ms = 0.0;
    std::vector<long long> h_perm;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

jac_status fail(jac_ctx* c, jac_status st, const std::string& msg)
{
    if (c) c->err = msg;
    else g_setup_error = msg;
    return st;
}

jac_status cuda_fail(jac_ctx* c, cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? JAC_ENOMEM : JAC_ECUDA, m);
}

}  // namespace

namespace jac {

// Host code throws only when an allocation fails (std::bad_alloc from a
// std::vector, std::length_error for a size past its maximum).  No exception
// may cross the C ABI, so every entry point that returns a status is a
// function-try-block whose handler turns the exception into JAC_ENOMEM (any
// other exception into JAC_EINVAL) and records the message.  Call it only
// from a catch handler.
jac_status host_exception(jac_ctx* c) noexcept
{
    jac_status st = JAC_EINVAL;
    const char* m = "unexpected host exception";
    try {
        throw;
    } catch (const std::bad_alloc&) {
        st = JAC_ENOMEM;
        m = "host allocation failed";
    } catch (const std::length_error&) {
        st = JAC_ENOMEM;
        m = "host allocation too large";
    } catch (...) {
    }
    try {
        fail(c, st, m);
    } catch (...) {
    }
    return st;
}

}  // namespace jac

namespace {

#define CK(ctx, call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);      \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemset(*p, 0, count * sizeof(T));
}

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

cudaStream_t stream_of(const jac_ctx* c) { return c->stream; }

jac_status copy_to_stage(jac_ctx* c, const double* src, int memory, size_t count, double* stage)
{
    if (memory == JAC_MEM_DEVICE) {
        CK(c, cudaMemcpyAsync(stage, src, count * sizeof(double), cudaMemcpyDeviceToDevice, stream_of(c)));
    } else if (memory == JAC_MEM_HOST) {
        CK(c, cudaMemcpyAsync(stage, src, count * sizeof(double), cudaMemcpyHostToDevice, stream_of(c)));
    } else {
        return fail(c, JAC_EINVAL, "memory must be JAC_MEM_HOST or JAC_MEM_DEVICE");
    }
    return JAC_OK;
}

double algorithmic_bytes_fp64(int64_t n, int64_t nnz_off)
{
    return 12.0 * nnz_off + 8.0 * n + 4.0 * (n + 1) + 8.0 * n + 8.0 * n + 8.0 * n;
}

double algorithmic_bytes_fp32(int64_t n, int64_t nnz_off)
{
    return 8.0 * nnz_off + 4.0 * (n + 1) + 4.0 * n + 4.0 * n + 4.0 * n;
}

DevMat devmat(const jac_ctx* c)
{
    DevMat m;
    m.n = (int)c->n;
    m.rowptr = c->d_rowptr;
    m.col = c->d_col;
    m.S64 = c->d_S64;
    m.S32 = c->d_S32;
    m.b = c->d_b;
    m.d = c->d_d;
    m.n_own = (int)(c->split ? c->n_own : c->n);
    m.slot_info = c->d_slot_info;
    m.mem_ptr = c->d_mem_ptr;
    m.mem_part = c->d_mem_part;
    m.mem_head = c->d_mem_head;
    return m;
}

DevVec devvec(const jac_ctx* c)
{
    DevVec v;
    v.x[0] = c->d_x[0];
    v.x[1] = c->d_x[1];
    v.x[2] = c->d_x[2];
    v.nbuf = c->nbuf;
    v.e[0] = c->d_e[0];
    v.e[1] = c->d_e[1];
    v.dlt = c->d_dlt;
    v.part = c->d_part;
    v.dec = c->d_part ? c->d_part + 2 * (size_t)c->nslots : nullptr;
    v.nslots = c->nslots;
    v.trace = c->d_trace;
    v.loc = c->d_loc;
    v.nloc = c->nloc;
    return v;
}

DevTiles devtiles(const jac_ctx* c)
{
    DevTiles t;
    t.row0 = c->d_row0;
    t.nnz0 = c->d_nnz0;
    t.row1 = c->d_row1 ? c->d_row1 : (c->d_row0 ? c->d_row0 + 1 : nullptr);
    t.nnz1 = c->d_nnz1 ? c->d_nnz1 : (c->d_nnz0 ? c->d_nnz0 + 1 : nullptr);
    t.cta0 = c->d_cta0;
    t.cta1 = c->d_cta1;
    t.blk0 = c->d_blk0;
    t.blk = c->d_blk;
    t.lcol = c->d_lcol;
    t.ntiles = c->ntiles;
    t.emax = c->emax;
    t.xcap = c->xcap;
    t.maxruns = c->maxruns;
    t.ntcap = c->ntcap;
    t.blkcap = c->blkcap;
    t.dep_ptr = c->d_dep_ptr;
    t.dep = c->d_dep;
    t.done = c->d_done;
    return t;
}

DevBatch devbatch(const jac_ctx* c)
{
    DevBatch b;
    b.nsys = c->nsys;
    b.npairs = c->npairs;
    b.tile_sys = c->d_tile_sys;
    b.sys_pair0 = c->d_sys_pair0;
    b.cta_pair0 = c->d_cta_pair0;
    b.cta_sys0 = c->d_cta_sys0;
    b.bnorm = c->d_bnorm;
    b.cnt = c->d_cnt;
    b.mask = c->d_mask;
    b.ksys = c->d_ksys;
    b.kpar = c->d_kpar;
    b.rel = c->d_rel;
    b.sys_status = c->d_sys_status;
    b.ndone = c->d_ndone;
    b.pss = c->d_pss;
    b.pmx = c->d_pmx;
    return b;
}

// Refinement cycles of a mixed graph step of the persistent kernels: K sweeps
// rounded up to whole cycles of inner_sweeps.
int mixed_cycles_per_step(const jac_ctx* c)
{
    const int m = std::max(2, c->o.inner_sweeps);
    return std::max(1, (c->K + m - 1) / m);
}

// Enqueue one "graph step": K sweeps (FP64) or one refinement cycle block (mixed).
jac_status enqueue_step(jac_ctx* c, bool mixed)
{
    cudaStream_t s = stream_of(c);
    if (c->batched) {
        if (!mixed) {
            CK(c, launch_reset_bar(c->d_ctl, s));
            CK(c, launch_batched(c->pfn64, c->grid, c->threads, c->smem, devmat(c), devvec(c), devtiles(c),
                                 devbatch(c), c->d_ctl, c->K, s));
            return JAC_OK;
        }
        // whole refinement cycles: the FP64 pass, then the FP32 sweeps, each a
        // launch of its own (a launch after a converged pass returns at once)
        for (int cyc = 0; cyc < mixed_cycles_per_step(c); ++cyc)
            for (const void* fn : {c->pfnmix, c->pfnmix32}) {
                CK(c, launch_reset_bar(c->d_ctl, s));
                CK(c, launch_batched(fn, c->grid, c->threads, c->smem, devmat(c), devvec(c), devtiles(c),
                                     devbatch(c), c->d_ctl, c->o.inner_sweeps, s));
            }
        return JAC_OK;
    }
    if (c->variant >= 2) {
        CK(c, launch_reset_bar(c->d_ctl, s));
        if (c->ns && !mixed) CK(c, cudaMemsetAsync(c->d_done, 0, sizeof(unsigned) * DONE_STRIDE * c->grid, s));
        if (mixed && c->pfnmix32) {
            // whole refinement cycles, two launches each (see the batched case)
            bool first = true;   // the barrier counter was reset above for the first launch
            for (int cyc = 0; cyc < mixed_cycles_per_step(c); ++cyc)
                for (const void* fn : {c->pfnmix, c->pfnmix32}) {
                    if (!first) CK(c, launch_reset_bar(c->d_ctl, s));
                    first = false;
                    CK(c, launch_persistent(fn, c->grid, c->threads, c->smem, devmat(c), devvec(c), devtiles(c),
                                            c->d_ctl, c->o.inner_sweeps, s));
                }
            return JAC_OK;
        }
        const void* fn = mixed ? c->pfnmix : (c->certify ? c->pfn64grid : c->pfn64);
        CK(c, launch_persistent(fn, c->grid, c->threads, c->smem, devmat(c), devvec(c), devtiles(c), c->d_ctl, c->K,
                                s));
    } else {
        if (!mixed) {
            for (int i = 0; i < c->K; ++i) CK(c, launch_row_sweep(PH_P64, devmat(c), devvec(c), c->d_ctl, s));
        } else {
            const int m = c->o.inner_sweeps;
            CK(c, launch_row_sweep(PH_P64R, devmat(c), devvec(c), c->d_ctl, s));
            for (int j = 1; j < m - 1; ++j) CK(c, launch_row_sweep(PH_P32, devmat(c), devvec(c), c->d_ctl, s));
            CK(c, launch_row_sweep(PH_P32L, devmat(c), devvec(c), c->d_ctl, s));
        }
    }
    return JAC_OK;
}

jac_status get_graph(jac_ctx* c, bool mixed, cudaGraphExec_t* out)
{
    cudaGraphExec_t& g = mixed ? c->gmix : (c->certify ? c->gcert : c->g64);
    if (!g) {
        cudaStream_t s = stream_of(c);
        cudaStream_t cap = s;
        bool own = false;
        if (!s) {   // legacy stream cannot be captured: capture on a private stream
            CK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            own = true;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaStream_t saved = c->stream;
            c->stream = cap;
            jac_status st = enqueue_step(c, mixed);
            c->stream = saved;
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (st != JAC_OK) {
                if (graph) cudaGraphDestroy(graph);
                if (own) cudaStreamDestroy(cap);
                return st;
            }
            e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (own) cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            g = nullptr;
            cudaGetLastError();
            return cuda_fail(c, e, "CUDA graph capture of the sweep loop");
        }
    }
    *out = g;
    return JAC_OK;
}

jac_status run_graph(jac_ctx* c, bool mixed)
{
    if (c->no_graph) return enqueue_step(c, mixed);
    cudaGraphExec_t g = nullptr;
    jac_status st = get_graph(c, mixed, &g);
    if (st != JAC_OK) {
        // Stream capture of this launch form is unavailable: launch directly.
        c->no_graph = true;
        cudaGetLastError();
        return enqueue_step(c, mixed);
    }
    CK(c, cudaGraphLaunch(g, stream_of(c)));
    return JAC_OK;
}

// Batched: gather each right-hand side's current iterate (some stopped ones
// live in the other ping-pong buffer) into x[0], restart k at 0 and re-arm
// every system's test.
jac_status batched_tile(jac_ctx* c, const std::vector<int32_t>& mask, bool alloc = false);

// ---------------------------------------------------------------- canaries
// With opts.debug every device vector's 16-element padding (past the last
// element any kernel may write) holds a byte pattern that is checked after
// each sweep or solve call: a stray write past the end shows up as an error.
constexpr unsigned char CANARY = 0xA5;

template <class T>
void add_canary(jac_ctx* c, const char* name, T* base, size_t used)
{
    if (base) c->canaries.push_back({name, reinterpret_cast<unsigned char*>(base + used), 16 * sizeof(T)});
}

jac_status set_canaries(jac_ctx* c)
{
    for (const auto& k : c->canaries) CK(c, cudaMemset(k.at, CANARY, k.bytes));
    return JAC_OK;
}

jac_status check_canaries(jac_ctx* c)
{
    std::vector<unsigned char> h;
    for (const auto& k : c->canaries) {
        h.assign(k.bytes, 0);
        CK(c, cudaMemcpy(h.data(), k.at, k.bytes, cudaMemcpyDeviceToHost));
        for (unsigned char v : h)
            if (v != CANARY) return fail(c, JAC_ECUDA, std::string("device buffer overrun detected past ") + k.name);
    }
    return JAC_OK;
}

jac_status batched_restart(jac_ctx* c)
{
    cudaStream_t s = stream_of(c);
    if (c->retiled) {   // a solve re-tiled for its last systems: every system iterates again
        CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
        const jac_status st = batched_tile(c, std::vector<int32_t>());
        if (st != JAC_OK) return st;
    }
    CK(c, launch_batched_gather_x(c->d_x[0], c->d_x[1], c->d_row_sys, c->d_mask, c->d_kpar, c->h_ctl[0].xbuf & 1,
                                  c->n, c->nrhs, nullptr, c->d_bstage, s));
    CK(c, cudaMemcpyAsync(c->d_x[0], c->d_bstage, (size_t)c->n * c->nrhs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(c, launch_batched_reset(devbatch(c), c->nrhs, s));
    CK(c, launch_reset_iterate(c->d_ctl, s));
    c->h_ctl[0].xbuf = 0;
    return JAC_OK;
}

jac_status status_from_ctl(jac_ctx* c, const JacCtl& h)
{
    if (h.status & ST_CONFIG)
        return fail(c, JAC_ECUDA, "a kernel was launched with less shared memory than its stage layout needs");
    if (h.status & ST_TIMEOUT)
        return fail(c, JAC_ETIMEOUT, "a device-side wait exceeded its bound (grid barrier or copy); iterate undefined");
    if ((h.status & ST_NUMERIC) || h.done == DONE_NUMERIC)
        return fail(c, JAC_ENUMERIC, "the residual became NaN or Inf (the iteration diverges)");
    return JAC_OK;
}

jac_status arm(jac_ctx* c, int test, int mixed, long long k_limit, long long k_delta, double tol)
{
    if (c->d_trace)
        CK(c, cudaMemsetAsync(c->d_trace, 0, 4 * sizeof(unsigned long long) * c->grid, stream_of(c)));
    if (c->d_loc) CK(c, cudaMemsetAsync(c->d_loc, 0, 3 * sizeof(unsigned long long) * c->nloc, stream_of(c)));
    CK(c, launch_arm(c->d_ctl, test, mixed, c->o.inner_sweeps, k_limit, k_delta, tol, c->o.norm, c->d_hist, c->hist_cap,
                     (long long)c->o.timeout_cycles, c->o.fault_skip_cta, stream_of(c)));
    return JAC_OK;
}

jac_status fetch_ctl(jac_ctx* c, JacCtl* dst)
{
    CK(c, cudaMemcpyAsync(dst, c->d_ctl, sizeof(JacCtl), cudaMemcpyDeviceToHost, stream_of(c)));
    return JAC_OK;
}

void destroy(jac_ctx* c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->g64) cudaGraphExecDestroy(c->g64);
    if (c->gmix) cudaGraphExecDestroy(c->gmix);
    if (c->gcert) cudaGraphExecDestroy(c->gcert);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    dfree(c->d_rowptr); dfree(c->d_col); dfree(c->d_S64); dfree(c->d_S32); dfree(c->d_b); dfree(c->d_d);
    dfree(c->d_x[0]); dfree(c->d_x[1]); dfree(c->d_x[2]);
    dfree(c->d_dep_ptr); dfree(c->d_dep); dfree(c->d_done); dfree(c->d_e[0]); dfree(c->d_e[1]); dfree(c->d_dlt);
    dfree(c->d_part); dfree(c->d_ctl); dfree(c->d_hist); dfree(c->d_perm); dfree(c->d_stage); dfree(c->d_stage2);
    dfree(c->d_bmap); dfree(c->d_slot_info);
    dfree(c->d_mem_ptr); dfree(c->d_mem_part); dfree(c->d_mem_head); dfree(c->d_loc);
    dfree(c->d_grad); dfree(c->d_orow); dfree(c->d_ocol); dfree(c->d_row0); dfree(c->d_nnz0);
    dfree(c->d_row1); dfree(c->d_nnz1); dfree(c->d_cta0); dfree(c->d_cta1);
    dfree(c->d_blk0); dfree(c->d_blk); dfree(c->d_lcol); dfree(c->d_trace);
    dfree(c->d_tile_sys); dfree(c->d_sys_pair0); dfree(c->d_cta_pair0); dfree(c->d_cta_sys0); dfree(c->d_bnorm);
    dfree(c->d_cnt); dfree(c->d_mask); dfree(c->d_ksys); dfree(c->d_kpar); dfree(c->d_rel); dfree(c->d_sys_status);
    dfree(c->d_ndone); dfree(c->d_pss); dfree(c->d_pmx); dfree(c->d_row_sys); dfree(c->d_sys_off); dfree(c->d_bstage);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    delete c;
}

// Host copy of a caller CSR that may live in device memory.
struct HostView {
    std::vector<int32_t> rp, cl;
    std::vector<double> vl;
    jac_csr csr{};
};

jac_status host_view(const jac_csr* A, HostView& hv, jac_ctx* err_ctx)
{
    if (!A) return fail(err_ctx, JAC_EINVAL, "A is NULL");
    if (A->memory == JAC_MEM_HOST) {
        hv.csr = *A;
        return JAC_OK;
    }
    if (A->memory != JAC_MEM_DEVICE) return fail(err_ctx, JAC_EINVAL, "A->memory must be HOST or DEVICE");
    if (A->n < 1 || A->nnz < 0) return fail(err_ctx, JAC_EINVAL, "bad n / nnz");
    hv.rp.resize(A->n + 1);
    hv.cl.resize(A->nnz);
    hv.vl.resize(A->nnz);
    cudaError_t e = cudaMemcpy(hv.rp.data(), A->rowptr, (A->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && A->nnz)
        e = cudaMemcpy(hv.cl.data(), A->col, A->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && A->nnz)
        e = cudaMemcpy(hv.vl.data(), A->val, A->nnz * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(err_ctx, e, "copy of the device CSR to the host");
    hv.csr = *A;
    hv.csr.rowptr = hv.rp.data();
    hv.csr.col = hv.cl.data();
    hv.csr.val = hv.vl.data();
    hv.csr.memory = JAC_MEM_HOST;
    return JAC_OK;
}

jac_status check_opts(const jac_opts& o, jac_ctx* err_ctx)
{
    if (o.precision != JAC_FP64 && o.precision != JAC_MIXED) return fail(err_ctx, JAC_EINVAL, "opts.precision");
    if (o.norm != JAC_NORM_REL2 && o.norm != JAC_NORM_INF) return fail(err_ctx, JAC_EINVAL, "opts.norm must be 2 or 0");
    if (o.sweeps_per_graph < 1 || o.sweeps_per_graph > 4096) return fail(err_ctx, JAC_EINVAL, "opts.sweeps_per_graph");
    if (o.inner_sweeps < 2 || o.inner_sweeps > 100000)
        return fail(err_ctx, JAC_EINVAL, "opts.inner_sweeps must be in [2, 100000]");
    if (o.nrhs != 1) return fail(err_ctx, JAC_EINVAL, "opts.nrhs > 1 is supported by jac_setup_batched only");
    if (o.variant < 0 || o.variant > 3) return fail(err_ctx, JAC_EINVAL, "opts.variant must be 0, 1, 2 or 3");
    if (o.tile_rows != 0 && o.tile_rows != 224 && o.tile_rows != 256 && o.tile_rows != 480)
        return fail(err_ctx, JAC_EINVAL, "opts.tile_rows must be 0, 224, 256 or 480");
    if (o.history < 0) return fail(err_ctx, JAC_EINVAL, "opts.history must be >= 0");
    if (o.ctas_per_sm != 0 && o.ctas_per_sm != 2 && o.ctas_per_sm != 3)
        return fail(err_ctx, JAC_EINVAL, "opts.ctas_per_sm must be 0, 2 or 3");
    if (o.lanes_per_row != 0 && o.lanes_per_row != 1 && o.lanes_per_row != 2 && o.lanes_per_row != 4 &&
        o.lanes_per_row != 8)
        return fail(err_ctx, JAC_EINVAL, "opts.lanes_per_row must be 0, 1, 2, 4 or 8");
    if (o.stages != 0 && o.stages != 2 && o.stages != 3 && o.stages != 4)
        return fail(err_ctx, JAC_EINVAL, "opts.stages must be 0, 2, 3 or 4");
    if (o.sync != JAC_SYNC_GRID && o.sync != JAC_SYNC_NEIGHBOUR && o.sync != JAC_SYNC_ASYNC)
        return fail(err_ctx, JAC_EINVAL, "opts.sync must be JAC_SYNC_GRID, JAC_SYNC_NEIGHBOUR or JAC_SYNC_ASYNC");
    if (o.stop != JAC_STOP_GLOBAL && o.stop != JAC_STOP_LOCAL)
        return fail(err_ctx, JAC_EINVAL, "opts.stop must be JAC_STOP_GLOBAL or JAC_STOP_LOCAL");
    if (o.stop == JAC_STOP_LOCAL) {
        if (o.precision != JAC_FP64 || o.norm != JAC_NORM_INF || o.sync != JAC_SYNC_GRID)
            return fail(err_ctx, JAC_EINVAL, "JAC_STOP_LOCAL needs JAC_FP64, JAC_NORM_INF and JAC_SYNC_GRID");
        if ((o.variant != 0 && o.variant != 2) || (o.tile_rows != 0 && o.tile_rows != 256) ||
            o.lanes_per_row == 8)
            return fail(err_ctx, JAC_EINVAL,
                        "JAC_STOP_LOCAL runs in the persistent kernel with 256-thread tiles and 1, 2 or 4 lanes per row");
    }
    return JAC_OK;
}

// ---------------------------------------------------------------- autotuner

// Device time per sweep of a freshly set-up context: a warm-up, then the
// median of three timed calls, each long enough (about 2 ms of device time or
// more) that launch and clock noise stay small next to the differences
// between geometries.  FP64: fixed sweeps; mixed: whole refinement cycles of a
// solve that cannot converge.  The iterate is reset to x^0 = 0 afterwards.
// A call that fails (e.g. a divergent iteration overflowing) ends the timing
// with what was measured so far.
double time_per_sweep(jac_ctx* c)
{
    constexpr double kTargetMs = 2.0;
    std::vector<double> t;
    double warm = 1e30;
    if (c->precision == JAC_MIXED && !c->batched) {
        int64_t k = 0;
        double rel = 0.0;
        const int64_t inner = std::max<int64_t>(2, c->o.inner_sweeps);
        const int64_t cyc = 2 * inner;
        jac_status st = jac_solve(c, 0.0, cyc - 1, &k, &rel);
        if ((st == JAC_OK || st == JAC_ENOTCONV) && k > 0 && c->last_ms > 0.0) warm = c->last_ms / (double)k;
        const int64_t ncyc = std::min<int64_t>(
            64, std::max<int64_t>(2, (int64_t)std::ceil(kTargetMs / std::max(warm * inner, 1e-6))));
        for (int rep = 0; rep < 3; ++rep) {
            jac_set_x(c, nullptr, JAC_MEM_HOST);
            st = jac_solve(c, 0.0, ncyc * inner - 1, &k, &rel);
            if ((st != JAC_OK && st != JAC_ENOTCONV) || k < ncyc * inner - 1 || !(c->last_ms > 0.0)) break;
            t.push_back(c->last_ms / (double)k);
        }
    } else {
        double rel = 0.0;
        if (jac_sweep(c, 8, &rel) == JAC_OK && c->last_ms > 0.0) warm = c->last_ms / 8.0;
        const int nsw = (int)std::min<double>(8192.0, std::max(32.0, std::ceil(kTargetMs / std::max(warm, 1e-6))));
        for (int rep = 0; rep < 3; ++rep) {
            if (jac_sweep(c, nsw, &rel) != JAC_OK || !(c->last_ms > 0.0)) break;
            t.push_back(c->last_ms / (double)nsw);
        }
    }
    jac_set_x(c, nullptr, JAC_MEM_HOST);
    if (t.empty()) return warm;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

// JAC_AUTOTUNE_LOG=1 in the environment: one line per timed candidate on stderr.
static bool autotune_log()
{
    const char* v = std::getenv("JAC_AUTOTUNE_LOG");
    return v && v[0] == '1';
}

struct Geometry {
    int variant, rows, ctas, lanes;   // lanes 0: automatic
    int sync = JAC_SYNC_GRID;
    int stages = 0;                   // 0: automatic
};

// Batched tiling over the systems still iterating (mask != all right-hand
// sides stopped; an empty mask = every system): each such system's rows cut
// into tiles of at most rows_per_tile rows and emax staged entries; CTAs own
// contiguous tile ranges balanced by the bytes a sweep moves; (CTA, system)
// partial slots in CTA order, so the slots of one system are contiguous.
// Fills the tile and pair arrays in place; at set-up (alloc) it first
// allocates them for the full tiling, which every later subset fits: the
// cuts of a system do not depend on the other systems, and a CTA has at most
// one partial slot per tile.
jac_status batched_tile(jac_ctx* c, const std::vector<int32_t>& mask, bool alloc)
{
    const int nsys = c->nsys, R = c->nrhs, G = c->grid;
    const int all = (1 << R) - 1;
    const std::vector<long long>& off = c->h_sys_off;
    const std::vector<int32_t>& rp = c->h_rowptr;
    std::vector<int32_t> r0v, r1v, p0v, p1v, tsys;
    int64_t rows_tiled = 0;
    for (int s = 0; s < nsys; ++s) {
        if (!mask.empty() && mask[s] == all) continue;
        long long r = off[s];
        const long long end = off[s + 1];
        rows_tiled += end - r;
        while (r < end) {
            long long rows = 0, ent = 0;
            while (r + rows < end && rows < c->rows_per_tile) {
                const long long len = rp[r + rows + 1] - rp[r + rows];
                if (rows > 0 && ent + len > c->emax) break;
                ent += len;
                ++rows;
                if (ent > c->emax) break;   // a single oversized row forms its own tile
            }
            r0v.push_back((int32_t)r);
            r1v.push_back((int32_t)(r + rows));
            p0v.push_back(rp[r]);
            p1v.push_back(rp[r + rows]);
            tsys.push_back(s);
            r += rows;
        }
    }
    const int nt = (int)r0v.size();
    if (alloc) {
        c->tile_cap = std::max(nt, 1);
        c->pair_cap = c->tile_cap + G;
        CK(c, dalloc(&c->d_row0, (size_t)c->tile_cap + 1));
        CK(c, dalloc(&c->d_row1, (size_t)c->tile_cap));
        CK(c, dalloc(&c->d_nnz0, (size_t)c->tile_cap + 1));
        CK(c, dalloc(&c->d_nnz1, (size_t)c->tile_cap));
        CK(c, dalloc(&c->d_tile_sys, (size_t)c->tile_cap + 1));
        CK(c, dalloc(&c->d_cta0, (size_t)G + 1));
        CK(c, dalloc(&c->d_cta_pair0, (size_t)G));
        CK(c, dalloc(&c->d_cta_sys0, (size_t)G));
        CK(c, dalloc(&c->d_sys_pair0, (size_t)nsys + 1));
        CK(c, dalloc(&c->d_pss, 2 * (size_t)c->pair_cap * R));
        CK(c, dalloc(&c->d_pmx, 2 * (size_t)c->pair_cap * R));
    }
    if (nt > c->tile_cap) return fail(c, JAC_ECUDA, "batched: tile capacity exceeded");
    std::vector<double> pre(nt + 1, 0.0);
    for (int i = 0; i < nt; ++i)
        pre[i + 1] = pre[i] + 12.0 * (p1v[i] - p0v[i]) + (4.0 + 24.0 * R) * (r1v[i] - r0v[i]);
    std::vector<int32_t> cta0(G + 1, 0);
    int cur = 0;
    for (int g = 1; g < G; ++g) {
        const double target = pre[nt] * (double)g / (double)G;
        while (cur < nt && pre[cur] + 0.5 * (pre[cur + 1] - pre[cur]) < target) ++cur;
        cta0[g] = cur;
    }
    cta0[G] = nt;
    std::vector<int32_t> cta_pair0(G, 0), cta_sys0(G, 0), sys_pair0(nsys + 1, -1);
    int npairs = 0, last_sys = -1;
    for (int g = 0; g < G; ++g) {
        cta_pair0[g] = npairs;
        const int tb = cta0[g], te = cta0[g + 1];
        if (tb == te) continue;
        cta_sys0[g] = tsys[tb];
        for (int i = tb; i < te; ++i) {
            const int s = tsys[i];
            if (s == last_sys && i > tb) continue;
            if (sys_pair0[s] < 0) sys_pair0[s] = npairs;
            else if (s != last_sys) return fail(c, JAC_ECUDA, "batched: internal tiling error");
            // every system between the CTA's first and this one gets a slot too (none: systems are tiled in order)
            last_sys = s;
            ++npairs;
        }
    }
    // systems without tiles (stopped): an empty slot range at the running position
    sys_pair0[nsys] = npairs;
    for (int s = nsys - 1; s >= 0; --s)
        if (sys_pair0[s] < 0) sys_pair0[s] = sys_pair0[s + 1];
    if (npairs > c->pair_cap) return fail(c, JAC_ECUDA, "batched: partial-slot capacity exceeded");
    auto up = [&](int* dst, const std::vector<int32_t>& v) -> cudaError_t {
        return v.empty() ? cudaSuccess : cudaMemcpy(dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice);
    };
    CK(c, up(c->d_row0, r0v));
    CK(c, up(c->d_row1, r1v));
    CK(c, up(c->d_nnz0, p0v));
    CK(c, up(c->d_nnz1, p1v));
    CK(c, up(c->d_tile_sys, tsys));
    CK(c, up(c->d_cta0, cta0));
    CK(c, up(c->d_cta_pair0, cta_pair0));
    CK(c, up(c->d_cta_sys0, cta_sys0));
    CK(c, up(c->d_sys_pair0, sys_pair0));
    c->ntiles = nt;
    c->npairs = npairs;
    c->tiled_rows = rows_tiled;
    c->retiled = !mask.empty();
    // the captured graphs hold the old tile count: capture again
    if (c->g64) { cudaGraphExecDestroy(c->g64); c->g64 = nullptr; }
    if (c->gmix) { cudaGraphExecDestroy(c->gmix); c->gmix = nullptr; }
    return JAC_OK;
}

}  // namespace

// =========================================================================
extern "C" {

void jac_opts_default(jac_opts* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = JAC_FP64;
    o->norm = JAC_NORM_REL2;
    o->sweeps_per_graph = 64;
    o->inner_sweeps = 128;
    o->nrhs = 1;
    o->transpose = 0;
    o->variant = 0;
    o->tile_rows = 0;
    o->history = 0;
    o->stream = nullptr;
    o->timeout_cycles = 0;
    o->fault_skip_cta = -1;
    o->device = -1;
    o->stop = JAC_STOP_GLOBAL;
}

const char* jac_last_error(const jac_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_setup_error.c_str();
}

void jac_free(jac_ctx* ctx) { destroy(ctx); }

jac_status jac_partition_plan(const jac_csr* A, jac_splitting s, int32_t nparts, const jac_opts* o_in,
                              int64_t* perm, int64_t* part_ptr, int64_t* nparts_out)
try {
    jac_opts o;
    jac_opts_default(&o);
    if (o_in) o = *o_in;
    if (!A || A->memory != JAC_MEM_HOST) return fail(nullptr, JAC_EINVAL, "A must be in host memory");
    if (!perm || !part_ptr) return fail(nullptr, JAC_EINVAL, "perm / part_ptr are NULL");
    HostCSR M;
    Error e = host_csr_from_abi(A, o.transpose != 0, M);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    Plan plan;
    e = make_plan(M, s, nparts, o, plan);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    for (int64_t r = 0; r < M.n; ++r) perm[r] = plan.perm[r];
    for (int64_t p = 0; p <= plan.nparts(); ++p) part_ptr[p] = plan.part_ptr[p];
    if (nparts_out) *nparts_out = plan.nparts();
    return JAC_OK;
} catch (...) {
    return host_exception(nullptr);
}

jac_status jac_dependency_lists(const jac_csr* A, jac_splitting s, int32_t nparts, const jac_opts* o_in,
                                int64_t* recv_ptr, int32_t* recv_from, int64_t* recv, int64_t* total)
try {
    jac_opts o;
    jac_opts_default(&o);
    if (o_in) o = *o_in;
    if (!A || A->memory != JAC_MEM_HOST) return fail(nullptr, JAC_EINVAL, "A must be in host memory");
    if (!recv_ptr || !total) return fail(nullptr, JAC_EINVAL, "recv_ptr / total are NULL");
    HostCSR M;
    Error e = host_csr_from_abi(A, o.transpose != 0, M);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    Plan plan;
    e = make_plan(M, s, nparts, o, plan);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    std::vector<int64_t> rp, rc;
    std::vector<int32_t> rf;
    dependency_lists(M, plan, rp, rf, rc);
    for (size_t p = 0; p < rp.size(); ++p) recv_ptr[p] = rp[p];
    if (recv) {
        if (*total < (int64_t)rc.size()) return fail(nullptr, JAC_EINVAL, "recv arrays too small");
        for (size_t q = 0; q < rc.size(); ++q) { recv[q] = rc[q]; if (recv_from) recv_from[q] = rf[q]; }
    }
    *total = (int64_t)rc.size();
    return JAC_OK;
} catch (...) {
    return host_exception(nullptr);
}

inline int64_t nnz_off_of(const ScaledForm& tf) { return tf.rowptr.empty() ? 0 : tf.rowptr.back(); }

// A context from a matrix already split and scaled: tf holds the kernel rows
// (tf.n of them; n for jac_setup, more with a split interface block), tf.d and
// the iterate the n rows.  sp: the split interface layout (jac_setup_local),
// else NULL.  pattern: the caller's CSR pattern for the adjoint gradient
// (forward jac_setup contexts), else NULL.  b: n doubles in b_memory.
// row_cost (NULL: the default model) sets how the persistent variants cut
// the CTA row ranges.
static jac_status setup_core(const Plan& plan, const ScaledForm& tf, int64_t n, int64_t nnz, int64_t halo_entries,
                             const SplitForm* sp, const HostCSR* pattern, const double* b, int32_t b_memory,
                             jac_opts o, int dev, const std::vector<double>* row_cost, jac_ctx** out)
{
    jac_status st = JAC_OK;
    std::unique_ptr<jac_ctx, void (*)(jac_ctx*)> c(new jac_ctx(), destroy);
    c->device = dev;
    c->stream = (cudaStream_t)o.stream;
    c->o = o;
    c->n = n;
    c->rows = tf.n;
    c->split = sp != nullptr;
    c->n_own = sp ? sp->n_own : n;
    c->nnz = nnz;
    c->nnz_off = tf.rowptr[tf.n];
    c->max_off = tf.max_off;
    c->max_row = tf.max_off + 1;
    c->splitting = plan.splitting;
    c->precision = o.precision;
    c->nparts = plan.nparts();
    c->interface_rows = plan.interface_rows;
    c->K = o.sweeps_per_graph;
    c->halo_entries = halo_entries;
    c->stop = o.stop;
    if (c->stop == JAC_STOP_LOCAL && (sp || o.nrhs != 1))
        return fail(nullptr, JAC_EINVAL, "JAC_STOP_LOCAL is supported by jac_setup contexts only");
    jac_ctx* C = c.get();
    const int64_t rows = tf.n, nnz_off = c->nnz_off;
    if (rows > INT32_MAX - 64) return fail(nullptr, JAC_EINVAL, "n too large");

    // ---- launch configuration
    cudaDeviceProp prop;
    CK(nullptr, cudaGetDeviceProperties(&prop, dev));
    Tiling tl;
    Windows win;
    // Default geometry: the persistent kernel with 8 math warps (256 threads),
    // 2 CTAs/SM and the plain row loop; the autotuner also tries 3 CTAs/SM
    // and the 7/15-warp software-pipelined geometries.
    c->variant = o.variant == 0 ? 2 : o.variant;
    c->rows_per_tile = o.tile_rows ? o.tile_rows : 256;
    c->stages = 4;
    if (c->variant == 3 && c->rows_per_tile != 256) c->variant = 2;
    const int target_per_sm = (c->variant == 2 && c->rows_per_tile == 256 && o.ctas_per_sm == 3) ? 3 : 2;
    if (target_per_sm == 3) c->stages = 3;
    // fewer, larger stages (2 CTAs/SM, 256 threads): room for whole tiles of long rows
    if (c->variant == 2 && c->rows_per_tile == 256 && target_per_sm == 2 && (o.stages == 2 || o.stages == 3))
        c->stages = o.stages;
    // Lanes per row (256-thread geometry only): long rows fill a stage's
    // entry budget with few rows, which leaves math warps without a row, and
    // a long FMA chain per thread; L lanes per row split both.  Each lane's
    // extra cost is the group's shuffle tree.  Auto: halve the entries per
    // lane while at least 8 remain (measured on GB300: 26-entry FE rows run
    // best with L = 2, 7-point rows with L = 1).
    c->lanes = 1;
    if (c->variant == 2 && c->rows_per_tile == 256) {
        const double avg = rows > 0 ? (double)nnz_off_of(tf) / (double)rows : 0.0;
        // local stopping is compiled for 1, 2 and 4 lanes
        const int lane_cap = (o.stop == JAC_STOP_LOCAL) ? 4 : 8;
        if (o.lanes_per_row) c->lanes = o.lanes_per_row;
        else while (c->lanes < lane_cap && avg / (2.0 * c->lanes) >= 8.0) c->lanes *= 2;
    } else if (o.lanes_per_row > 1) {
        return fail(nullptr, JAC_EINVAL, "opts.lanes_per_row > 1 needs variant 2 with 256-thread tiles");
    }
    if (c->variant >= 2) {
        const int rows = c->rows_per_tile / c->lanes;     // rows of a tile
        int64_t cap_entries = (int64_t)std::max<int64_t>(1, tf.max_off) * rows;
        int64_t stage_budget;
        if (c->variant == 3) {
            // 2 CTAs/SM x 3 stages of (matrix data + run list + x window) in ~210 KB
            c->stages = 3;
            c->xcap = 1280;
            c->maxruns = 16;
            stage_budget = 36 * 1024 - (c->xcap + 8) * 8;
        } else {
            // 2 CTAs/SM x 4 stages for 224/256-thread tiles (or 3 / 2 larger
            // stages), 3 CTAs/SM x 3 stages, 1 CTA/SM x 4 stages for 480-row tiles
            stage_budget = c->rows_per_tile <= 256 ? 26 * 1024 : 52 * 1024;
            if (c->rows_per_tile == 256 && target_per_sm == 2 && c->stages == 3) stage_budget = 36 * 1024;
            if (c->rows_per_tile == 256 && target_per_sm == 2 && c->stages == 2) stage_budget = 54 * 1024;
        }
        const int64_t budget_entries = std::max<int64_t>(rows, (stage_budget - 16 * rows - 1024) / 12);
        c->emax = (int)std::min<int64_t>(cap_entries, budget_entries);
        if (c->variant == 3) {
            c->pfn64 = halo_kernel(c->stages, false);
            c->pfnmix = halo_kernel(c->stages, true);
        } else {
            c->sync = (c->variant == 2 && c->rows_per_tile == 256) ? o.sync : JAC_SYNC_GRID;
            c->ns = c->sync == JAC_SYNC_NEIGHBOUR;
            // kernel form 3: the grid-synchronised FP64 kernel over a split interface layout;
            // form 4: the grid-synchronised FP64 kernel with the local stopping tests
            const int form = sp ? 3 : c->stop == JAC_STOP_LOCAL ? 4 : c->sync;
            c->pfn64 = persistent_kernel(c->rows_per_tile, c->stages, false, c->lanes, form);
            c->pfn64grid = persistent_kernel(c->rows_per_tile, c->stages, false, c->lanes, sp ? 3 : JAC_SYNC_GRID);
            // split layouts are FP64 only: no mixed kernels.  A mixed cycle runs as
            // two launches: the FP64 residual pass, then the FP32 inner sweeps.
            c->pfnmix = sp ? nullptr : persistent_kernel(c->rows_per_tile, c->stages, true, c->lanes, 0, 1);
            c->pfnmix32 = sp ? nullptr : persistent_kernel(c->rows_per_tile, c->stages, true, c->lanes, 0, 2);
            c->smem = persistent_smem_bytes(rows, c->emax, c->stages);
        }
        c->threads = (c->variant == 3) ? 256 + 32 : persistent_threads(c->rows_per_tile);
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        auto occupancy = [&](int smem_bytes) -> int {
            if (!c->pfn64 || (!c->pfnmix && !sp)) return 0;
            if (c->pfnmix32 && c->variant == 2) {
                int a4 = 0;
                if (cudaFuncSetAttribute(c->pfnmix32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
                        cudaSuccess ||
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a4, c->pfnmix32, c->threads, smem_bytes) !=
                        cudaSuccess || a4 < 1) {
                    cudaGetLastError();
                    return 0;
                }
            }
            const void* fmix = c->pfnmix ? c->pfnmix : c->pfn64;
            if (cudaFuncSetAttribute(c->pfn64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess ||
                cudaFuncSetAttribute(fmix, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            int a = 0, b2 = 0, a3 = 1 << 20;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, c->pfn64, c->threads, smem_bytes) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, fmix, c->threads, smem_bytes) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            if (c->pfn64grid && c->pfn64grid != c->pfn64 &&
                (cudaFuncSetAttribute(c->pfn64grid, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
                     cudaSuccess ||
                 cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a3, c->pfn64grid, c->threads, smem_bytes) !=
                     cudaSuccess)) {
                cudaGetLastError();
                return 0;
            }
            return std::min(std::min(std::min(a, b2), a3), target_per_sm);
        };
        int per_sm = 0;
        if (c->variant == 3) {
            // The tile table's size depends on the CTA count, which depends on
            // the shared memory per CTA: try 2 CTAs/SM, then 1.
            for (int guess = 2; guess >= 1 && per_sm == 0; --guess) {
                const int ctas = guess * prop.multiProcessorCount;
                make_tiling(tf, plan, rows, c->emax, ctas, tl, row_cost);
                make_windows(tf, tl, c->xcap, c->maxruns, c->emax, win);
                int ntcap = 0, blkcap = 0;
                for (int g = 0; g < ctas; ++g) {
                    ntcap = std::max(ntcap, tl.cta0[g + 1] - tl.cta0[g]);
                    blkcap = std::max(blkcap, win.blk0[tl.cta0[g + 1]] - win.blk0[tl.cta0[g]]);
                }
                const int smem_b = halo_smem_bytes(rows, c->emax, c->xcap, ntcap, blkcap, c->stages);
                if (occupancy(smem_b) >= guess) {
                    per_sm = guess;
                    c->smem = smem_b;
                    c->ntcap = ntcap;
                    c->blkcap = blkcap;
                }
            }
            c->fallback_tiles = win.fallback_tiles;
            c->window_elems = win.window_elems;
        } else {
            per_sm = occupancy(c->smem);
        }
        if (per_sm < 1 || !coop) {
            if (o.variant >= 2) {
                char msg[200];
                std::snprintf(msg, sizeof(msg),
                              "persistent kernel cannot be made co-resident (rows %d, smem %d B, %d CTAs/SM, coop %d)",
                              rows, c->smem, per_sm, coop);
                return fail(nullptr, JAC_EINVAL, msg);
            }
            c->variant = 1;
        } else {
            c->grid = per_sm * prop.multiProcessorCount;
            c->sms = prop.multiProcessorCount;
        }
    }
    if (c->stop == JAC_STOP_LOCAL && (c->variant != 2 || !c->pfn64))
        return fail(nullptr, JAC_EINVAL,
                    "JAC_STOP_LOCAL: the persistent kernel (256-thread tiles, 1, 2 or 4 lanes) cannot run here");
    if (c->variant == 1) {
        c->grid = (int)((n + 255) / 256);
        c->emax = 0;
    }
    // a split interface layout without calibrated costs: slot rows get their own estimate
    std::vector<double> split_cost;
    if (sp && !row_cost) {
        split_cost.resize(rows);
        for (int64_t r = 0; r < rows; ++r) {
            const int64_t len = tf.rowptr[r + 1] - tf.rowptr[r];
            split_cost[r] = r < sp->n_own ? default_row_cost(len) : slot_row_cost(len);
        }
        row_cost = &split_cost;
    }
    if (c->variant == 2 && !sp) {
        make_tiling(tf, plan, c->rows_per_tile / c->lanes, c->emax, c->grid, tl, row_cost);
    } else if (c->variant == 2) {
        make_split_tiling(*sp, c->rows_per_tile / c->lanes, c->emax, c->grid, tl, row_cost);
    }
    if (c->variant >= 2) {
        c->ntiles = (int)tl.ntiles();
        // what the balance calibration needs: each CTA's rows and the cost model used
        c->h_cta_row0.resize(c->grid + 1);
        for (int g = 0; g <= c->grid; ++g) c->h_cta_row0[g] = tl.row0[tl.cta0[g]];
        c->h_cta_row1.clear();
        if (!tl.cta1.empty()) {
            c->h_cta_row1.resize(c->grid + 1);
            for (int g = 0; g <= c->grid; ++g) c->h_cta_row1[g] = tl.row0[tl.cta1[g]];
        }
        c->h_row_cost.resize(rows);
        for (int64_t r = 0; r < rows; ++r)
            c->h_row_cost[r] = row_cost ? (*row_cost)[r] : default_row_cost(tf.rowptr[r + 1] - tf.rowptr[r]);
    }
    std::vector<int32_t> dep_ptr, dep;
    if (c->ns) {
        // each CTA's neighbours: the CTAs that own a row it reads (Sec. 4.2.2's
        // dependency lists at CTA granularity)
        const int G = c->grid;
        std::vector<int32_t> cta_of(rows);
        for (int g = 0; g < G; ++g)
            for (int64_t r = c->h_cta_row0[g]; r < c->h_cta_row0[g + 1]; ++r) cta_of[r] = g;
        std::vector<int32_t> stamp(G, -1);
        dep_ptr.assign(G + 1, 0);
        for (int g = 0; g < G; ++g) {
            for (int64_t r = c->h_cta_row0[g]; r < c->h_cta_row0[g + 1]; ++r)
                for (int64_t e = tf.rowptr[r]; e < tf.rowptr[r + 1]; ++e) {
                    const int h = cta_of[tf.col[e]];
                    if (h != g && stamp[h] != g) {
                        stamp[h] = g;
                        dep.push_back(h);
                    }
                }
            dep_ptr[g + 1] = (int32_t)dep.size();
        }
        c->dep_edges = (int64_t)dep.size();
    }
    c->nslots = c->grid;

    // ---- device buffers
    CK(nullptr, dalloc(&c->d_rowptr, rows + 1 + 16));
    CK(nullptr, dalloc(&c->d_col, nnz_off + 16));
    CK(nullptr, dalloc(&c->d_S64, nnz_off + 16));
    CK(nullptr, dalloc(&c->d_b, rows + 16));
    if (sp) {
        CK(nullptr, dalloc(&c->d_bmap, rows + 16));
        CK(nullptr, dalloc(&c->d_slot_info, sp->slot_info.size() + 16));
        CK(nullptr, cudaMemcpy(c->d_bmap, sp->bmap.data(), rows * sizeof(long long), cudaMemcpyHostToDevice));
        if (!sp->slot_info.empty())
            CK(nullptr, cudaMemcpy(c->d_slot_info, sp->slot_info.data(), sp->slot_info.size() * 4,
                                   cudaMemcpyHostToDevice));
    }
    CK(nullptr, dalloc(&c->d_d, n + 16));
    CK(nullptr, dalloc(&c->d_x[0], n + 16));
    CK(nullptr, dalloc(&c->d_x[1], n + 16));
    if (c->ns) {
        // neighbour-synchronised sweeps rotate the iterate through three
        // buffers (see k_persistent); the grid barrier ping-pongs two, which
        // keeps more of them resident in L2
        c->nbuf = 3;
        CK(nullptr, dalloc(&c->d_x[2], n + 16));
    }
    if (o.precision == JAC_MIXED) {
        CK(nullptr, dalloc(&c->d_S32, nnz_off + 16));
        CK(nullptr, dalloc(&c->d_e[0], n + 16));
        CK(nullptr, dalloc(&c->d_e[1], n + 16));
        CK(nullptr, dalloc(&c->d_dlt, n + 16));
    }
    CK(nullptr, dalloc(&c->d_part, 2 * (size_t)c->nslots + 4 + 2));
    if (c->stop == JAC_STOP_LOCAL) {
        std::vector<int32_t> mem_ptr, mem_part, mem_head;
        const Error el = local_row_sets(plan, o, mem_ptr, mem_part, mem_head, c->h_set_id);
        if (!el.ok()) return fail(nullptr, el.st, el.msg);
        c->nloc = (int)c->h_set_id.size();
        CK(nullptr, dalloc(&c->d_mem_ptr, mem_ptr.size()));
        CK(nullptr, dalloc(&c->d_mem_part, mem_part.size() + 8));
        CK(nullptr, dalloc(&c->d_mem_head, mem_head.size() + 1));
        if (!mem_head.empty())
            CK(nullptr, cudaMemcpy(c->d_mem_head, mem_head.data(), mem_head.size() * 4, cudaMemcpyHostToDevice));
        CK(nullptr, dalloc(&c->d_loc, 3 * (size_t)c->nloc));
        CK(nullptr, cudaMemcpy(c->d_mem_ptr, mem_ptr.data(), mem_ptr.size() * 4, cudaMemcpyHostToDevice));
        if (!mem_part.empty())
            CK(nullptr, cudaMemcpy(c->d_mem_part, mem_part.data(), mem_part.size() * 4, cudaMemcpyHostToDevice));
        CK(nullptr, cudaMemset(c->d_loc, 0, 3 * sizeof(unsigned long long) * c->nloc));
    }
    if (c->variant >= 2) CK(nullptr, dalloc(&c->d_trace, 4 * (size_t)c->grid));
    CK(nullptr, dalloc(&c->d_ctl, 1));
    CK(nullptr, dalloc(&c->d_perm, n));
    CK(nullptr, dalloc(&c->d_stage, n + 16));
    CK(nullptr, cudaMallocHost((void**)&c->h_ctl, 2 * sizeof(JacCtl)));
    std::memset(c->h_ctl, 0, 2 * sizeof(JacCtl));
    if (o.history > 0) {
        c->hist_cap = o.history;
        CK(nullptr, dalloc(&c->d_hist, c->hist_cap));
    }
    CK(nullptr, cudaEventCreate(&c->ev0));
    CK(nullptr, cudaEventCreate(&c->ev1));
    if (c->variant == 3) {
        CK(nullptr, dalloc(&c->d_blk0, win.blk0.size()));
        CK(nullptr, dalloc(&c->d_blk, win.blk.size() + 16));
        CK(nullptr, dalloc(&c->d_lcol, win.lcol.size() + 16));
        CK(nullptr, cudaMemcpy(c->d_blk0, win.blk0.data(), win.blk0.size() * 4, cudaMemcpyHostToDevice));
        CK(nullptr, cudaMemcpy(c->d_blk, win.blk.data(), win.blk.size() * 4, cudaMemcpyHostToDevice));
        if (!win.lcol.empty())
            CK(nullptr, cudaMemcpy(c->d_lcol, win.lcol.data(), win.lcol.size() * 4, cudaMemcpyHostToDevice));
    }
    if (c->ns) {
        CK(nullptr, dalloc(&c->d_dep_ptr, dep_ptr.size()));
        CK(nullptr, dalloc(&c->d_dep, dep.size() + 1));
        CK(nullptr, dalloc(&c->d_done, (size_t)DONE_STRIDE * c->grid));
        CK(nullptr, cudaMemcpy(c->d_dep_ptr, dep_ptr.data(), dep_ptr.size() * 4, cudaMemcpyHostToDevice));
        if (!dep.empty()) CK(nullptr, cudaMemcpy(c->d_dep, dep.data(), dep.size() * 4, cudaMemcpyHostToDevice));
    }
    if (c->variant >= 2) {
        CK(nullptr, dalloc(&c->d_row0, tl.row0.size()));
        CK(nullptr, dalloc(&c->d_nnz0, tl.nnz0.size()));
        CK(nullptr, dalloc(&c->d_cta0, tl.cta0.size()));
        CK(nullptr, cudaMemcpy(c->d_row0, tl.row0.data(), tl.row0.size() * 4, cudaMemcpyHostToDevice));
        CK(nullptr, cudaMemcpy(c->d_nnz0, tl.nnz0.data(), tl.nnz0.size() * 4, cudaMemcpyHostToDevice));
        CK(nullptr, cudaMemcpy(c->d_cta0, tl.cta0.data(), tl.cta0.size() * 4, cudaMemcpyHostToDevice));
        if (!tl.cta1.empty()) {
            CK(nullptr, dalloc(&c->d_cta1, tl.cta1.size()));
            CK(nullptr, cudaMemcpy(c->d_cta1, tl.cta1.data(), tl.cta1.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    CK(nullptr, cudaMemcpy(c->d_rowptr, tf.rowptr.data(), (rows + 1) * 4, cudaMemcpyHostToDevice));
    if (nnz_off) {
        CK(nullptr, cudaMemcpy(c->d_col, tf.col.data(), nnz_off * 4, cudaMemcpyHostToDevice));
        CK(nullptr, cudaMemcpy(c->d_S64, tf.S.data(), nnz_off * 8, cudaMemcpyHostToDevice));
        if (o.precision == JAC_MIXED) {
            std::vector<float> t32(nnz_off);
            for (int64_t k = 0; k < nnz_off; ++k) t32[k] = (float)tf.S[k];
            CK(nullptr, cudaMemcpy(c->d_S32, t32.data(), nnz_off * 4, cudaMemcpyHostToDevice));
        }
    }
    CK(nullptr, cudaMemcpy(c->d_d, tf.d.data(), n * 8, cudaMemcpyHostToDevice));
    c->h_perm.assign(plan.perm.begin(), plan.perm.end());
    CK(nullptr, cudaMemcpy(c->d_perm, c->h_perm.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    // original pattern for the adjoint gradient (forward contexts)
    if (pattern) {
        const HostCSR& P = *pattern;
        CK(nullptr, dalloc(&c->d_orow, n + 1));
        CK(nullptr, dalloc(&c->d_ocol, (size_t)P.nnz()));
        CK(nullptr, cudaMemcpy(c->d_orow, P.rowptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice));
        if (P.nnz()) CK(nullptr, cudaMemcpy(c->d_ocol, P.col.data(), P.nnz() * 4, cudaMemcpyHostToDevice));
    }
    if (o.debug) {
        const size_t nn = (size_t)n;
        add_canary(C, "rowptr", c->d_rowptr, (size_t)rows + 1);
        add_canary(C, "col", c->d_col, (size_t)nnz_off);
        add_canary(C, "S64", c->d_S64, (size_t)nnz_off);
        add_canary(C, "S32", c->d_S32, (size_t)nnz_off);
        add_canary(C, "b", c->d_b, (size_t)rows);
        if (sp) {
            add_canary(C, "bmap", c->d_bmap, (size_t)rows);
            add_canary(C, "slot_info", c->d_slot_info, sp->slot_info.size());
        }
        add_canary(C, "d", c->d_d, nn);
        add_canary(C, "x[0]", c->d_x[0], nn);
        add_canary(C, "x[1]", c->d_x[1], nn);
        add_canary(C, "x[2]", c->d_x[2], nn);
        add_canary(C, "e[0]", c->d_e[0], nn);
        add_canary(C, "e[1]", c->d_e[1], nn);
        add_canary(C, "r (FP32)", c->d_dlt, nn);
        add_canary(C, "stage", c->d_stage, nn);
        const jac_status stc = set_canaries(C);
        if (stc != JAC_OK) return fail(nullptr, stc, C->err);
    }
    // right-hand side and control block
    cudaStream_t sm = stream_of(C);
    if (b) {
        st = copy_to_stage(C, b, b_memory, (size_t)n, c->d_stage);
        if (st != JAC_OK) return fail(nullptr, st, C->err);
    }
    CK(nullptr, launch_gather_b(sp ? c->d_bmap : c->d_perm, b ? c->d_stage : nullptr, c->d_b, (int)rows, (int)n,
                                c->d_ctl, sm));
    CK(nullptr, launch_reset_iterate(c->d_ctl, sm));
    CK(nullptr, launch_arm(c->d_ctl, 0, 0, o.inner_sweeps, 0, 0, -1.0, o.norm, c->d_hist, c->hist_cap, (long long)o.timeout_cycles,
                     o.fault_skip_cta, sm));
    if (fetch_ctl(C, &c->h_ctl[0]) != JAC_OK) return fail(nullptr, JAC_ECUDA, C->err);
    CK(nullptr, sm ? cudaStreamSynchronize(sm) : cudaDeviceSynchronize());
    *out = c.release();
    return JAC_OK;
}


// One context with fixed options from a CSR matrix.
// The host-side work of jac_setup that no kernel geometry changes: the
// validated matrix, the splitting and the scaled form.  The autotuner builds
// it once and sets every candidate up from it.
struct Prepared {
    HostView hv;
    HostCSR M;
    Plan plan;
    ScaledForm tf;
    int64_t halo_entries = 0;
};

static jac_status prepare(const jac_csr* A, jac_splitting s, int32_t nparts, const jac_opts& o, int dev,
                          Prepared& p)
{
    DeviceGuard guard(dev);
    jac_status st = host_view(A, p.hv, nullptr);
    if (st != JAC_OK) return st;
    Error e = host_csr_from_abi(&p.hv.csr, o.transpose != 0, p.M);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    e = make_plan(p.M, s, nparts, o, p.plan);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    e = make_scaled_form(p.M, p.plan, p.tf);
    if (!e.ok()) return fail(nullptr, e.st, e.msg);
    std::vector<int64_t> rp, rc;
    std::vector<int32_t> rf;
    dependency_lists(p.M, p.plan, rp, rf, rc);
    p.halo_entries = (int64_t)rc.size();
    return JAC_OK;
}

static jac_status setup_prepared(const Prepared& p, const jac_csr* A, const double* b, jac_opts o, int dev,
                                 const std::vector<double>* row_cost, jac_ctx** out)
{
    *out = nullptr;
    if (o.timeout_cycles == 0) o.timeout_cycles = 4000000000ull;
    jac_status st = check_opts(o, nullptr);
    if (st != JAC_OK) return st;
    DeviceGuard guard(dev);
    // without transpose, M is the caller's pattern (the adjoint gradient's)
    return setup_core(p.plan, p.tf, p.M.n, p.M.nnz(), p.halo_entries, nullptr, o.transpose ? nullptr : &p.M, b,
                      A->memory, o, dev, row_cost, out);
}

static jac_status device_of(const jac_opts& o, int* dev)
{
    *dev = o.device;
    if (*dev < 0 && cudaGetDevice(dev) != cudaSuccess) return fail(nullptr, JAC_ECUDA, "no CUDA device");
    return JAC_OK;
}

static jac_status setup_single(const jac_csr* A, const double* b, jac_splitting s, int32_t nparts, jac_opts o,
                               const std::vector<double>* row_cost, jac_ctx** out)
{
    *out = nullptr;
    if (o.timeout_cycles == 0) o.timeout_cycles = 4000000000ull;
    jac_status st = check_opts(o, nullptr);
    if (st != JAC_OK) return st;
    int dev = 0;
    st = device_of(o, &dev);
    if (st != JAC_OK) return st;
    Prepared p;
    st = prepare(A, s, nparts, o, dev, p);
    if (st != JAC_OK) return st;
    return setup_prepared(p, A, b, o, dev, row_cost, out);
}

// Autotuner: set up every candidate geometry with `make`, time a few sweeps
// of each on this matrix and keep the fastest; then re-cut its CTA row ranges
// from the measured per-CTA compute times while that keeps paying.
using MakeCtx = std::function<jac_status(const jac_opts&, const std::vector<double>*, jac_ctx**)>;
//
// cand[0] is the cost model's prior (the geometry the row lengths point to).
// Another candidate replaces it only if it is more than 5 % faster, so that
// two geometries within timing noise of each other do not swap from one
// set-up to the next.
static jac_status tune(const jac_opts& o, const std::vector<Geometry>& cand, const MakeCtx& make, jac_ctx** out)
{
    const bool async = (o.sync == JAC_SYNC_ASYNC);
    const bool log = autotune_log();
    jac_ctx* best = nullptr;
    jac_opts best_o = o;
    double best_ms = 1e30;
    jac_ctx* prior = nullptr;
    jac_opts prior_o = o;
    double prior_ms = 1e30;
    std::string first_err;
    for (size_t gi = 0; gi < cand.size(); ++gi) {
        const Geometry& g = cand[gi];
        jac_opts o2 = o;
        o2.autotune = 0;
        o2.variant = g.variant;
        o2.tile_rows = g.rows;
        o2.ctas_per_sm = g.ctas;
        if (g.lanes) o2.lanes_per_row = g.lanes;
        o2.stages = g.stages;
        o2.sync = async ? JAC_SYNC_ASYNC : g.sync;
        jac_ctx* c = nullptr;
        const jac_status st = make(o2, nullptr, &c);
        if (st != JAC_OK) {
            if (first_err.empty()) first_err = g_setup_error;
            if (st != JAC_EINVAL) return st;   // invalid matrix etc.: no geometry will do
            continue;
        }
        const double ms = time_per_sweep(c);
        if (log)
            std::fprintf(stderr, "autotune: variant %d rows %d ctas/SM %d lanes %d sync %d stages %d: %.3f us/sweep%s\n",
                         c->variant, c->rows_per_tile, c->grid / std::max(1, c->sms), c->lanes, c->sync, c->stages,
                         ms * 1e3,
                         gi == 0 ? " (prior)" : "");
        if (gi == 0) {
            prior = c;
            prior_o = o2;
            prior_ms = ms;
        } else if (ms < best_ms) {
            if (best) jac_free(best);
            best = c;
            best_o = o2;
            best_ms = ms;
        } else {
            jac_free(c);
        }
    }
    if (prior && (!best || !(best_ms < 0.95 * prior_ms))) {
        if (best) jac_free(best);
        best = prior;
        best_o = prior_o;
        best_ms = prior_ms;
    } else if (prior) {
        jac_free(prior);
    }
    if (!best) return fail(nullptr, JAC_EINVAL, "autotune: no kernel geometry could be set up: " + first_err);
    // Balance calibration: the sweep waits for the slowest CTA, so scale the
    // cost estimate of every row by its CTA's measured time per unit of
    // estimated cost and cut the ranges again.
    for (int it = 0; it < 3 && best->variant >= 2 && best->n > 0; ++it) {
        const int G = best->grid;
        std::vector<double> comp(G, 0.0);
        int64_t nct = 0;
        if (jac_get_trace(best, comp.data(), nullptr, G, &nct) != JAC_OK || nct != G) break;
        std::vector<double> w = best->h_row_cost;
        // a CTA's rows: one range, or two with a split interface layout
        auto ranges = [&](int g) {
            std::pair<int64_t, int64_t> a{best->h_cta_row0[g], best->h_cta_row0[g + 1]}, b{0, 0};
            if (!best->h_cta_row1.empty()) b = {best->h_cta_row1[g], best->h_cta_row1[g + 1]};
            return std::make_pair(a, b);
        };
        for (int g = 0; g < G; ++g) {
            const auto rg = ranges(g);
            double W = 0.0;
            for (int64_t r = rg.first.first; r < rg.first.second; ++r) W += w[r];
            for (int64_t r = rg.second.first; r < rg.second.second; ++r) W += w[r];
            if (W <= 0.0 || !(comp[g] > 0.0)) continue;
            const double f = comp[g] / W;
            for (int64_t r = rg.first.first; r < rg.first.second; ++r) w[r] *= f;
            for (int64_t r = rg.second.first; r < rg.second.second; ++r) w[r] *= f;
        }
        jac_ctx* c = nullptr;
        if (make(best_o, &w, &c) != JAC_OK) break;
        const double ms = time_per_sweep(c);
        if (ms < best_ms) {
            jac_free(best);
            best = c;
            best_ms = ms;
        } else {
            jac_free(c);
            break;
        }
    }
    *out = best;
    return JAC_OK;
}

jac_status jac_setup(const jac_csr* A, const double* b, jac_splitting s, int32_t nparts, const jac_opts* o_in,
                     jac_ctx** out)
try {
    if (!out) return fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    jac_opts o;
    jac_opts_default(&o);
    if (o_in) o = *o_in;
    if (!o.autotune) return setup_single(A, b, s, nparts, o, nullptr, out);
    // Autotuner: set up every kernel geometry, time a few sweeps of each on
    // this matrix and keep the fastest; then re-cut its CTA row ranges from
    // the measured per-CTA compute times while that keeps paying.
    if (o.variant || o.tile_rows || o.ctas_per_sm)
        return fail(nullptr, JAC_EINVAL, "autotune needs variant = tile_rows = ctas_per_sm = 0");
    const bool async = (o.sync == JAC_SYNC_ASYNC);
    // local stopping runs in the grid-synchronised 256-thread geometry with 1, 2 or 4 lanes
    const bool local_stop = (o.stop == JAC_STOP_LOCAL);
    // the host-side work, once for every candidate (after the options every
    // candidate shares are checked)
    jac_status st0 = check_opts(o, nullptr);
    if (st0 != JAC_OK) return st0;
    int dev = 0;
    st0 = device_of(o, &dev);
    if (st0 != JAC_OK) return st0;
    Prepared prep;
    st0 = prepare(A, s, nparts, o, dev, prep);
    if (st0 != JAC_OK) return st0;
    // the automatic lane count (its own arithmetic: see jac_opts.lanes_per_row)
    int la = o.lanes_per_row;
    if (la == 0) {
        jac_ctx* probe = nullptr;
        jac_opts op = o;
        op.autotune = 0;
        op.variant = 2;
        op.tile_rows = 256;
        if (setup_prepared(prep, A, b, op, dev, nullptr, &probe) == JAC_OK) {
            la = probe->lanes;
            jac_free(probe);
        }
    }
    // The cost model's prior: one lane per row with 3 CTAs/SM and 3 stages
    // (short rows, FP64-pipe and gather bound); long rows (2+ lanes) with
    // 2 CTAs/SM and 2 large stages that hold whole tiles of 256/L rows.
    std::vector<Geometry> cand;
    if (la >= 2 && !async) cand.push_back({2, 256, 2, 0, JAC_SYNC_GRID, 2});
    else cand.push_back({2, 256, 3, 0});
    auto add = [&](const Geometry& g) {
        if (local_stop && (g.variant != 2 || g.rows != 256 || g.sync != JAC_SYNC_GRID || g.lanes == 8)) return;
        for (const Geometry& h : cand)
            if (h.variant == g.variant && h.rows == g.rows && h.ctas == g.ctas && h.lanes == g.lanes &&
                h.sync == g.sync && h.stages == g.stages)
                return;
        cand.push_back(g);
    };
    add({2, 256, 2, 0});
    add({2, 256, 3, 0});
    // asynchronous relaxation runs in the 256-thread geometry only
    if (!async) {
        add({2, 224, 0, 0});
        add({2, 480, 0, 0});
        add({3, 256, 0, 0});
    }
    if (o.precision == JAC_FP64 && !async) {
        add({2, 256, 2, 0, JAC_SYNC_NEIGHBOUR});
        add({2, 256, 3, 0, JAC_SYNC_NEIGHBOUR});
    }
    if (o.lanes_per_row == 0 && la >= 1) {
        // the lane counts next to the automatic one
        for (int L : {la / 2, la * 2})
            if (L >= 1 && L <= 8) {
                add({2, 256, 2, L});
                add({2, 256, 3, L});
            }
        // long rows: larger stages hold whole tiles of 256/L rows
        if (la >= 2)
            for (int L : {la, la * 2})
                if (L <= 8) {
                    add({2, 256, 2, L == la ? 0 : L, JAC_SYNC_GRID, 3});
                    add({2, 256, 2, L == la ? 0 : L, JAC_SYNC_GRID, 2});
                }
    }
    return tune(o, cand, [&](const jac_opts& oc, const std::vector<double>* rc, jac_ctx** pc) {
        return setup_prepared(prep, A, b, oc, dev, rc, pc);
    }, out);
} catch (...) {
    return host_exception(nullptr);
}

jac_status jac_setup_local(int64_t n, int32_t nsub, const jac_local* sub, const double* b, const jac_opts* o_in,
                           jac_ctx** out)
try {
    if (!out) return fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    jac_opts o;
    jac_opts_default(&o);
    if (o_in) o = *o_in;
    if (o.timeout_cycles == 0) o.timeout_cycles = 4000000000ull;
    if (o.stop != JAC_STOP_GLOBAL) return fail(nullptr, JAC_EINVAL, "JAC_STOP_LOCAL is supported by jac_setup contexts only");
    jac_status st = check_opts(o, nullptr);
    if (st != JAC_OK) return st;
    if (o.precision != JAC_FP64 || o.nrhs != 1 || o.transpose || (o.variant != 0 && o.variant != 2) ||
        (o.tile_rows != 0 && o.tile_rows != 256) || o.sync != JAC_SYNC_GRID || o.lanes_per_row > 4)
        return fail(nullptr, JAC_EINVAL,
                    "jac_setup_local: FP64, nrhs 1, no transpose, variant 0/2 with 256-thread tiles, grid sync and "
                    "lanes_per_row <= 4 only");
    if (o.autotune && o.ctas_per_sm)
        return fail(nullptr, JAC_EINVAL, "autotune needs ctas_per_sm = 0");
    // Lane counts a row's subdomains fit (one warp of 32 / L rows holds them all).
    const int32_t mmax = split_max_multiplicity(n, nsub, sub);
    std::vector<int> lanes_ok;
    for (int L : {1, 2, 4})
        if (mmax == 0 || mmax <= 32 / L) lanes_ok.push_back(L);
    // automatic lane count: jac_setup's rule on the average local row, capped by the above
    int auto_lanes = 1;
    {
        double rows = 0.0, ent = 0.0;
        for (int32_t s2 = 0; sub && s2 < nsub; ++s2) {
            rows += std::max(0, sub[s2].n);
            ent += (double)std::max<int64_t>(0, sub[s2].nnz) - std::max(0, sub[s2].n);
        }
        const double avg = rows > 0 ? ent / rows : 0.0;
        while (auto_lanes < 4 && avg / (2.0 * auto_lanes) >= 8.0) auto_lanes *= 2;
        while (auto_lanes > 1 && std::find(lanes_ok.begin(), lanes_ok.end(), auto_lanes) == lanes_ok.end())
            auto_lanes /= 2;
    }
    // validate everything on the host before the first CUDA call
    std::map<int, SplitForm> forms;
    auto form_for = [&](int L, const SplitForm** f) -> jac_status {
        auto it = forms.find(L);
        if (it == forms.end()) {
            SplitForm sf;
            Error e = make_split_form(n, nsub, sub, 32 / L, sf);
            if (!e.ok()) return fail(nullptr, e.st, e.msg);
            it = forms.emplace(L, std::move(sf)).first;
        }
        *f = &it->second;
        return JAC_OK;
    };
    const int L0 = o.lanes_per_row ? o.lanes_per_row : auto_lanes;
    const SplitForm* f0 = nullptr;
    st = form_for(L0, &f0);
    if (st != JAC_OK) return st;
    int dev = o.device;
    if (dev < 0) {
        if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, JAC_ECUDA, "no CUDA device");
    }
    DeviceGuard guard(dev);
    auto make = [&](const jac_opts& oc, const std::vector<double>* rc, jac_ctx** pc) -> jac_status {
        jac_opts o2 = oc;
        o2.variant = 2;
        o2.tile_rows = 256;
        if (!o2.lanes_per_row) o2.lanes_per_row = L0;
        const SplitForm* f = nullptr;
        const jac_status s2 = form_for(o2.lanes_per_row, &f);
        if (s2 != JAC_OK) return s2;
        return setup_core(f->plan, f->tf, n, f->nnz_local, f->partials, f, nullptr, b, JAC_MEM_HOST, o2, dev, rc, pc);
    };
    if (!o.autotune) return make(o, nullptr, out);
    // prior first (the rule of jac_setup's autotuner), then every geometry of each lane count
    const int Lp = o.lanes_per_row ? o.lanes_per_row : L0;
    std::vector<Geometry> cand;
    if (Lp >= 2) cand.push_back({2, 256, 2, Lp, JAC_SYNC_GRID, 2});
    else cand.push_back({2, 256, 3, Lp});
    auto add = [&](const Geometry& g) {
        for (const Geometry& h : cand)
            if (h.ctas == g.ctas && h.lanes == g.lanes && h.stages == g.stages) return;
        cand.push_back(g);
    };
    for (int L : lanes_ok) {
        if (o.lanes_per_row && L != o.lanes_per_row) continue;
        add({2, 256, 2, L});
        add({2, 256, 3, L});
        if (L >= 2) {
            add({2, 256, 2, L, JAC_SYNC_GRID, 3});
            add({2, 256, 2, L, JAC_SYNC_GRID, 2});
        }
    }
    return tune(o, cand, make, out);
} catch (...) {
    return host_exception(nullptr);
}

jac_status jac_setup_batched(int32_t nsys, const jac_csr* A, const double* const* b, const jac_opts* o_in,
                             jac_ctx** out)
try {
    if (!out) return fail(nullptr, JAC_EINVAL, "out is NULL");
    *out = nullptr;
    jac_opts o;
    jac_opts_default(&o);
    if (o_in) o = *o_in;
    if (o.stop != JAC_STOP_GLOBAL) return fail(nullptr, JAC_EINVAL, "JAC_STOP_LOCAL is supported by jac_setup contexts only");
    if (o.autotune) {
        if (o.tile_rows) return fail(nullptr, JAC_EINVAL, "autotune needs tile_rows = 0");
        jac_ctx* best = nullptr;
        double best_ms = 1e30;
        for (int rows : {224, 96}) {
            jac_opts o2 = o;
            o2.autotune = 0;
            o2.tile_rows = rows;
            jac_ctx* c = nullptr;
            const jac_status st = jac_setup_batched(nsys, A, b, &o2, &c);
            if (st != JAC_OK) {
                if (st != JAC_EINVAL) return st;
                continue;
            }
            const double ms = time_per_sweep(c);
            if (autotune_log())
                std::fprintf(stderr, "autotune (batched): rows %d: %.3f us/sweep%s\n", rows, ms * 1e3,
                             rows == 224 ? " (prior)" : "");
            // 224-row tiles are the prior; 96-row tiles must be more than 5 % faster
            if (!best || ms < 0.95 * best_ms) {
                if (best) jac_free(best);
                best = c;
                best_ms = ms;
            } else {
                jac_free(c);
            }
        }
        if (!best) return fail(nullptr, JAC_EINVAL, "autotune: no batched geometry could be set up");
        *out = best;
        return JAC_OK;
    }
    if (o.timeout_cycles == 0) o.timeout_cycles = 4000000000ull;
    const int nrhs = o.nrhs;
    if (nrhs != 1 && nrhs != 2 && nrhs != 4) return fail(nullptr, JAC_EINVAL, "batched: opts.nrhs must be 1, 2 or 4");
    {
        jac_opts chk = o;
        chk.nrhs = 1;
        chk.tile_rows = 0;
        chk.lanes_per_row = 0;
        jac_status st = check_opts(chk, nullptr);
        if (st != JAC_OK) return st;
    }
    if (nsys < 1 || nsys > 65536 || !A) return fail(nullptr, JAC_EINVAL, "batched: need 1 <= nsys <= 65536 systems");
    const int memory = A[0].memory;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, JAC_ECUDA, "no CUDA device");
    DeviceGuard guard(dev);

    // ---- pack the systems block-diagonally in iteration-matrix form
    ScaledForm big;
    big.rowptr.push_back(0);
    std::vector<long long> off(nsys + 1, 0);
    for (int s = 0; s < nsys; ++s) {
        if (A[s].memory != memory) return fail(nullptr, JAC_EINVAL, "batched: all systems must use the same memory");
        HostView hv;
        jac_status st = host_view(&A[s], hv, nullptr);
        if (st != JAC_OK) return st;
        HostCSR M;
        Error e = host_csr_from_abi(&hv.csr, o.transpose != 0, M);
        if (!e.ok()) return fail(nullptr, e.st, "system " + std::to_string(s) + ": " + e.msg);
        Plan p1;
        e = make_plan(M, JAC_BANDROW, 1, o, p1);
        ScaledForm tf;
        if (e.ok()) e = make_scaled_form(M, p1, tf);
        if (!e.ok()) return fail(nullptr, e.st, "system " + std::to_string(s) + ": " + e.msg);
        const long long base = off[s], ebase = big.rowptr.back();
        if (base + M.n > INT32_MAX - 64 || ebase + (long long)tf.col.size() > INT32_MAX - 64)
            return fail(nullptr, JAC_EINVAL, "batched: packed system exceeds 2^31 rows or entries");
        for (int64_t r = 0; r < M.n; ++r) big.rowptr.push_back((int32_t)(ebase + tf.rowptr[r + 1]));
        for (size_t q = 0; q < tf.col.size(); ++q) big.col.push_back((int32_t)(tf.col[q] + base));
        big.S.insert(big.S.end(), tf.S.begin(), tf.S.end());
        big.d.insert(big.d.end(), tf.d.begin(), tf.d.end());
        big.max_off = std::max(big.max_off, tf.max_off);
        off[s + 1] = base + M.n;
    }
    const int64_t n = off[nsys];
    big.n = n;
    const int64_t nnz_off = big.rowptr[n];
    Plan plan;
    plan.part_ptr.assign(off.begin(), off.end());
    plan.perm.resize(n);
    std::iota(plan.perm.begin(), plan.perm.end(), 0);
    plan.iperm = plan.perm;

    std::unique_ptr<jac_ctx, void (*)(jac_ctx*)> c(new jac_ctx(), destroy);
    jac_ctx* C = c.get();
    c->device = dev;
    c->stream = (cudaStream_t)o.stream;
    c->o = o;
    c->batched = true;
    c->nsys = nsys;
    c->nrhs = nrhs;
    c->n = n;
    c->rows = n;
    c->nnz = nnz_off + n;
    c->nnz_off = nnz_off;
    c->max_off = big.max_off;
    c->max_row = big.max_off + 1;
    c->splitting = JAC_BANDROW;
    c->precision = o.precision;
    c->nparts = nsys;
    c->K = o.sweeps_per_graph;
    c->variant = 2;
    c->h_sys_off = off;

    // ---- launch configuration: 7 math warps + producer, 2 CTAs/SM, 4 stages
    cudaDeviceProp prop;
    CK(nullptr, cudaGetDeviceProperties(&prop, dev));
    const int rows = o.tile_rows ? o.tile_rows : 224;
    if (rows != 224 && rows != 96) return fail(nullptr, JAC_EINVAL, "batched: opts.tile_rows must be 0, 96 or 224");
    c->rows_per_tile = rows;
    c->stages = 4;
    {
        const int64_t cap_entries = std::max<int64_t>(1, big.max_off) * rows;
        const int64_t budget = 27 * 1024 - (int64_t)rows * (4 + 8 * nrhs) - 1024;
        c->emax = (int)std::min<int64_t>(cap_entries, std::max<int64_t>(rows, budget / 12));
    }
    c->pfn64 = batched_kernel(nrhs, false, rows, 0);
    c->pfnmix = batched_kernel(nrhs, true, rows, 1);
    c->pfnmix32 = batched_kernel(nrhs, true, rows, 2);
    c->smem = batched_smem_bytes(rows, c->emax, nrhs, c->stages);
    c->threads = batched_threads(rows);
    int per_sm = 0;
    {
        CK(nullptr, cudaFuncSetAttribute(c->pfn64, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem));
        CK(nullptr, cudaFuncSetAttribute(c->pfnmix, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem));
        CK(nullptr, cudaFuncSetAttribute(c->pfnmix32, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem));
        int a1 = 0, a2 = 0, a3 = 0;
        CK(nullptr, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a1, c->pfn64, c->threads, c->smem));
        CK(nullptr, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a2, c->pfnmix, c->threads, c->smem));
        CK(nullptr, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a3, c->pfnmix32, c->threads, c->smem));
        per_sm = std::min(std::min(std::min(a1, a2), a3), rows == 96 ? 4 : 2);
    }
    if (per_sm < 1) return fail(nullptr, JAC_EINVAL, "batched kernel cannot be made co-resident");
    c->grid = per_sm * prop.multiProcessorCount;
    c->sms = prop.multiProcessorCount;
    c->nslots = c->grid;
    c->h_rowptr = big.rowptr;

    // ---- device memory
    const size_t nv = (size_t)n * nrhs;
    CK(nullptr, dalloc(&c->d_rowptr, n + 1 + 16));
    CK(nullptr, dalloc(&c->d_col, nnz_off + 16));
    CK(nullptr, dalloc(&c->d_S64, nnz_off + 16));
    CK(nullptr, dalloc(&c->d_b, nv + 16 * nrhs));
    CK(nullptr, dalloc(&c->d_d, n + 16));
    CK(nullptr, dalloc(&c->d_x[0], nv + 16 * nrhs));
    CK(nullptr, dalloc(&c->d_x[1], nv + 16 * nrhs));
    if (o.precision == JAC_MIXED) {
        CK(nullptr, dalloc(&c->d_S32, nnz_off + 16));
        CK(nullptr, dalloc(&c->d_e[0], nv + 16 * nrhs));
        CK(nullptr, dalloc(&c->d_e[1], nv + 16 * nrhs));
        CK(nullptr, dalloc(&c->d_dlt, nv + 16 * nrhs));
    }
    CK(nullptr, dalloc(&c->d_part, 2 * (size_t)c->nslots + 4 + 2));
    CK(nullptr, dalloc(&c->d_ctl, 1));
    CK(nullptr, dalloc(&c->d_bstage, nv + 16));
    CK(nullptr, cudaMallocHost((void**)&c->h_ctl, 2 * sizeof(JacCtl)));
    std::memset(c->h_ctl, 0, 2 * sizeof(JacCtl));
    CK(nullptr, cudaEventCreate(&c->ev0));
    CK(nullptr, cudaEventCreate(&c->ev1));
    CK(nullptr, dalloc(&c->d_bnorm, (size_t)nsys * nrhs));
    CK(nullptr, dalloc(&c->d_cnt, 2 * (size_t)nsys));
    CK(nullptr, dalloc(&c->d_mask, (size_t)nsys));
    CK(nullptr, dalloc(&c->d_ksys, (size_t)nsys * nrhs));
    CK(nullptr, dalloc(&c->d_kpar, (size_t)nsys * nrhs));
    CK(nullptr, dalloc(&c->d_rel, (size_t)nsys * nrhs));
    CK(nullptr, dalloc(&c->d_sys_status, (size_t)nsys));
    CK(nullptr, dalloc(&c->d_ndone, 1));
    CK(nullptr, dalloc(&c->d_row_sys, (size_t)n));
    CK(nullptr, dalloc(&c->d_sys_off, (size_t)nsys + 1));
    auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    std::vector<int32_t> row_sys(n);
    for (int s = 0; s < nsys; ++s)
        for (long long r = off[s]; r < off[s + 1]; ++r) row_sys[r] = s;
    CK(nullptr, up(c->d_rowptr, big.rowptr.data(), (n + 1) * 4));
    CK(nullptr, up(c->d_col, big.col.data(), nnz_off * 4));
    CK(nullptr, up(c->d_S64, big.S.data(), nnz_off * 8));
    if (o.precision == JAC_MIXED && nnz_off) {
        std::vector<float> t32(nnz_off);
        for (int64_t q = 0; q < nnz_off; ++q) t32[q] = (float)big.S[q];
        CK(nullptr, up(c->d_S32, t32.data(), nnz_off * 4));
    }
    CK(nullptr, up(c->d_d, big.d.data(), n * 8));
    CK(nullptr, up(c->d_row_sys, row_sys.data(), row_sys.size() * 4));
    {
        const jac_status st_t = batched_tile(C, std::vector<int32_t>(), true);
        if (st_t != JAC_OK) return fail(nullptr, st_t, C->err);
    }
    CK(nullptr, up(c->d_sys_off, off.data(), off.size() * 8));
    // right-hand sides: packed n x nrhs, then c = b / a_ii and ||b_s,q||
    cudaStream_t sm = stream_of(C);
    if (b) {
        for (int s = 0; s < nsys; ++s) {
            const size_t cnt = (size_t)(off[s + 1] - off[s]) * nrhs;
            if (!b[s]) {
                CK(nullptr, cudaMemsetAsync(c->d_bstage + off[s] * nrhs, 0, cnt * 8, sm));
                continue;
            }
            CK(nullptr, cudaMemcpyAsync(c->d_bstage + off[s] * nrhs, b[s], cnt * 8,
                                        memory == JAC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        sm));
        }
    }
    CK(nullptr, cudaMemcpyAsync(c->d_b, c->d_bstage, (size_t)n * nrhs * 8, cudaMemcpyDeviceToDevice, sm));
    CK(nullptr, launch_batched_bnorm(c->d_bstage, c->d_sys_off, nsys, nrhs, c->d_bnorm, sm));
    CK(nullptr, launch_batched_reset(devbatch(C), nrhs, sm));
    CK(nullptr, launch_reset_iterate(c->d_ctl, sm));
    CK(nullptr, launch_arm(c->d_ctl, 0, 0, o.inner_sweeps, 0, 0, -1.0, o.norm, nullptr, 0,
                           (long long)o.timeout_cycles, -1, sm));
    if (fetch_ctl(C, &c->h_ctl[0]) != JAC_OK) return fail(nullptr, JAC_ECUDA, C->err);
    CK(nullptr, sm ? cudaStreamSynchronize(sm) : cudaDeviceSynchronize());
    *out = c.release();
    return JAC_OK;
} catch (...) {
    return host_exception(nullptr);
}

jac_status jac_set_x(jac_ctx* c, const double* x, int32_t memory)
try {
    if (!c) return JAC_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    if (c->batched) {
        const size_t cnt = (size_t)c->n * c->nrhs;
        if (x) {
            if (memory != JAC_MEM_HOST && memory != JAC_MEM_DEVICE) return fail(c, JAC_EINVAL, "bad memory");
            CK(c, cudaMemcpyAsync(c->d_x[0], x, cnt * 8,
                                  memory == JAC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
            CK(c, launch_batched_scale(c->d_x[0], c->d_d, c->n, c->nrhs, s));
        } else {
            CK(c, cudaMemsetAsync(c->d_x[0], 0, cnt * 8, s));
        }
        CK(c, launch_batched_reset(devbatch(c), c->nrhs, s));
        CK(c, launch_reset_iterate(c->d_ctl, s));
        if (fetch_ctl(c, &c->h_ctl[0]) != JAC_OK) return JAC_ECUDA;
        CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
        c->sweeps_total = 0;
        return JAC_OK;
    }
    if (x) {
        jac_status st = copy_to_stage(c, x, memory, (size_t)c->n, c->d_stage);
        if (st != JAC_OK) return st;
    }
    CK(c, launch_gather_rows(c->d_perm, x ? c->d_stage : nullptr, c->d_d, c->d_x[0], (int)c->n, 1, s));
    CK(c, launch_reset_iterate(c->d_ctl, s));
    if (fetch_ctl(c, &c->h_ctl[0]) != JAC_OK) return JAC_ECUDA;
    CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
    c->sweeps_total = 0;
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_set_b(jac_ctx* c, const double* b, int32_t memory)
try {
    if (!c) return JAC_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    if (c->batched) {
        const size_t cnt = (size_t)c->n * c->nrhs;
        if (b) CK(c, cudaMemcpyAsync(c->d_bstage, b, cnt * 8,
                                     memory == JAC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        else CK(c, cudaMemsetAsync(c->d_bstage, 0, cnt * 8, s));
        CK(c, cudaMemcpyAsync(c->d_b, c->d_bstage, cnt * 8, cudaMemcpyDeviceToDevice, s));
        CK(c, launch_batched_bnorm(c->d_bstage, c->d_sys_off, c->nsys, c->nrhs, c->d_bnorm, s));
        CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
        return JAC_OK;
    }
    if (b) {
        jac_status st = copy_to_stage(c, b, memory, (size_t)c->n, c->d_stage);
        if (st != JAC_OK) return st;
    }
    CK(c, launch_gather_b(c->split ? c->d_bmap : c->d_perm, b ? c->d_stage : nullptr, c->d_b, (int)c->rows,
                          (int)c->n, c->d_ctl, s));
    CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_sweep(jac_ctx* c, int32_t k, double* relres_out)
try {
    if (!c) return JAC_EINVAL;
    if (k < 0) return fail(c, JAC_EINVAL, "k must be >= 0");
    if (k == 0) {
        if (relres_out) *relres_out = c->h_ctl[0].relres;
        return JAC_OK;
    }
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    if (c->batched) {
        jac_status st0 = batched_restart(c);
        if (st0 != JAC_OK) return st0;
    }
    jac_status st = arm(c, 0, 0, 0, k, -1.0);
    if (st != JAC_OK) return st;
    const int launches = (k + c->K - 1) / c->K;
    CK(c, cudaEventRecord(c->ev0, s));
    for (int i = 0; i < launches; ++i) {
        st = run_graph(c, false);
        if (st != JAC_OK) return st;
    }
    CK(c, cudaEventRecord(c->ev1, s));
    st = fetch_ctl(c, &c->h_ctl[0]);
    if (st != JAC_OK) return st;
    CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->last_ms = ms;
    const JacCtl& h = c->h_ctl[0];
    st = status_from_ctl(c, h);
    if (st != JAC_OK) return st;
    c->sweeps_total += h.evals;
    if (relres_out) *relres_out = h.relres;
    if (!c->canaries.empty()) return check_canaries(c);
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

static jac_status solve_impl(jac_ctx* c, double tol, int64_t maxit, int64_t* sweeps_out, double* relres_out);

jac_status jac_solve(jac_ctx* c, double tol, int64_t maxit, int64_t* sweeps_out, double* relres_out)
try {
    if (!c) return JAC_EINVAL;
    if (c->sync != JAC_SYNC_ASYNC || c->precision != JAC_FP64 || c->batched)
        return solve_impl(c, tol, maxit, sweeps_out, relres_out);
    // Asynchronous relaxation until CTA 0's estimate of the test value passes
    // (or maxit passes), then the synchronous test of the resulting iterate,
    // which continues with synchronous sweeps if the estimate was optimistic.
    jac_status st = solve_impl(c, tol, maxit, nullptr, nullptr);
    if (st != JAC_OK && st != JAC_ENOTCONV) return st;
    const double ms_async = c->last_ms;
    c->certify = true;
    st = solve_impl(c, tol, maxit, sweeps_out, relres_out);
    c->certify = false;
    c->last_ms += ms_async;
    return st;
} catch (...) {
    if (c) c->certify = false;
    return host_exception(c);
}

static jac_status solve_impl(jac_ctx* c, double tol, int64_t maxit, int64_t* sweeps_out, double* relres_out)
{
    if (!c) return JAC_EINVAL;
    if (maxit < 0) return fail(c, JAC_EINVAL, "maxit must be >= 0");
    if (!(tol >= 0.0)) return fail(c, JAC_EINVAL, "tol must be >= 0");
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    const bool mixed = (c->precision == JAC_MIXED);
    if (c->batched) {
        jac_status st0 = batched_restart(c);
        if (st0 != JAC_OK) return st0;
    }
    jac_status st = arm(c, 1, mixed ? 1 : 0, maxit, -1, tol);
    if (st != JAC_OK) return st;
    CK(c, cudaEventRecord(c->ev0, s));
    // Launch graph steps, keeping one step in flight while the previous
    // step's control block is inspected on the host.
    JacCtl* ha = &c->h_ctl[0];
    JacCtl* hb = &c->h_ctl[1];
    // the two events are destroyed on every return path
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    CK(c, cudaEventCreateWithFlags(&ev.a, cudaEventDisableTiming));
    CK(c, cudaEventCreateWithFlags(&ev.b, cudaEventDisableTiming));
    cudaEvent_t& ea = ev.a;
    cudaEvent_t& eb = ev.b;
    st = run_graph(c, mixed);
    if (st == JAC_OK) st = fetch_ctl(c, ha);
    if (st != JAC_OK) return st;
    cudaEventRecord(ea, s);
    long long last_k = -1;
    int stalled = 0;
    // Every step runs K sweeps unless the solve is over, so a finished solve
    // needs at most (maxit + inner + 1) / K + 2 steps; more means a defect.
    const long long per_step = (c->variant == 1 && mixed) ? c->o.inner_sweeps
                               : (mixed && (c->batched || c->pfnmix32))
                                   ? (long long)mixed_cycles_per_step(c) * std::max(2, c->o.inner_sweeps)
                                                       : c->K;
    const long long step_cap = (maxit + (long long)c->o.inner_sweeps + 1) / per_step + 4;
    long long steps = 1;
    for (;;) {
        if (++steps > step_cap) {
            cudaStreamSynchronize(s);
            return fail(c, JAC_ECUDA, "the sweep loop did not terminate within its step bound");
        }
        st = run_graph(c, mixed);
        if (st == JAC_OK) st = fetch_ctl(c, hb);
        if (st != JAC_OK) return st;
        cudaEventRecord(eb, s);
        cudaError_t e = cudaEventSynchronize(ea);
        if (e != cudaSuccess) return cuda_fail(c, e, "solve loop");
        if (ha->done != DONE_RUNNING || ha->status != 0) break;
        if (c->batched) {
            // Systems that have stopped leave their CTAs idle while the grid waits
            // for the rest: once the rows still iterating fall below 95 % of the
            // tiled rows, cut tiles over those systems only (between launches).
            // Measured on GB300, 256 systems x 4 right-hand sides: FP64 2.02 s at
            // 70 %, 1.87 s at 85 %, 1.84 s at 95 %, 1.91 s at 98 %, 1.93 s when
            // any system stops (each re-tiling costs a host round trip).
            std::vector<int32_t> mask(c->nsys);
            CK(c, cudaStreamSynchronize(s));
            CK(c, cudaMemcpy(mask.data(), c->d_mask, mask.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
            const int all = (1 << c->nrhs) - 1;
            int64_t active = 0;
            for (int q = 0; q < c->nsys; ++q)
                if (mask[q] != all) active += c->h_sys_off[q + 1] - c->h_sys_off[q];
            if (active > 0 && active * 20 < c->tiled_rows * 19) {
                st = batched_tile(c, mask);
                if (st != JAC_OK) return st;
            }
        }
        const long long prog = ha->k * 4 + ha->phase + ha->evals;
        if (prog == last_k) {
            if (++stalled > 4) {
                cudaStreamSynchronize(s);
                return fail(c, JAC_ECUDA, "the sweep loop made no progress");
            }
        } else {
            stalled = 0;
        }
        last_k = prog;
        std::swap(ha, hb);
        std::swap(ea, eb);
    }
    CK(c, cudaEventRecord(c->ev1, s));
    // ev1 follows eb on the stream: once it has completed, so has every step
    cudaError_t e = cudaEventSynchronize(c->ev1);
    if (e != cudaSuccess) return cuda_fail(c, e, "solve loop");
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->last_ms = ms;
    // the later copy (hb) holds the final state; keep it in slot 0
    c->h_ctl[0] = *hb;
    const JacCtl& h = c->h_ctl[0];
    st = status_from_ctl(c, h);
    if (st != JAC_OK) return st;
    c->sweeps_total = h.k;
    c->outer_last = h.outer;
    if (c->batched) {
        // every system stopped on its own: converged, or at maxit
        std::vector<int> sst(c->nsys);
        std::vector<double> rel((size_t)c->nsys * c->nrhs);
        CK(c, cudaMemcpy(sst.data(), c->d_sys_status, sst.size() * sizeof(int), cudaMemcpyDeviceToHost));
        CK(c, cudaMemcpy(rel.data(), c->d_rel, rel.size() * sizeof(double), cudaMemcpyDeviceToHost));
        double worst = 0.0;
        for (double r : rel) worst = std::max(worst, r);
        if (sweeps_out) *sweeps_out = h.k;
        if (relres_out) *relres_out = worst;
        bool limit = false;
        for (int v : sst) {
            if (v == DONE_NUMERIC) return fail(c, JAC_ENUMERIC, "a residual became NaN or Inf");
            if (v != DONE_CONVERGED) limit = true;
        }
        if (limit) return fail(c, JAC_ENOTCONV, "maxit reached before the tolerance in some system");
        return JAC_OK;
    }
    if (sweeps_out) *sweeps_out = h.k;
    if (relres_out) *relres_out = h.relres;
    if (!c->canaries.empty()) {
        const jac_status stc = check_canaries(c);
        if (stc != JAC_OK) return stc;
    }
    if (h.done == DONE_LIMIT) return fail(c, JAC_ENOTCONV, "maxit reached before the tolerance");
    if (h.done != DONE_CONVERGED) return fail(c, JAC_ECUDA, "solve ended in an unexpected state");
    return JAC_OK;
}

jac_status jac_get_x(jac_ctx* c, double* x, int32_t memory)
try {
    if (!c || !x) return c ? fail(c, JAC_EINVAL, "x is NULL") : JAC_EINVAL;
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    const int xb = c->h_ctl[0].xbuf;
    double* src = c->d_stage;
    size_t cnt = (size_t)c->n;
    if (c->batched) {
        src = c->d_bstage;
        cnt = (size_t)c->n * c->nrhs;
        CK(c, launch_batched_gather_x(c->d_x[0], c->d_x[1], c->d_row_sys, c->d_mask, c->d_kpar, xb, c->n, c->nrhs,
                                      c->d_d, src, s));
    } else {
        CK(c, launch_scatter_rows(c->d_perm, c->d_x[xb], c->d_d, c->d_stage, (int)c->n, 1, s));
    }
    if (memory == JAC_MEM_DEVICE) {
        CK(c, cudaMemcpyAsync(x, src, cnt * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if (memory == JAC_MEM_HOST) {
        CK(c, cudaMemcpyAsync(x, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    } else {
        return fail(c, JAC_EINVAL, "memory must be JAC_MEM_HOST or JAC_MEM_DEVICE");
    }
    CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_get_history(jac_ctx* c, double* out, int64_t max, int64_t* count)
try {
    if (!c || !count) return JAC_EINVAL;
    const int64_t have = std::min<int64_t>(c->h_ctl[0].evals, c->hist_cap);
    const int64_t m = std::min<int64_t>(have, std::max<int64_t>(max, 0));
    if (m > 0 && out) {
        DeviceGuard g(c->device);
        CK(c, cudaMemcpy(out, c->d_hist, m * sizeof(double), cudaMemcpyDeviceToHost));
    }
    *count = out ? m : have;
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_get_batch_results(jac_ctx* c, int64_t* sweeps, double* relres)
try {
    if (!c) return JAC_EINVAL;
    if (!c->batched) {
        if (sweeps) sweeps[0] = c->h_ctl[0].k;
        if (relres) relres[0] = c->h_ctl[0].relres;
        return JAC_OK;
    }
    DeviceGuard g(c->device);
    const size_t cnt = (size_t)c->nsys * c->nrhs;
    if (sweeps) {
        std::vector<long long> k(cnt);
        CK(c, cudaMemcpy(k.data(), c->d_ksys, cnt * sizeof(long long), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < cnt; ++i) sweeps[i] = k[i];
    }
    if (relres) CK(c, cudaMemcpy(relres, c->d_rel, cnt * sizeof(double), cudaMemcpyDeviceToHost));
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_adjoint_grad(jac_ctx* c, const double* lambda, const double* x, double* dA, int32_t memory)
try {
    if (!c || !lambda || !x || !dA) return c ? fail(c, JAC_EINVAL, "NULL argument") : JAC_EINVAL;
    if (!c->d_orow)
        return fail(c, JAC_EINVAL, "jac_adjoint_grad needs a forward jac_setup context (not transposed, batched or "
                                   "built from local matrices)");
    DeviceGuard g(c->device);
    cudaStream_t s = stream_of(c);
    if (!c->d_stage2) CK(c, dalloc(&c->d_stage2, c->n + 16));
    if (!c->d_grad) CK(c, dalloc(&c->d_grad, (size_t)c->nnz + 16));
    jac_status st = copy_to_stage(c, lambda, memory, (size_t)c->n, c->d_stage);
    if (st != JAC_OK) return st;
    st = copy_to_stage(c, x, memory, (size_t)c->n, c->d_stage2);
    if (st != JAC_OK) return st;
    CK(c, launch_adjoint_grad(c->d_orow, c->d_ocol, c->d_stage, c->d_stage2, c->d_grad, (int)c->n, s));
    CK(c, cudaMemcpyAsync(dA, c->d_grad, c->nnz * sizeof(double),
                          memory == JAC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(c, s ? cudaStreamSynchronize(s) : cudaDeviceSynchronize());
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_get_trace(jac_ctx* c, double* compute_ms, double* wait_ms, int64_t max, int64_t* ctas)
try {
    if (!c || !ctas) return JAC_EINVAL;
    *ctas = c->d_trace ? c->grid : 0;
    if (!c->d_trace || max <= 0) return JAC_OK;
    DeviceGuard g(c->device);
    std::vector<unsigned long long> h(4 * (size_t)c->grid);
    CK(c, cudaMemcpy(h.data(), c->d_trace, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    const int64_t m = std::min<int64_t>(max, c->grid);
    for (int64_t i = 0; i < m; ++i) {
        if (compute_ms) compute_ms[i] = h[4 * i] * 1e-6;
        if (wait_ms) wait_ms[i] = h[4 * i + 1] * 1e-6;
    }
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

jac_status jac_stats(jac_ctx* c, jac_stats_t* out)
try {
    if (!c || !out) return JAC_EINVAL;
    std::memset(out, 0, sizeof(*out));
    const JacCtl& h = c->h_ctl[0];
    out->n = c->n;
    out->nnz = c->nnz;
    out->nparts = c->nparts;
    out->interface_rows = c->interface_rows;
    out->ntiles = c->ntiles;
    out->ctas = c->grid;
    out->halo_entries = c->halo_entries;
    out->max_row = c->max_row;
    out->k = h.k;
    out->sweeps_total = c->sweeps_total;
    out->outer_iterations = c->outer_last;
    out->halo_fallback_tiles = c->fallback_tiles;
    out->halo_window_elems = c->window_elems;
    out->last_relres = h.relres;
    out->last_res2 = h.res2;
    out->last_resinf = h.resinf;
    out->last_ms = c->last_ms;
    out->bytes_per_sweep_fp64 = algorithmic_bytes_fp64(c->n, c->nnz_off);
    if (c->split)   // kernel rows (rowptr, b, slot metadata) beyond the n iterate rows
        out->bytes_per_sweep_fp64 += 4.0 * (double)(c->rows - c->n) + 8.0 * (double)(c->rows - c->n) +
                                     4.0 * (double)(c->rows - c->n_own);
    out->bytes_per_sweep_fp32 = algorithmic_bytes_fp32(c->n, c->nnz_off);
    out->variant = c->variant;
    out->precision = c->precision;
    out->splitting = c->splitting;
    out->nrhs = c->nrhs;
    out->tile_rows = c->variant >= 2 ? c->rows_per_tile : 0;
    out->lanes_per_row = c->variant >= 2 ? c->lanes : 1;
    out->sync = c->sync;
    out->stages = c->variant >= 2 ? c->stages : 0;
    out->stop = c->stop;
    const int lp = c->h_ctl[0].loc_part;
    out->stop_part = (c->stop == JAC_STOP_LOCAL && lp >= 0 && lp < (int)c->h_set_id.size()) ? c->h_set_id[lp] : -1;
    out->stop_local = out->stop_part >= 0 ? c->h_ctl[0].loc_val : 0.0;
    out->ctas_per_sm = (c->variant >= 2 && c->n > 0 && c->grid > 0) ? c->grid / std::max(1, c->sms) : 0;
    return JAC_OK;
} catch (...) {
    return host_exception(c);
}

}  // extern "C"
