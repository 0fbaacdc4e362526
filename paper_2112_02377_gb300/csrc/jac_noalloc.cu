// jac_sweep_noalloc: synchronous Jacobi sweeps that allocate no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code running under a caching allocator or memory pool that owns
// every byte of the device, code that must not hit a device-wide
// synchronisation inside cudaMalloc/cudaFree (real-time loops, work issued
// from a callback), or plug-ins whose host application forbids allocation
// after start-up.  For them this file offers one entry point that works only
// on the caller's buffers plus a fixed scratch area that is part of the
// library image itself.
//
// The scratch is a file-scope static __device__ array (JAC_NOALLOC_SCRATCH_BYTES
// bytes, 256-byte aligned).  Every GPU that loads the library holds it until
// the process exits.  Host code cannot use the array's name as a device
// address, so the first call in each CUDA context (the device's primary
// context for runtime-API callers; again after cudaDeviceReset, which makes a
// new one) looks the address up with cudaGetSymbolAddress, with that device
// current, and caches it per context; make that first call before any stream
// capture.  Under CUDA's default lazy module loading that look-up is also
// when the library's device code is loaded into the context and the array's
// device memory is committed.  All calls share the one array and it keeps the
// last call's contents: each call clears the parts that must start at zero,
// and calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/jacobi.h"

// cuCtxGetCurrent / cuCtxGetId, fetched through the runtime's driver entry
// points so that the library does not link libcuda directly.
typedef struct CUctx_st* jac_cu_context;
typedef int (*jac_cu_ctx_get_current_fn)(jac_cu_context*);
typedef int (*jac_cu_ctx_get_id_fn)(jac_cu_context, unsigned long long*);

namespace jac {
void record_thread_error(const std::string& msg);   // jac_api.cu
jac_status host_exception(jac_ctx* c) noexcept;    // jac_api.cu
}

namespace {

constexpr long long kMaxRows = 4194304;                          // 2^22 rows
constexpr int kBlock = 256;
constexpr long long kMaxBlocks = (kMaxRows + kBlock - 1) / kBlock;
// layout: [ x scratch: kMaxRows doubles ][ partials: 3 x kMaxBlocks doubles ][ control: 64 bytes ]
// (partials: sum r_i^2, max |r_i| and sum b_i^2 of each block)
constexpr size_t kOffPartial = (size_t)kMaxRows * sizeof(double);
constexpr size_t kOffCtl = kOffPartial + 3 * (size_t)kMaxBlocks * sizeof(double);
constexpr size_t kScratchBytes = kOffCtl + 64;
static_assert(kScratchBytes == JAC_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NoallocCtl {
    unsigned int ticket;    // blocks finished in the current launch
    unsigned int pad;
    double bb;              // ||b||_2^2
    double ss;              // sum r_i^2 of the last evaluated iterate
    double mx;              // max |r_i|
};

// One sweep, one thread per row, on a CSR matrix that stores its diagonal:
//   s_i = sum_{j != i} a_ij x_j (stored order),  x'_i = (b_i - s_i) / a_ii,
//   r_i = (b_i - s_i) - a_ii x_i,
// with the residual sums (and ||b||^2, from the b_i each thread reads anyway)
// reduced by the last block to finish, in block order.
__global__ void __launch_bounds__(kBlock) k_noalloc_sweep(int n, const int* __restrict__ rowptr,
                                                          const int* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ x,
                                                          double* __restrict__ y, unsigned char* scratch)
{
    double* part = reinterpret_cast<double*>(scratch + kOffPartial);
    NoallocCtl* ctl = reinterpret_cast<NoallocCtl*>(scratch + kOffCtl);
    __shared__ double s_ss[kBlock / 32], s_mx[kBlock / 32], s_bb[kBlock / 32];
    __shared__ int s_last;
    const int i = blockIdx.x * kBlock + threadIdx.x;
    double ssq = 0.0, amx = 0.0, bsq = 0.0;
    if (i < n) {
        double s = 0.0, d = 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int j = col[e];
            if (j == i) d = val[e];
            else s = __fma_rn(val[e], x[j], s);
        }
        const double bi = b[i];
        bsq = bi * bi;
        const double t = bi - s;
        y[i] = t / d;
        const double r = __fma_rn(-d, x[i], t);
        ssq = r * r;
        amx = fabs(r);
        // a zero or missing diagonal, or an overflow, is reported as NaN
        if (d == 0.0 || !(amx <= 1.7976931348623157e308)) amx = __longlong_as_double(0x7ff8000000000000ll);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ssq += __shfl_down_sync(0xffffffffu, ssq, o);
        bsq += __shfl_down_sync(0xffffffffu, bsq, o);
        const double m = __shfl_down_sync(0xffffffffu, amx, o);
        amx = (m > amx || m != m) ? m : amx;
    }
    if ((threadIdx.x & 31) == 0) {
        s_ss[threadIdx.x >> 5] = ssq;
        s_mx[threadIdx.x >> 5] = amx;
        s_bb[threadIdx.x >> 5] = bsq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0, c = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) {
            a += s_ss[w];
            c += s_bb[w];
            m = (s_mx[w] > m || s_mx[w] != s_mx[w]) ? s_mx[w] : m;
        }
        part[blockIdx.x] = a;
        part[kMaxBlocks + blockIdx.x] = m;
        part[2 * kMaxBlocks + blockIdx.x] = c;
        __threadfence();
        s_last = (atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double a = 0.0, m = 0.0, c = 0.0;
        for (unsigned q = 0; q < gridDim.x; ++q) {
            a += part[q];
            c += part[2 * kMaxBlocks + q];
            const double v = part[kMaxBlocks + q];
            m = (v > m || v != v) ? v : m;
        }
        ctl->ss = a;
        ctl->mx = m;
        ctl->bb = c;
        ctl->ticket = 0;
    }
}

std::mutex g_mu;
// scratch address per CUDA context (its process-unique id); a small table,
// reused round-robin once full
constexpr int kCtxSlots = 64;
struct AddrSlot {
    unsigned long long ctx_id;
    unsigned char* addr;
};
AddrSlot g_slots[kCtxSlots] = {};
int g_next_slot = 0;
jac_cu_ctx_get_current_fn g_get_current = nullptr;
jac_cu_ctx_get_id_fn g_get_id = nullptr;

jac_status fail(jac_status st, const std::string& m)
{
    jac::record_thread_error(m);      // readable through jac_last_error(NULL)
    return st;
}

}  // namespace

extern "C" jac_status jac_sweep_noalloc(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                                        const double* b, const double* x_in, double* x_out, int32_t k,
                                        double* relres_out, void* stream)
try {
    if (n < 1) return fail(JAC_EINVAL, "jac_sweep_noalloc: n must be >= 1");
    if (n > kMaxRows)
        return fail(JAC_EINVAL, "jac_sweep_noalloc: n exceeds the fixed scratch limit of 4194304 rows");
    if (k < 0) return fail(JAC_EINVAL, "jac_sweep_noalloc: k must be >= 0");
    if (!rowptr || !col || !val || !b || !x_in || !x_out)
        return fail(JAC_EINVAL, "jac_sweep_noalloc: NULL pointer");
    if (x_in == x_out) return fail(JAC_EINVAL, "jac_sweep_noalloc: x_in and x_out must not alias");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(JAC_ECUDA, std::string("jac_sweep_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(JAC_EINVAL, "jac_sweep_noalloc: device ordinal out of range");
    unsigned char* scratch = nullptr;
    {
        // One-time set-up per CUDA context (with its device current): the
        // device address of the static scratch array.  The array lives in the
        // context's copy of the module, so a new context (cudaDeviceReset, a
        // caller's own driver-API context) gets its own look-up.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_get_current || !g_get_id) {
            cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
            void* f1 = nullptr;
            void* f2 = nullptr;
            e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
            if (e == cudaSuccess)
                e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
            if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess)
                return fail(JAC_ECUDA, "jac_sweep_noalloc: the driver's cuCtxGetCurrent/cuCtxGetId are unavailable");
            g_get_current = reinterpret_cast<jac_cu_ctx_get_current_fn>(f1);
            g_get_id = reinterpret_cast<jac_cu_ctx_get_id_fn>(f2);
        }
        jac_cu_context cu = nullptr;
        if (g_get_current(&cu) != 0 || !cu) {
            // no context is current yet on this thread: make the device's
            // primary context current (cudaSetDevice initialises it)
            e = cudaSetDevice(dev);
            if (e != cudaSuccess || g_get_current(&cu) != 0 || !cu)
                return fail(JAC_ECUDA, "jac_sweep_noalloc: no CUDA context is current on this thread");
        }
        unsigned long long id = 0;
        if (g_get_id(cu, &id) != 0) return fail(JAC_ECUDA, "jac_sweep_noalloc: cuCtxGetId failed");
        for (int q = 0; q < kCtxSlots; ++q)
            if (g_slots[q].addr && g_slots[q].ctx_id == id) scratch = g_slots[q].addr;
        if (!scratch) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess)
                return fail(JAC_ECUDA, std::string("jac_sweep_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            scratch = static_cast<unsigned char*>(p);
            g_slots[g_next_slot] = AddrSlot{id, scratch};
            g_next_slot = (g_next_slot + 1) % kCtxSlots;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nn = (int)n;
    const int blocks = (int)((n + kBlock - 1) / kBlock);
    double* xs = reinterpret_cast<double*>(scratch);
    // the ticket must start at zero: a previous call may have been interrupted
    e = cudaMemsetAsync(scratch + kOffCtl, 0, sizeof(NoallocCtl), s);
    if (e == cudaSuccess && k == 0)
        e = cudaMemcpyAsync(x_out, x_in, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    // ping-pong between x_out and the scratch vector so that sweep k-1 writes x_out
    const double* src = x_in;
    for (int i = 0; i < k && e == cudaSuccess; ++i) {
        double* dst = ((k - 1 - i) % 2 == 0) ? x_out : xs;
        k_noalloc_sweep<<<blocks, kBlock, 0, s>>>(nn, rowptr, col, val, b, src, dst, scratch);
        e = cudaGetLastError();
        src = dst;
    }
    NoallocCtl h;
    std::memset(&h, 0, sizeof(h));
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, scratch + kOffCtl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(JAC_ECUDA, std::string("jac_sweep_noalloc: ") + cudaGetErrorString(e));
    if (k > 0) {
        if (!(h.ss <= 1.7976931348623157e308) || !(h.mx <= 1.7976931348623157e308))
            return fail(JAC_ENUMERIC, "jac_sweep_noalloc: the residual became NaN or Inf (zero diagonal or divergence)");
        if (relres_out) *relres_out = h.bb > 0.0 ? std::sqrt(h.ss) / std::sqrt(h.bb) : std::sqrt(h.ss);
    }
    return JAC_OK;
} catch (...) {
    // an error message that could not be allocated, or a failed mutex lock
    return jac::host_exception(nullptr);
}
