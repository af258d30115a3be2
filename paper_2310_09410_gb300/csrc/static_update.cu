// Allocation-free global update (opf_global_update_static, see include/opf.h).
//
// The same computation as the global update behind opf_get_solution, for
// callers that cannot allocate device memory: control loops that forbid
// allocation once they run (an allocation may block or fail at any time), and
// hosts whose device memory is handed out only by their own allocator (a
// framework's caching allocator that owns the whole device).  Its scratch (one
// FP64 objective partial per block of 256 globals) is a file-scope __device__
// array instead of memory from a handle, so the call allocates nothing.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <string>

#include "opf_internal.h"

namespace {

constexpr int kThreads = 256;

// Per-block partial sums of c^T x.  Shared by every call in a CUDA context and
// kept between calls; each call writes the entries it later reads.
static __device__ __align__(256) double g_static_partials[OPF_STATIC_MAX_BLOCKS];

// x_i = clip((sum of u over the copies of global i - c_i) / (rho N_i), lb_i, ub_i)
// and the block's share of c^T x.
__global__ void __launch_bounds__(kThreads) k_global_update_static(int n, const int *seg_off, const double *u,
                                                                   const double *c, const double *lb,
                                                                   const double *ub, double rho, double *x,
                                                                   double *partials) {
    __shared__ double red[kThreads];
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double o = 0.0;
    if (i < n) {
        const int a = seg_off[i], b = seg_off[i + 1];
        double sigma = 0.0;
        for (int q = a; q < b; ++q) sigma += u[q];
        double xv = (sigma - c[i]) / (rho * (double)(b - a));
        if (xv < lb[i]) xv = lb[i];
        if (xv > ub[i]) xv = ub[i];
        x[i] = xv;
        o = c[i] * xv;
    }
    red[threadIdx.x] = o;
    __syncthreads();
    for (int w = kThreads >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// Objective: the block partials summed in block order by one thread.
__global__ void k_sum_partials_static(int nblk, const double *partials, double *objective) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partials[b];
        *objective = s;
    }
}

// Driver entry points fetched through the runtime (no link-time dependency
// on the driver library).
using PFN_streamCtx = CUresult (*)(CUstream, CUcontext *);
using PFN_curCtx = CUresult (*)(CUcontext *);
using PFN_ctxId = CUresult (*)(CUcontext, unsigned long long *);
using PFN_push = CUresult (*)(CUcontext);
using PFN_pop = CUresult (*)(CUcontext *);

struct Drv {
    PFN_streamCtx streamCtx = nullptr;
    PFN_curCtx curCtx = nullptr;
    PFN_ctxId ctxId = nullptr;
    PFN_push push = nullptr;
    PFN_pop pop = nullptr;
    bool ok = false;
};

template <typename F>
bool entry(const char *name, F *out) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *out = reinterpret_cast<F>(p);
    return true;
}

const Drv &drv() {
    static Drv d;
    static std::once_flag once;
    std::call_once(once, [] {
        d.ok = entry("cuStreamGetCtx", &d.streamCtx) && entry("cuCtxGetCurrent", &d.curCtx) &&
               entry("cuCtxGetId", &d.ctxId) && entry("cuCtxPushCurrent", &d.push) &&
               entry("cuCtxPopCurrent", &d.pop);
    });
    return d;
}

// Device address of g_static_partials per CUDA context, keyed by the
// context's process-unique id (a destroyed and re-created context, e.g. after
// cudaDeviceReset, gets a new id, so a stale address is never reused).
std::mutex g_mu;
std::map<unsigned long long, double *> g_dev_ptr;

int fail(int code, const std::string &msg) {
    opf::set_last_error("opf_global_update_static: " + msg);
    return code;
}

}  // namespace

extern "C" int opf_global_update_static(int32_t n, const int32_t *seg_off, const double *u, const double *c,
                                        const double *lb, const double *ub, double rho, double *x,
                                        double *objective, void *stream) {
    if (n < 1 || !seg_off || !u || !c || !lb || !ub || !x || !objective || !(rho > 0.0))
        return fail(OPF_E_INVALID, "need n >= 1, rho > 0 and non-null device pointers");
    const long long nblk = ((long long)n + kThreads - 1) / kThreads;
    if (nblk > OPF_STATIC_MAX_BLOCKS)
        return fail(OPF_E_CAPACITY, "n = " + std::to_string(n) + " exceeds OPF_STATIC_MAX_GLOBALS (" +
                                        std::to_string(OPF_STATIC_MAX_GLOBALS) + ")");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Drv &d = drv();
    if (!d.ok) return fail(OPF_E_CUDA, "driver entry points for context queries unavailable");
    // The context the kernels will run in: the stream's (a stream of an SM
    // partition belongs to its own context), else the current one.
    CUcontext ctx = nullptr;
    if (s) {
        if (d.streamCtx((CUstream)s, &ctx) != CUDA_SUCCESS || !ctx) return fail(OPF_E_CUDA, "cuStreamGetCtx failed");
    } else {
        if (d.curCtx(&ctx) != CUDA_SUCCESS) return fail(OPF_E_CUDA, "cuCtxGetCurrent failed");
        if (!ctx) {
            // No context yet on this thread: the runtime makes the current
            // device's primary context on its first call, here a symbol query.
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess) return fail(OPF_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            if (d.curCtx(&ctx) != CUDA_SUCCESS || !ctx) return fail(OPF_E_CUDA, "no current context");
        }
    }
    unsigned long long id = 0;
    if (d.ctxId(ctx, &id) != CUDA_SUCCESS) return fail(OPF_E_CUDA, "cuCtxGetId failed");
    double *partials = nullptr;
    {
        // set-up, once per context with that context current: the device
        // address of the static array (host code must not use its name as an
        // address)
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_dev_ptr.find(id);
        if (it != g_dev_ptr.end()) {
            partials = it->second;
        } else {
            if (d.push(ctx) != CUDA_SUCCESS) return fail(OPF_E_CUDA, "cuCtxPushCurrent failed");
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
            CUcontext popped = nullptr;
            d.pop(&popped);
            if (e != cudaSuccess || !p)
                return fail(OPF_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            partials = static_cast<double *>(p);
            g_dev_ptr[id] = partials;
        }
    }
    k_global_update_static<<<(unsigned)nblk, kThreads, 0, s>>>(n, seg_off, u, c, lb, ub, rho, x, partials);
    k_sum_partials_static<<<1, 32, 0, s>>>((int)nblk, partials, objective);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(OPF_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return OPF_OK;
}
