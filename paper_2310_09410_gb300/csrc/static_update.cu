// Allocation-free global update (opf_global_update_static, see include/opf.h).
//
// The same computation as the global update behind opf_get_solution, for
// callers that cannot allocate device memory: work enqueued while a CUDA
// stream is being captured (cudaMalloc cannot be captured), control loops that
// forbid allocation once running, and hosts whose device memory is handed out
// only by their own allocator.  Its scratch (one FP64 objective partial per
// block of 256 globals) is a file-scope __device__ array instead of memory
// from a handle, so the call allocates nothing.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "opf_internal.h"

namespace {

constexpr int kThreads = 256;

// Per-block partial sums of c^T x.  Shared by every call on a device and kept
// between calls; each call writes the entries it later reads.
static __device__ __align__(256) double g_static_partials[OPF_STATIC_MAX_BLOCKS];

// x_i = clip((sum of u over the copies of global i - c_i) / (rho N_i), lb_i, ub_i)
// (Eq. closed_1) and the block's share of c^T x.
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

std::mutex g_mu;
constexpr int kMaxDevices = 64;
double *g_dev_ptr[kMaxDevices] = {nullptr};

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(OPF_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(OPF_E_CAPACITY, "device ordinal beyond 63");
    double *partials = nullptr;
    {
        // set-up, once per device with that device current: the device address
        // of the static array (host code must not use its name as an address)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess || !p)
                return fail(OPF_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_dev_ptr[dev] = static_cast<double *>(p);
        }
        partials = g_dev_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_global_update_static<<<(unsigned)nblk, kThreads, 0, s>>>(n, seg_off, u, c, lb, ub, rho, x, partials);
    k_sum_partials_static<<<1, 32, 0, s>>>((int)nblk, partials, objective);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(OPF_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return OPF_OK;
}
