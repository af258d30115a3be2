// Roofline probes: the FP32 (and FP64) FMA rate this device reaches under
// the clocks it runs at right now, for the denominator of the batched
// engine's fraction (that engine is bound by FP32 instruction issue, not by
// memory) and of the FP64 iterations.
//
// Every thread runs 8 independent FMA chains acc = acc * m + a; with 8 chains
// of 4-cycle latency per warp and 2 x 1024 threads per SM, each SM
// sub-partition always has an FMA ready, so the kernel reads the FP32 pipe's
// throughput.  The sums are stored so no chain is dead code.
#include <cuda_runtime.h>

#include <string>

#include "opf_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024, 2) k_fma_peak(int iters, float m, float a, float *out) {
    float acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (float)(threadIdx.x + k);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], m, a);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same with FP64 chains (this part runs FP64 FMAs at a small fraction of
// the FP32 rate: the denominator for FP64 iterations).
__global__ void __launch_bounds__(1024, 2) k_dfma_peak(int iters, double m, double a, double *out) {
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (double)(threadIdx.x + k);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], m, a);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int opf_probe_dfma(int32_t blocks, int32_t threads, int32_t iters, double *out, void *stream,
                              double *flops) {
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !out) {
        opf::set_last_error("opf_probe_dfma: need blocks >= 1, 32 <= threads <= 1024 (multiple of 32), "
                            "iters >= 1 and an output buffer");
        return OPF_E_INVALID;
    }
    k_dfma_peak<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999, 1e-3, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        opf::set_last_error(std::string("opf_probe_dfma: ") + cudaGetErrorString(e));
        return OPF_E_CUDA;
    }
    if (flops) *flops = 2.0 * kChains * 16.0 * (double)iters * (double)threads * (double)blocks;
    return OPF_OK;
}

extern "C" int opf_probe_fma(int32_t blocks, int32_t threads, int32_t iters, float *out, void *stream,
                             double *flops) {
    if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !out) {
        opf::set_last_error("opf_probe_fma: need blocks >= 1, 32 <= threads <= 1024 (multiple of 32), "
                            "iters >= 1 and an output buffer");
        return OPF_E_INVALID;
    }
    k_fma_peak<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999f, 1e-3f, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        opf::set_last_error(std::string("opf_probe_fma: ") + cudaGetErrorString(e));
        return OPF_E_CUDA;
    }
    if (flops) *flops = 2.0 * kChains * 16.0 * (double)iters * (double)threads * (double)blocks;
    return OPF_OK;
}
