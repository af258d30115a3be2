// SM partitions (green contexts): a stream whose kernels run only on a
// subset of the device's SMs, so that long single-instance solves of large
// feeders and the batched engine's resident CTAs do not take each other's SMs.
// The driver entry points are fetched through the runtime (no link-time
// dependency on the driver library).
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>

#include "opf_internal.h"

using namespace opf;

namespace {

using PFN_getRes = CUresult (*)(CUdevice, CUdevResource *, CUdevResourceType);
using PFN_split = CUresult (*)(CUdevResource *, unsigned int *, const CUdevResource *, CUdevResource *,
                               unsigned int, unsigned int);
using PFN_desc = CUresult (*)(CUdevResourceDesc *, CUdevResource *, unsigned int);
using PFN_gctx = CUresult (*)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int);
using PFN_gstream = CUresult (*)(CUstream *, CUgreenCtx, unsigned int, int);
using PFN_gdestroy = CUresult (*)(CUgreenCtx);
using PFN_sdestroy = CUresult (*)(CUstream);
using PFN_devget = CUresult (*)(CUdevice *, int);
using PFN_sgetg = CUresult (*)(CUstream, CUgreenCtx *);
using PFN_gres = CUresult (*)(CUgreenCtx, CUdevResource *, CUdevResourceType);

struct Fns {
    PFN_getRes getRes = nullptr;
    PFN_split split = nullptr;
    PFN_desc desc = nullptr;
    PFN_gctx gctx = nullptr;
    PFN_gstream gstream = nullptr;
    PFN_gdestroy gdestroy = nullptr;
    PFN_sdestroy sdestroy = nullptr;
    PFN_devget devget = nullptr;
    PFN_sgetg sgetg = nullptr;
    PFN_gres gres = nullptr;
    bool ok = false;
};

std::mutex g_mu;
std::map<void *, CUgreenCtx> g_streams;

template <typename F>
bool entry(const char *name, F *out) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 13000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *out = reinterpret_cast<F>(p);
    return true;
}

const Fns &fns() {
    static Fns f;
    static std::once_flag once;
    std::call_once(once, [] {
        f.ok = entry("cuDeviceGetDevResource", &f.getRes) && entry("cuDevSmResourceSplitByCount", &f.split) &&
               entry("cuDevResourceGenerateDesc", &f.desc) && entry("cuGreenCtxCreate", &f.gctx) &&
               entry("cuGreenCtxStreamCreate", &f.gstream) && entry("cuGreenCtxDestroy", &f.gdestroy) &&
               entry("cuStreamDestroy", &f.sdestroy) && entry("cuDeviceGet", &f.devget) &&
               entry("cuStreamGetGreenCtx", &f.sgetg) && entry("cuGreenCtxGetDevResource", &f.gres);
    });
    return f;
}

}  // namespace

extern "C" int opf_stream_create_partition(int32_t device, int32_t n_sm, int32_t priority, void **stream,
                                           int32_t *sm_count) {
    if (!stream || n_sm == 0) return OPF_E_INVALID;
    *stream = nullptr;
    if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
        set_last_error("partition: no such device");
        return OPF_E_CUDA;
    }
    const Fns &f = fns();
    if (!f.ok) { set_last_error("partition: green contexts unavailable in this driver"); return OPF_E_CUDA; }
    CUdevice dev;
    if (f.devget(&dev, device) != CUDA_SUCCESS) return OPF_E_CUDA;
    CUdevResource all;
    if (f.getRes(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) {
        set_last_error("partition: cuDeviceGetDevResource failed");
        return OPF_E_CUDA;
    }
    const unsigned want = (unsigned)(n_sm > 0 ? n_sm : -n_sm);
    if (want >= all.sm.smCount) { set_last_error("partition: more SMs than the device has"); return OPF_E_INVALID; }
    CUdevResource part, rest;
    unsigned nb = 1;
    if (f.split(&part, &nb, &all, &rest, 0, want) != CUDA_SUCCESS || nb != 1) {
        set_last_error("partition: cuDevSmResourceSplitByCount failed");
        return OPF_E_CUDA;
    }
    CUdevResource chosen = n_sm > 0 ? part : rest;
    CUdevResourceDesc desc;
    CUgreenCtx g;
    CUstream st;
    if (f.desc(&desc, &chosen, 1) != CUDA_SUCCESS || f.gctx(&g, desc, dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) {
        set_last_error("partition: cuGreenCtxCreate failed");
        return OPF_E_CUDA;
    }
    if (f.gstream(&st, g, CU_STREAM_NON_BLOCKING, priority) != CUDA_SUCCESS) {
        f.gdestroy(g);
        set_last_error("partition: cuGreenCtxStreamCreate failed");
        return OPF_E_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_streams[(void *)st] = g;
    }
    *stream = (void *)st;
    if (sm_count) *sm_count = (int32_t)chosen.sm.smCount;
    return OPF_OK;
}

extern "C" int opf_stream_destroy_partition(void *stream) {
    CUgreenCtx g = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_streams.find(stream);
        if (it == g_streams.end()) return OPF_E_INVALID;
        g = it->second;
        g_streams.erase(it);
    }
    const Fns &f = fns();
    f.sdestroy((CUstream)stream);
    f.gdestroy(g);
    return OPF_OK;
}

// A second non-blocking stream on the same SMs as `s`: in s's green context
// when s belongs to one, else an ordinary stream of the current device.
int opf::stream_sibling(cudaStream_t s, cudaStream_t *out) {
    const Fns &f = fns();
    CUgreenCtx g = nullptr;
    if (s && f.ok && f.sgetg((CUstream)s, &g) == CUDA_SUCCESS && g) {
        CUstream st;
        if (f.gstream(&st, g, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) return OPF_E_CUDA;
        *out = (cudaStream_t)st;
        return OPF_OK;
    }
    return cudaStreamCreateWithFlags(out, cudaStreamNonBlocking) == cudaSuccess ? OPF_OK : OPF_E_CUDA;
}

int opf::stream_sm_count(cudaStream_t s, int device) {
    const Fns &f = fns();
    CUgreenCtx g = nullptr;
    if (s && f.ok && f.sgetg((CUstream)s, &g) == CUDA_SUCCESS && g) {
        CUdevResource r;
        if (f.gres(g, &r, CU_DEV_RESOURCE_TYPE_SM) == CUDA_SUCCESS && r.sm.smCount > 0) return (int)r.sm.smCount;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n;
}
