// Persistent grid engine: one instance spread over every co-resident CTA of a
// cooperative launch, many iterations of Algorithm 1 per launch.
//
// CTA `rank` owns a contiguous range of subsystems.  For the whole launch its
// factor columns, its slots' state (x_s - x_ref, lambda - lambda_ref), the
// shifted data of its slots' globals and the padded local vectors stay in
// shared memory; only u = rho x_s - lambda crosses CTAs, through a
// double-buffered array in L2 (global-sorted order, each global's copies
// contiguous).  Per iteration, with one grid barrier:
//   A. per own slot k: sigma = sum of u_in over the copies of g(k), the global
//      update of Eq. closed_1 for g(k) (recomputed by every CTA holding a copy
//      of it), x stored at the slot's padded-v position;
//   B. per own factor column: t_c = <F_c, x + lambda/rho>;
//   C. per own slot: the local update of Eq. closed_2 (x_s = v - F t or F t,
//      plus bbar), the dual update of Eq. ADMM-3, u_out = rho x_s - lambda;
//   -- grid barrier --
// On tested iterations each CTA adds the Sec. III-C sums of its slots in FP64
// and stores them; after the barrier every CTA sums the P partials in the
// same fixed order and takes the same stopping decision (rank 0 publishes
// the status).  The barrier wait is bounded: past the limit the CTA records
// a fault in the status and leaves, and the others follow.
// (Waiting only for the CTAs that share a global, through per-CTA epoch
// flags, measured slower on the 8500-bus feeder than this barrier: each
// iteration then paid a fence for the flag and the delays of the slowest
// CTAs spread along the chains of neighbours.)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "opf_internal.h"
#include "test_rule.cuh"

namespace opf {
namespace {

constexpr unsigned long long kBarrierLimitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Barrier `target / P` of this launch over all P CTAs (the counter is zeroed
// before the launch and gains P per barrier).  Thread 0 arrives with a
// release add (ordering the CTA's writes, made before the __syncthreads,
// before the arrival) and waits with acquire loads; a wait past the limit
// sets *fault.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, unsigned long long target,
                                             volatile int *fault) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(bar) : "memory");
        if (ld_acquire_gpu(bar) < target) {
            const unsigned long long t0 = global_ns();
            unsigned polls = 0;
            while (ld_acquire_gpu(bar) < target) {
                if ((++polls & 63u) == 0 && global_ns() - t0 > kBarrierLimitNs) {
                    *fault = 1;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return *fault == 0;
}

template <typename T>
__device__ __forceinline__ void stage(T *dst, const T *src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

template <typename T>
__device__ __forceinline__ T dot_fv(const T *__restrict__ f, const T *__restrict__ v, int npad);

template <>
__device__ __forceinline__ float dot_fv<float>(const float *__restrict__ f, const float *__restrict__ v, int npad) {
    float a0 = 0.0f, a1 = 0.0f;
    for (int r = 0; r < npad; r += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(f + r);
        const float4 b = *reinterpret_cast<const float4 *>(v + r);
        a0 = fmaf(a.x, b.x, a0);
        a1 = fmaf(a.y, b.y, a1);
        a0 = fmaf(a.z, b.z, a0);
        a1 = fmaf(a.w, b.w, a1);
    }
    return a0 + a1;
}

template <>
__device__ __forceinline__ double dot_fv<double>(const double *__restrict__ f, const double *__restrict__ v,
                                                 int npad) {
    double a0 = 0.0, a1 = 0.0;
    for (int r = 0; r < npad; r += 2) {
        const double2 a = *reinterpret_cast<const double2 *>(f + r);
        const double2 b = *reinterpret_cast<const double2 *>(v + r);
        a0 = fma(a.x, b.x, a0);
        a1 = fma(a.y, b.y, a1);
    }
    return a0 + a1;
}

// Part `part` (0..3) of <f, v> over the zero-padded column: 4-row vectors at
// rows 4 part, 4 part + 16, ...
template <typename T>
__device__ __forceinline__ T dot_fv_part(const T *__restrict__ f, const T *__restrict__ v, int npad, int part);

template <>
__device__ __forceinline__ float dot_fv_part<float>(const float *__restrict__ f, const float *__restrict__ v,
                                                    int npad, int part) {
    float a0 = 0.0f, a1 = 0.0f;
    for (int r = 4 * part; r < npad; r += 16) {
        const float4 a = *reinterpret_cast<const float4 *>(f + r);
        const float4 b = *reinterpret_cast<const float4 *>(v + r);
        a0 = fmaf(a.x, b.x, a0);
        a1 = fmaf(a.y, b.y, a1);
        a0 = fmaf(a.z, b.z, a0);
        a1 = fmaf(a.w, b.w, a1);
    }
    return a0 + a1;
}

template <>
__device__ __forceinline__ double dot_fv_part<double>(const double *__restrict__ f, const double *__restrict__ v,
                                                      int npad, int part) {
    double a0 = 0.0, a1 = 0.0;
    for (int r = 4 * part; r < npad; r += 16) {
        const double2 a = *reinterpret_cast<const double2 *>(f + r);
        const double2 b = *reinterpret_cast<const double2 *>(v + r);
        const double2 c = *reinterpret_cast<const double2 *>(f + r + 2);
        const double2 d = *reinterpret_cast<const double2 *>(v + r + 2);
        a0 = fma(a.x, b.x, a0);
        a1 = fma(a.y, b.y, a1);
        a0 = fma(c.x, d.x, a0);
        a1 = fma(c.y, d.y, a1);
    }
    return a0 + a1;
}

// Column stride of a staged factor with npad rows: npad, plus 4 words when
// npad is a multiple of 8, so that the 16-byte column reads of 8 consecutive
// threads (consecutive columns) fall in distinct bank groups.
__host__ __device__ __forceinline__ int fstride(int npad) { return npad + ((npad & 7) == 0 ? 4 : 0); }

// Part ranges: pr[field * (P + 1) + rank].
enum { GR_K = 0, GR_S, GR_J, GR_F, GR_V, GR_NFIELDS };

template <typename T, bool SPLIT>
__global__ void __launch_bounds__(kPersistMaxThreads) k_persist_engine(IterArgs<T> g, PersistLayout lay, PersistPtrs pp, T *U,
                                                         int bar_extra, int n_iters, int check_every, DevStatus *st,
                                                         double rho_d, cudaGraphConditionalHandle cond,
                                                         int use_cond) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int P = lay.P, rank = (int)blockIdx.x, P1 = P + 1, L = lay.L;
    const int *pr = pp.pr;
    unsigned long long *bar = pp.sync;          // grid barrier counter
    double *part = pp.part;                     // P x 6 partial sums of the tested iteration
    if (st->done) {
        if (use_cond && rank == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const int k0 = pr[GR_K * P1 + rank], nk = pr[GR_K * P1 + rank + 1] - k0;
    const int s0 = pr[GR_S * P1 + rank], ns = pr[GR_S * P1 + rank + 1] - s0;
    const int j0 = pr[GR_J * P1 + rank], nj = pr[GR_J * P1 + rank + 1] - j0;
    const int v0 = pr[GR_V * P1 + rank], nv = pr[GR_V * P1 + rank + 1] - v0;
    T *F = reinterpret_cast<T *>(sm + lay.off_F);
    int4 *srec = reinterpret_cast<int4 *>(sm + lay.off_srec);
    int *items = reinterpret_cast<int *>(sm + lay.off_items);
    int *meta = reinterpret_cast<int *>(sm + lay.off_meta);
    int *segp = reinterpret_cast<int *>(sm + lay.off_segp);
    int *pk = reinterpret_cast<int *>(sm + lay.off_pk);
    T *bt = reinterpret_cast<T *>(sm + lay.off_bt);
    T *ds = reinterpret_cast<T *>(sm + lay.off_ds);
    T *mu = reinterpret_cast<T *>(sm + lay.off_mu);
    T *kct = reinterpret_cast<T *>(sm + lay.off_ct);
    T *klb = reinterpret_cast<T *>(sm + lay.off_lbt);
    T *kub = reinterpret_cast<T *>(sm + lay.off_ubt);
    T *vbx = reinterpret_cast<T *>(sm + lay.off_vbx);
    T *vbw = reinterpret_cast<T *>(sm + lay.off_vbw);
    T *tb = reinterpret_cast<T *>(sm + lay.off_tb);
    T *recip = reinterpret_cast<T *>(sm + lay.off_recip);
    double *xrs = reinterpret_cast<double *>(sm + lay.off_xrs);    // x_ref of each slot's global
    double *lrs = reinterpret_cast<double *>(sm + lay.off_lrs);    // lambda_ref of each slot
    double *cobj = reinterpret_cast<double *>(sm + lay.off_cobj);  // c of the global on its first copy, else 0
    volatile int *flags = reinterpret_cast<volatile int *>(sm + lay.off_misc);          // [0] fault, [1] stop
    DevStatus *loc = reinterpret_cast<DevStatus *>(sm + lay.off_misc + 16);
    double(*red)[6] = reinterpret_cast<double(*)[6]>(sm + lay.off_misc + 16 + ((sizeof(DevStatus) + 15) & ~15));

    stage<int4>(srec, g.srec + s0, ns);
    stage<int>(items, g.citems + j0, nj);
    stage<int>(meta, g.cmeta + k0, nk);
    stage<int>(segp, g.segp + k0, nk);
    stage<int>(pk, g.pk + k0, nk);
    stage<T>(bt, g.bt + k0, nk);
    stage<T>(ds, g.ds + k0, nk);
    stage<T>(mu, g.mu + k0, nk);
    stage<T>(recip, g.recip, 256);
    stage<double>(lrs, g.lamr + k0, nk);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const int gi = g.gk[k0 + k];
        kct[k] = g.ct[gi];
        klb[k] = g.lbt[gi];
        kub[k] = g.ubt[gi];
        xrs[k] = g.xr[gi];
        cobj[k] = (g.pk[k0 + k] == (g.segp[k0 + k] >> 8)) ? g.c64[gi] : 0.0;
    }
    for (int i = threadIdx.x; i < nv; i += blockDim.x) { vbx[i] = (T)0; vbw[i] = (T)0; }
    __syncthreads();
    // factors: one warp per own subsystem, columns re-strided
    for (int i = threadIdx.x >> 5; i < ns; i += blockDim.x >> 5) {
        const int4 r = srec[i];
        const int f = r.w >> 10, npad = (r.w >> 1) & 0x1ff, cs = fstride(npad);
        const T *src = g.F + g.sub2[s0 + i].x;
        for (int e = threadIdx.x & 31; e < f * npad; e += 32) {
            const int c = e / npad;
            F[r.x + c * cs + (e - c * npad)] = src[e];
        }
    }
    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = 0;
        *loc = *st;
    }
    __syncthreads();
    const T rho = g.rho, inv_rho = g.inv_rho;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const int mt = meta[k];
        vbw[srec[mt >> 8].y + (mt & 255)] = mu[k] * inv_rho;
    }
    __syncthreads();
    unsigned long long nb = 0;
    for (int it = 0; it < n_iters; ++it) {
        const bool chk = ((it + 1) % check_every) == 0 || it == n_iters - 1;
        const T *Uin = U + (size_t)(it & 1) * L;
        T *Uout = U + (size_t)((it + 1) & 1) * L;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        // A: global update of each own slot's global, x at the slot's v position
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int sp = segp[k];
            const int us = sp >> 8, cnt = sp & 255;
            // the copies' u in flight together, summed in segment order
            T sigma = 0;
            constexpr int SEGW = sizeof(T) == 4 ? 8 : 4;    // copies' loads in flight
            for (int q0 = 0; q0 < cnt; q0 += SEGW) {
                T v[SEGW];
#pragma unroll
                for (int j = 0; j < SEGW; ++j) v[j] = (q0 + j < cnt) ? __ldcg(Uin + us + q0 + j) : (T)0;
#pragma unroll
                for (int j = 0; j < SEGW; ++j)
                    if (q0 + j < cnt) sigma += v[j];
            }
            T x = (sigma - kct[k]) * recip[cnt];
            const T lo = klb[k], hi = kub[k];
            if (x < lo) x = lo;
            if (x > hi) x = hi;
            const int mt = meta[k];
            const int pos = srec[mt >> 8].y + (mt & 255);
            vbx[pos] = x;
            vbw[pos] = x + vbw[pos];   // v = x + lambda / rho until phase C
            if (chk) {
                const double xd = xrs[k] + (double)x;
                acc[2] += xd * xd;
                acc[5] += cobj[k] * xd;
            }
        }
        __syncthreads();
        // B: t = F^T v per own factor column.  SPLIT plans (small CTAs, given
        // threads for it): each column on a group of 4 lanes (rows r, r + 16,
        // .. of a lane in 4-row vectors, then a shuffle sum), so the longest
        // column is no longer one lane's dependent chain; otherwise one lane
        // per column.  The split loop's bound is rounded to whole warps.
        if (!SPLIT || 4 * nj > (int)blockDim.x) {
            for (int j = threadIdx.x; j < nj; j += blockDim.x) {
                const int itm = items[j];
                const int4 r = srec[itm >> 8];
                const int c = itm & 255, npad = (r.w >> 1) & 0x1ff;
                tb[r.z + c] = dot_fv<T>(F + r.x + c * fstride(npad), vbw + r.y, npad);
            }
        } else {
            const int nj4 = ((4 * nj + 31) >> 5) << 5;
            for (int jj = threadIdx.x; jj < nj4; jj += blockDim.x) {
                const int j = jj >> 2, part = jj & 3;
                T acc = (T)0;
                int itm = 0;
                if (j < nj) {
                    itm = items[j];
                    const int4 r = srec[itm >> 8];
                    const int c = itm & 255, npad = (r.w >> 1) & 0x1ff;
                    acc = dot_fv_part<T>(F + r.x + c * fstride(npad), vbw + r.y, npad, part);
                }
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (j < nj && part == 0) tb[srec[itm >> 8].z + (itm & 255)] = acc;
            }
        }
        __syncthreads();
        // C: projection, dual update, u to the next iteration's buffer
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int mt = meta[k];
            const int4 r = srec[mt >> 8];
            const int row = mt & 255;
            const int f = r.w >> 10, cs = fstride((r.w >> 1) & 0x1ff), mode = r.w & 1;
            const T *Fr = F + r.x + row;
            const T *tt = tb + r.z;
            T y0 = 0, y1 = 0;
            int c = 0;
            for (; c + 1 < f; c += 2) {
                y0 += Fr[c * cs] * tt[c];
                y1 += Fr[(c + 1) * cs] * tt[c + 1];
            }
            if (c < f) y0 += Fr[c * cs] * tt[c];
            const int pos = r.y + row;
            const T x = vbx[pos];
            const T v = vbw[pos];
            const T xm = (mode ? (y0 + y1) : v - (y0 + y1)) + bt[k];
            const T res = x - xm;
            const T mu_new = mu[k] + rho * res;
            const T d_old = ds[k];
            ds[k] = xm;
            mu[k] = mu_new;
            vbw[pos] = mu_new * inv_rho;
            __stcg(Uout + pk[k], rho * xm - mu_new);
            if (chk) {
                const double xsd = xrs[k] + (double)xm;
                const double dd = (double)xm - (double)d_old;
                acc[0] += (double)res * (double)res;
                acc[1] += dd * dd;
                acc[3] += xsd * xsd;
                const double lamd = lrs[k] + (double)mu_new;
                acc[4] += lamd * lamd;
            }
        }
        if (chk) {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[q] = warp_sum_d(acc[q]);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 6; ++q) red[w][q] = acc[q];
            __syncthreads();
            if (threadIdx.x == 0) {
                double t[6] = {0, 0, 0, 0, 0, 0};
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
#pragma unroll
                    for (int q = 0; q < 6; ++q) t[q] += red[i][q];
#pragma unroll
                for (int q = 0; q < 6; ++q) __stcg(part + rank * 6 + q, t[q]);
            }
        }
        ++nb;
        if (!grid_barrier(bar, nb * (unsigned long long)(P + bar_extra), flags)) break;
        if (chk) {
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                double s6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    double v = 0.0;
                    for (int r = lane; r < P; r += 32) v += __ldcg(part + r * 6 + q);
                    s6[q] = warp_sum_d(v);
                }
                if (lane == 0) {
                    const int since = ((it + 1) % check_every) == 0 ? check_every : ((it + 1) % check_every);
                    apply_test(loc, s6, rho_d, since);
                    flags[1] = loc->done;
                    if (rank == 0) {
                        st->iter = loc->iter;
                        st->pres = loc->pres;
                        st->dres = loc->dres;
                        st->eprim = loc->eprim;
                        st->edual = loc->edual;
                        st->obj = loc->obj;
                        st->converged = loc->converged;
                        st->numeric = loc->numeric;
                        st->done = loc->done;
                    }
                }
            }
            __syncthreads();
            if (flags[1]) break;
        }
    }
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        g.mu[k0 + k] = mu[k];
        g.ds[k0 + k] = ds[k];
    }
    if (threadIdx.x == 0 && flags[0]) {
        atomicExch(&st->fault, 1);
        atomicExch(&st->done, 1);
    }
    if (use_cond && rank == 0 && threadIdx.x == 0)
        cudaGraphSetConditional(cond, (flags[0] || flags[1]) ? 0u : 1u);
}

}  // namespace

template <typename T>
int prepare_persist_engine(unsigned bytes) {
    for (const void *fn : {(const void *)k_persist_engine<T, false>, (const void *)k_persist_engine<T, true>})
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
            return -1;
    return 0;
}

// CTAs per SM that both variants reach.
template <typename T>
int persist_occupancy(int threads, unsigned bytes) {
    int n = 1 << 30;
    for (const void *fn : {(const void *)k_persist_engine<T, false>, (const void *)k_persist_engine<T, true>}) {
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, fn, threads, bytes) != cudaSuccess) return 0;
        n = std::min(n, m);
    }
    return n;
}

template <typename T>
int launch_persist_engine(const IterArgs<T> &g, const PersistLayout &lay, const PersistPtrs &pp, T *U,
                          int bar_extra, int n_iters, int check_every, DevStatus *st, double rho,
                          cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
    // the barrier counter starts at 0 in every launch
    if (cudaMemsetAsync(pp.sync, 0, sizeof(unsigned long long), s) != cudaSuccess) return -1;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(lay.P, 1, 1);
    cfg.blockDim = dim3(lay.threads, 1, 1);
    cfg.dynamicSmemBytes = lay.bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e =
        lay.split ? cudaLaunchKernelEx(&cfg, k_persist_engine<T, true>, g, lay, pp, U, bar_extra, n_iters, check_every,
                                       st, rho, cond, use_cond)
                  : cudaLaunchKernelEx(&cfg, k_persist_engine<T, false>, g, lay, pp, U, bar_extra, n_iters,
                                       check_every, st, rho, cond, use_cond);
    return e == cudaSuccess ? 0 : -1;
}

#define OPF_PERSIST_INST(T)                                                                                   \
    template int prepare_persist_engine<T>(unsigned);                                                        \
    template int persist_occupancy<T>(int, unsigned);                                                        \
    template int launch_persist_engine<T>(const IterArgs<T> &, const PersistLayout &, const PersistPtrs &,  \
                                          T *, int, int, int, DevStatus *, double,                            \
                                          cudaGraphConditionalHandle, int, cudaStream_t);
OPF_PERSIST_INST(float)
OPF_PERSIST_INST(double)
#undef OPF_PERSIST_INST

}  // namespace opf
