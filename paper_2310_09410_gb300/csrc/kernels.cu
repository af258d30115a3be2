// Device kernels of the ADMM library (sm_103a).
//
//  k_precompute   Algorithm 1 precomputation (Sec. III-B), FP64, one warp per
//                 subsystem: Gram-Schmidt with re-orthogonalisation on the rows
//                 of A_s gives an orthonormal basis Q of row(A_s); the same
//                 operations on b_s give bbar_s = A_s^+ b_s = sum_k beta_k q_k.
//                 -Abar_s = I - Q^T Q is stored as whichever factor is smaller:
//                 Q itself (mode 0, M = I - F F^T) or an orthonormal null-space
//                 basis N from pivoted Gram-Schmidt on the columns of I - Q^T Q
//                 (mode 1, M = F F^T).
//  k_tile_iter    one ADMM iteration of Algorithm 1, one CTA per tile of
//                 consecutive subsystems: global update (Eq. closed_1)
//                 recomputed per slot from the slot's segment of
//                 u = rho x_s - lambda of the previous iteration, local update
//                 (Eq. closed_2) x_s = M_s v + bbar_s with v = x_g + lambda/rho,
//                 dual update (Eq. ADMM-3), and on tested iterations the
//                 Sec. III-C sums in FP64 (k_check applies the test).
//  k_cluster_engine  the same iterations run by one thread-block cluster for
//                 many iterations with the whole instance resident in the
//                 cluster's shared memory (globals exchanged through DSMEM).
//  k_warp_engine  one warp per subsystem for a whole solve, factors in
//                 registers or shared memory, one barrier per iteration.
//
// Every quantity may be shifted by an FP64 reference point (x_ref per global,
// lambda_ref per slot): the kernels iterate on d = x_s - x_ref[g] and
// mu = lambda - lambda_ref with shifted data c~ = c + sum lambda_ref,
// bounds - x_ref and bbar~ = M (x_ref[g] + lambda_ref/rho) + bbar - x_ref[g].
// This is the same algorithm after a change of variables; with a zero
// reference it is plain ADMM.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "opf_internal.h"
#include "test_rule.cuh"

namespace opf {


// ------------------------------------------------------------------ helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool SMEM, typename T>
__device__ __forceinline__ T ld(const T *p) {
    if constexpr (SMEM) return *p;
    else return __ldg(p);
}

// ============================================================ precompute

// Coefficients c_k = <rows_k, v> for k < nr of the lane-distributed vector v
// (entries v[t] at column lane + 32 t): per-lane partials go through a
// shared/global transpose so the nr warp reductions run side by side.
__device__ __forceinline__ void project_coeffs(const double *rows, int n, int nr, const double v[RMAX],
                                               int T, int lane, double *red, double *coef) {
    for (int k = 0; k < nr; ++k) {
        double p = 0.0;
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int c = lane + 32 * t;
            if (t < T && c < n) p += rows[(long long)k * n + c] * v[t];
        }
        red[k * 32 + lane] = p;
    }
    __syncwarp();
    for (int k = lane; k < nr; k += 32) {
        double acc = 0.0;
        for (int i = 0; i < 32; ++i) acc += red[k * 32 + i];
        coef[k] = acc;
    }
    __syncwarp();
}

__device__ __forceinline__ double warp_norm(const double v[RMAX]) {
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < RMAX; ++t) s += v[t] * v[t];
    return sqrt(warp_sum(s));
}

// One warp per subsystem.  Rows of A_s (turned into Q in place), the null-space
// rows N and the reduction scratch live in shared memory when the subsystem
// fits (m <= sh_m, n <= sh_n), otherwise in the per-subsystem global scratch.
__global__ void __launch_bounds__(32) k_precompute(PreArgs a) {
    extern __shared__ __align__(16) double shp[];
    const int s = blockIdx.x;
    const int lane = threadIdx.x;
    if (s >= a.S) return;
    const int m = a.sm[s], n = a.sn[s];
    const int T = (n + 31) >> 5;
    const bool use_sh = m <= a.sh_m && n <= a.sh_n;
    const int mm = m > 0 ? m : 1;
    double *Q, *N, *red, *coef, *beta;
    if (use_sh) {
        Q = shp;
        N = Q + a.sh_m * a.sh_n;
        red = N + a.sh_n * a.sh_n;
        coef = red + 32 * (a.sh_m > a.sh_n ? a.sh_m : a.sh_n);
        beta = coef + (a.sh_m > a.sh_n ? a.sh_m : a.sh_n);
        for (int i = lane; i < m * n; i += 32) Q[i] = a.W[a.aoff[s] + i];
        for (int i = lane; i < m; i += 32) beta[i] = a.Bw[a.boff[s] + i];
    } else {
        Q = a.W + a.aoff[s];
        N = a.P + a.poff[s];
        red = N + (long long)n * n;
        coef = red + 32 * (m > n ? m : n);
        beta = a.Bw + a.boff[s];
    }
    (void)mm;
    __syncwarp();
    double bmax = 0.0;
    for (int j = lane; j < m; j += 32) bmax = fmax(bmax, fabs(beta[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    // T (optional): the identity under the same row operations, so that beta = T b
    const bool want_t = a.pinv != nullptr;
    double *Ta = nullptr, *Tr = nullptr;
    if (want_t) {
        Ta = a.Tw + a.toff[s];
        Tr = Ta + (long long)m * m;
        for (int i = lane; i < m * m; i += 32) Ta[i] = (i / m == i % m) ? 1.0 : 0.0;
        __syncwarp();
    }
    int nrj = 0;
    // classical Gram-Schmidt, applied twice, on the rows; b follows the same operations
    int r = 0, bad = 0;
    for (int j = 0; j < m; ++j) {
        double v[RMAX];
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int c = lane + 32 * t;
            v[t] = (t < T && c < n) ? Q[(long long)j * n + c] : 0.0;
        }
        double bj = beta[j];
        const double n0 = warp_norm(v);
        for (int pass = 0; pass < 2 && r > 0; ++pass) {
            project_coeffs(Q, n, r, v, T, lane, red, coef);
            for (int k = 0; k < r; ++k) {
                const double ck = coef[k];
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    const int c = lane + 32 * t;
                    if (t < T && c < n) v[t] -= ck * Q[(long long)k * n + c];
                }
                bj -= ck * beta[k];
                if (want_t)
                    for (int i = lane; i < m; i += 32) Ta[(long long)j * m + i] -= ck * Ta[(long long)k * m + i];
            }
            __syncwarp();
        }
        const double nr = warp_norm(v);
        if (n0 > 0.0 && nr > 1e-10 * n0) {
            const double inv = 1.0 / nr;
#pragma unroll
            for (int t = 0; t < RMAX; ++t) {
                const int c = lane + 32 * t;
                if (t < T && c < n) Q[(long long)r * n + c] = v[t] * inv;
            }
            __syncwarp();
            if (lane == 0) beta[r] = bj * inv;
            if (want_t)
                for (int i = lane; i < m; i += 32) Ta[(long long)r * m + i] = Ta[(long long)j * m + i] * inv;
            ++r;
        } else {
            if (want_t) {
                for (int i = lane; i < m; i += 32) Tr[(long long)nrj * m + i] = Ta[(long long)j * m + i];
                ++nrj;
            }
            if (fabs(bj) > 1e-9 * (1.0 + bmax)) bad = 1;
        }
        __syncwarp();
    }
    // A_s^+ = Q^T T_acc (n x m)
    if (want_t) {
        double *Pi = a.pinv + a.pioff[s];
        for (int c = lane; c < n; c += 32)
            for (int i = 0; i < m; ++i) {
                double acc = 0.0;
                for (int k = 0; k < r; ++k) acc += Q[(long long)k * n + c] * Ta[(long long)k * m + i];
                Pi[(long long)c * m + i] = acc;
            }
        if (lane == 0) a.nrej[s] = nrj;
        __syncwarp();
    }
    // bbar = sum_k beta_k q_k
    const int so = a.soff[s];
    for (int c = lane; c < n; c += 32) {
        double acc = 0.0;
        for (int k = 0; k < r; ++k) acc += beta[k] * Q[(long long)k * n + c];
        a.bbar[so + c] = acc;
    }
    double *F = a.F + a.foff[s];
    if (r <= n - r) {
        for (int k = 0; k < r; ++k)
            for (int c = lane; c < n; c += 32) F[(long long)k * n + c] = Q[(long long)k * n + c];
        if (lane == 0) { a.sf[s] = r; a.smode[s] = 0; }
    } else {
        // orthonormal basis of null(A_s): pivot on the column c with the largest
        // remaining norm d_c = 1 - sum_k Q_kc^2 - sum_t N_tc^2, take
        // e_c - Q^T Q e_c - N^T N e_c, orthogonalise once more, normalise
        const int nf = n - r;
        double d[RMAX];
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            const int c = lane + 32 * t;
            double acc = 1.0;
            if (t < T && c < n) {
                for (int k = 0; k < r; ++k) { const double q = Q[(long long)k * n + c]; acc -= q * q; }
            } else {
                acc = -1.0;
            }
            d[t] = acc;
        }
        for (int st = 0; st < nf; ++st) {
            double best = -2.0;
            int bc = 0x7fffffff;
#pragma unroll
            for (int t = 0; t < RMAX; ++t) {
                const int c = lane + 32 * t;
                if (t < T && c < n && d[t] > best) { best = d[t]; bc = c; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
                if (ob > best || (ob == best && oc < bc)) { best = ob; bc = oc; }
            }
            double v[RMAX];
#pragma unroll
            for (int t = 0; t < RMAX; ++t) {
                const int c = lane + 32 * t;
                double acc = (c == bc) ? 1.0 : 0.0;
                if (t < T && c < n) {
                    for (int k = 0; k < r; ++k) acc -= Q[(long long)k * n + bc] * Q[(long long)k * n + c];
                    for (int k = 0; k < st; ++k) acc -= N[(long long)k * n + bc] * N[(long long)k * n + c];
                } else {
                    acc = 0.0;
                }
                v[t] = acc;
            }
            // second pass against Q and the null rows found so far
            if (r > 0) {
                project_coeffs(Q, n, r, v, T, lane, red, coef);
                for (int k = 0; k < r; ++k) {
                    const double ck = coef[k];
#pragma unroll
                    for (int t = 0; t < RMAX; ++t) {
                        const int c = lane + 32 * t;
                        if (t < T && c < n) v[t] -= ck * Q[(long long)k * n + c];
                    }
                }
                __syncwarp();
            }
            if (st > 0) {
                project_coeffs(N, n, st, v, T, lane, red, coef);
                for (int k = 0; k < st; ++k) {
                    const double ck = coef[k];
#pragma unroll
                    for (int t = 0; t < RMAX; ++t) {
                        const int c = lane + 32 * t;
                        if (t < T && c < n) v[t] -= ck * N[(long long)k * n + c];
                    }
                }
                __syncwarp();
            }
            const double nn = warp_norm(v);
            const double inv = nn > 0.0 ? 1.0 / nn : 0.0;
#pragma unroll
            for (int t = 0; t < RMAX; ++t) {
                const int c = lane + 32 * t;
                if (t < T && c < n) {
                    const double x = v[t] * inv;
                    N[(long long)st * n + c] = x;
                    d[t] -= x * x;
                }
            }
            __syncwarp();
        }
        for (int k = 0; k < nf; ++k)
            for (int c = lane; c < n; c += 32) F[(long long)k * n + c] = N[(long long)k * n + c];
        if (lane == 0) { a.sf[s] = nf; a.smode[s] = 1; }
    }
    if (lane == 0) a.status[s] = bad;
}

// Factors written at capacity offsets (n x f, column stride n) are packed into
// the iteration layout: column stride npad = n rounded up to 4 with zero
// padding, consecutive subsystems, FP64 and FP32 copies.
__global__ void k_pack_factors(int S, const int4 *sub, const int4 *sub2, const long long *cap_off,
                               const double *src, double *dst64, float *dst32) {
    const int s = blockIdx.x;
    if (s >= S) return;
    const int4 h = sub[s], q = sub2[s];
    const int n = h.y, f = h.z, npad = q.y;
    const double *a = src + cap_off[s];
    for (int i = threadIdx.x; i < f * npad; i += blockDim.x) {
        const int c = i / npad, r = i - c * npad;
        const double v = r < n ? a[(long long)c * n + r] : 0.0;
        dst64[q.x + i] = v;
        dst32[q.x + i] = (float)v;
    }
}

// ============================================================ iteration
// A tile is a run of consecutive subsystems [s0, s1) (device order); one CTA
// processes a tile in three phases separated by barriers:
//   0. per slot k: global update x = clip((sum of u over the copies of its
//      global - c~) / (rho N), lb~, ub~) (Eq. closed_1), v = x + mu / rho;
//   1. per (subsystem, factor column c): t_c = <F_c, v> over the zero-padded
//      column with 16-byte vector loads;
//   2. per slot: y = (F t)_r, x_s = (v - y or y) + bbar~ (Eq. closed_2),
//      mu += rho (x - x_s) (Eq. ADMM-3), u = rho x_s - mu, and on tested
//      iterations the Sec. III-C sums in FP64.
// Per-subsystem records: sub = (first slot, n, f, mode), sub2 = (factor
// offset, npad, padded-v prefix, f prefix); entry S is a sentinel.

template <typename T>
__device__ __forceinline__ T dot_padded(const T *__restrict__ f, const T *__restrict__ v, int npad);

template <>
__device__ __forceinline__ float dot_padded<float>(const float *__restrict__ f, const float *__restrict__ v,
                                                   int npad) {
    float acc = 0.0f;
    for (int r = 0; r < npad; r += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(f + r);
        const float4 b = *reinterpret_cast<const float4 *>(v + r);
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        acc = fmaf(a.w, b.w, acc);
    }
    return acc;
}

template <>
__device__ __forceinline__ double dot_padded<double>(const double *__restrict__ f,
                                                     const double *__restrict__ v, int npad) {
    double acc = 0.0;
    for (int r = 0; r < npad; r += 2) {
        const double2 a = *reinterpret_cast<const double2 *>(f + r);
        const double2 b = *reinterpret_cast<const double2 *>(v + r);
        acc = fma(a.x, b.x, acc);
        acc = fma(a.y, b.y, acc);
    }
    return acc;
}

template <typename T, bool CHECK>
__device__ __forceinline__ void tile_iteration(const IterArgs<T> &a, int s0, int s1,
                                               const T *__restrict__ u_in, T *__restrict__ u_out,
                                               T *xb, T *vb, T *tb, const T *recip, double acc[6]) {
    const int4 h0 = a.sub[s0], h1 = a.sub[s1];
    const int4 q0 = a.sub2[s0];
    const int k0 = h0.x, k1 = h1.x;
    const int v0 = q0.z, j0 = q0.w, j1 = a.sub2[s1].w;
    // phase 0
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
        const int mt = a.meta[k];
        const int s = mt >> 8, r = mt & 255;
        const int sp = a.segp[k];
        const int us = sp >> 8, cnt = sp & 255;
        T sigma = 0;
        for (int q = 0; q < cnt; ++q) sigma += u_in[us + q];
        const int g = a.gk[k];
        T x = (sigma - a.ct[g]) * recip[cnt];
        const T lo = a.lbt[g], hi = a.ubt[g];
        if (x < lo) x = lo;
        if (x > hi) x = hi;
        xb[k - k0] = x;
        const int4 q2 = a.sub2[s];
        T *vs = vb + (q2.z - v0);
        vs[r] = x + a.mu[k] * a.inv_rho;
        if (r == 0)
            for (int p = a.sub[s].y; p < q2.y; ++p) vs[p] = (T)0;
    }
    __syncthreads();
    // phase 1
    for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
        const int it = a.items[j];
        const int s = it >> 8, c = it & 255;
        const int4 q2 = a.sub2[s];
        tb[q2.w - j0 + c] = dot_padded<T>(a.F + q2.x + (long long)c * q2.y, vb + (q2.z - v0), q2.y);
    }
    __syncthreads();
    // phase 2
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
        const int mt = a.meta[k];
        const int s = mt >> 8, r = mt & 255;
        const int4 h = a.sub[s];
        const int4 q2 = a.sub2[s];
        const T *Fr = a.F + q2.x + r;
        const T *tt = tb + (q2.w - j0);
        T y = 0;
        for (int c = 0; c < h.z; ++c) y += Fr[(long long)c * q2.y] * tt[c];
        const T v = vb[q2.z - v0 + r];
        const T x = xb[k - k0];
        const T xm = (h.w ? y : v - y) + a.bt[k];
        const T res = x - xm;
        const T mu_new = a.mu[k] + a.rho * res;
        const T d_old = a.ds[k];
        a.mu[k] = mu_new;
        a.ds[k] = xm;
        const int pos = a.pk[k];
        u_out[pos] = a.rho * xm - mu_new;
        if constexpr (CHECK) {
            const int g = a.gk[k];
            const double xr = a.xr[g];
            const double xgd = xr + (double)x;
            const double xsd = xr + (double)xm;
            const double dd = (double)xm - (double)d_old;
            acc[0] += (double)res * (double)res;
            acc[1] += dd * dd;
            acc[2] += xgd * xgd;
            acc[3] += xsd * xsd;
            const double lamd = a.lamr[k] + (double)mu_new;
            acc[4] += lamd * lamd;
            if (pos == (a.segp[k] >> 8)) acc[5] += a.c64[g] * xgd;
        }
    }
}

// Block sum of the six FP64 accumulators (fixed order); result in thread 0.
__device__ __forceinline__ void block_sum6(double acc[6], double (*red)[6]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
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
        for (int q = 0; q < 6; ++q) acc[q] = t[q];
    }
}

// Whole-grid engine: one CTA per tile, one launch per iteration.
template <typename T, bool CHECK>
__global__ void __launch_bounds__(256) k_tile_iter(IterArgs<T> a, const T *__restrict__ u_in,
                                                   T *__restrict__ u_out, double *partials,
                                                   const DevStatus *st, int xcap, int vcap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (st->done) return;
    T *vb = reinterpret_cast<T *>(smem_raw);
    T *xb = vb + vcap;
    T *tb = xb + xcap;
    const int s0 = a.tile_s0[blockIdx.x], s1 = a.tile_s0[blockIdx.x + 1];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    tile_iteration<T, CHECK>(a, s0, s1, u_in, u_out, xb, vb, tb, a.recip, acc);
    if constexpr (CHECK) {
        __shared__ double red[8][6];
        block_sum6(acc, red);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 6; ++q) partials[blockIdx.x * 6 + q] = acc[q];
    }
}

// Fixed-order reduction of the per-block partials (deterministic).
__global__ void __launch_bounds__(256) k_check(const double *partials, int nblk, DevStatus *st,
                                               double rho, int add_iters,
                                               cudaGraphConditionalHandle cond, int use_cond) {
    if (st->done) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    __shared__ double red[256][6];
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 6; ++q) t[q] += partials[b * 6 + q];
#pragma unroll
    for (int q = 0; q < 6; ++q) red[threadIdx.x][q] = t[q];
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) red[threadIdx.x][q] += red[threadIdx.x + w][q];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s[6];
        for (int q = 0; q < 6; ++q) s[q] = red[0][q];
        apply_test(st, s, rho, add_iters);
        if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
    }
}

// Iterations without a test advance the counter here (opf_step).
__global__ void k_add_iters(DevStatus *st, long long n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) st->iter += n;
}

// ============================================================ cluster engine
// One instance resident in the shared memory of a thread-block cluster of P
// CTAs (P = 1 .. 16); up to n_iters iterations per launch, tested every
// check_every.  CTA `rank` owns a contiguous range of subsystems (its local
// slots and factor columns) and a contiguous range of globals (their copies'
// entries of u, in u order).  Per iteration:
//   A. owner, per global i: sigma = sum of u over its copies, x_i = clip(...)
//      (Eq. closed_1); x is stored at each copy's padded-v position in the
//      CTA that holds the copy (distributed shared memory store);
//   -- cluster barrier --
//   B. per factor column: t_c = <F_c, x + w> with w = mu / rho;
//   -- CTA barrier --
//   C. per slot: y = (F t)_r, x_s = (v - y or y) + bbar~ (Eq. closed_2),
//      mu += rho (x - x_s) (Eq. ADMM-3), w = mu / rho, and u = rho x_s - mu
//      stored in the owner CTA of the slot's global;
//   -- cluster barrier --
// Remote traffic is stores only; the barriers (release / acquire) order them.
namespace cg = cooperative_groups;

template <typename T>
__device__ void copy_in(void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return;
    const unsigned char *sb = reinterpret_cast<const unsigned char *>(src);
    unsigned char *db = reinterpret_cast<unsigned char *>(dst);
    if (((reinterpret_cast<size_t>(src) | reinterpret_cast<size_t>(dst)) & 15) == 0) {
        const int4 *s4 = reinterpret_cast<const int4 *>(src);
        int4 *d4 = reinterpret_cast<int4 *>(dst);
        const size_t n4 = bytes / 16;
        for (size_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
        for (size_t i = n4 * 16 + threadIdx.x; i < bytes; i += blockDim.x) db[i] = sb[i];
    } else {
        for (size_t i = threadIdx.x; i < bytes; i += blockDim.x) db[i] = sb[i];
    }
}

template <typename T>
__device__ __forceinline__ T dot_padded2(const T *__restrict__ f, const T *__restrict__ x,
                                         const T *__restrict__ w, int npad);

template <>
__device__ __forceinline__ float dot_padded2<float>(const float *__restrict__ f, const float *__restrict__ x,
                                                    const float *__restrict__ w, int npad) {
    float a0 = 0.0f, a1 = 0.0f;
    for (int r = 0; r < npad; r += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(f + r);
        const float4 b = *reinterpret_cast<const float4 *>(x + r);
        const float4 c = *reinterpret_cast<const float4 *>(w + r);
        a0 = fmaf(a.x, b.x + c.x, a0);
        a1 = fmaf(a.y, b.y + c.y, a1);
        a0 = fmaf(a.z, b.z + c.z, a0);
        a1 = fmaf(a.w, b.w + c.w, a1);
    }
    return a0 + a1;
}

template <>
__device__ __forceinline__ double dot_padded2<double>(const double *__restrict__ f, const double *__restrict__ x,
                                                      const double *__restrict__ w, int npad) {
    double a0 = 0.0, a1 = 0.0;
    for (int r = 0; r < npad; r += 2) {
        const double2 a = *reinterpret_cast<const double2 *>(f + r);
        const double2 b = *reinterpret_cast<const double2 *>(x + r);
        const double2 c = *reinterpret_cast<const double2 *>(w + r);
        a0 = fma(a.x, b.x + c.x, a0);
        a1 = fma(a.y, b.y + c.y, a1);
    }
    return a0 + a1;
}

// Part ranges: pr[field * (P + 1) + rank], fields in this order.
enum { PR_K = 0, PR_S, PR_J, PR_F, PR_V, PR_T, PR_G, PR_U, PR_NFIELDS };

template <typename T>
__global__ void __launch_bounds__(1024) k_cluster_engine(IterArgs<T> g, ClusterLayout lay, const int *pr,
                                                         T *u_glob, int n_iters, int check_every,
                                                         DevStatus *st, double rho_d,
                                                         cudaGraphConditionalHandle cond, int use_cond) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int P = lay.P;
    const int rank = (int)cl.block_rank();
    const int P1 = P + 1;
    if (st->done) {
        if (use_cond && rank == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const int k0 = pr[PR_K * P1 + rank], nk = pr[PR_K * P1 + rank + 1] - k0;
    const int s0 = pr[PR_S * P1 + rank], ns = pr[PR_S * P1 + rank + 1] - s0;
    const int j0 = pr[PR_J * P1 + rank], nj = pr[PR_J * P1 + rank + 1] - j0;
    const int f0 = pr[PR_F * P1 + rank], nf = pr[PR_F * P1 + rank + 1] - f0;
    const int v0 = pr[PR_V * P1 + rank], nv = pr[PR_V * P1 + rank + 1] - v0;
    const int g0 = pr[PR_G * P1 + rank], ng = pr[PR_G * P1 + rank + 1] - g0;
    const int u0 = pr[PR_U * P1 + rank], nu = pr[PR_U * P1 + rank + 1] - u0;
    const int L = lay.L;
    T *F = reinterpret_cast<T *>(sm + lay.off_F);
    int4 *srec = reinterpret_cast<int4 *>(sm + lay.off_srec);
    int *items = reinterpret_cast<int *>(sm + lay.off_items);
    int *meta = reinterpret_cast<int *>(sm + lay.off_meta);
    int *udst = reinterpret_cast<int *>(sm + lay.off_udst);
    T *bt = reinterpret_cast<T *>(sm + lay.off_bt);
    T *ds = reinterpret_cast<T *>(sm + lay.off_ds);
    T *mu = reinterpret_cast<T *>(sm + lay.off_mu);
    T *vbx = reinterpret_cast<T *>(sm + lay.off_vbx);
    T *vbw = reinterpret_cast<T *>(sm + lay.off_vbw);
    T *tb = reinterpret_cast<T *>(sm + lay.off_tb);
    int *gsegp = reinterpret_cast<int *>(sm + lay.off_gsegp);
    T *ct = reinterpret_cast<T *>(sm + lay.off_ct);
    T *lbt = reinterpret_cast<T *>(sm + lay.off_lbt);
    T *ubt = reinterpret_cast<T *>(sm + lay.off_ubt);
    T *uloc = reinterpret_cast<T *>(sm + lay.off_uloc);
    int *cdst = reinterpret_cast<int *>(sm + lay.off_cdst);
    T *recip = reinterpret_cast<T *>(sm + lay.off_recip);
    double *red = reinterpret_cast<double *>(sm + lay.off_red);    // [16][6], used in rank 0
    // FP64 data of the stopping test, staged once per launch (the reference
    // point only changes between launches)
    double *xrg = reinterpret_cast<double *>(sm + lay.off_xrg);    // x_ref of owned globals
    double *cg64 = reinterpret_cast<double *>(sm + lay.off_cg);    // costs of owned globals
    double *xrs = reinterpret_cast<double *>(sm + lay.off_xrs);    // x_ref of each local slot's global
    double *lrs = reinterpret_cast<double *>(sm + lay.off_lrs);    // lambda_ref of each local slot
    int *stop = reinterpret_cast<int *>(sm + lay.off_red + 16 * 6 * sizeof(double));
    copy_in<T>(F, g.F + f0, (size_t)nf * sizeof(T));
    copy_in<T>(srec, g.srec + s0, (size_t)ns * sizeof(int4));
    copy_in<T>(items, g.citems + j0, (size_t)nj * sizeof(int));
    copy_in<T>(meta, g.cmeta + k0, (size_t)nk * sizeof(int));
    copy_in<T>(udst, g.udst + k0, (size_t)nk * sizeof(int));
    copy_in<T>(bt, g.bt + k0, (size_t)nk * sizeof(T));
    copy_in<T>(ds, g.ds + k0, (size_t)nk * sizeof(T));
    copy_in<T>(mu, g.mu + k0, (size_t)nk * sizeof(T));
    copy_in<T>(gsegp, g.gsegp + g0, (size_t)ng * sizeof(int));
    copy_in<T>(ct, g.ct + g0, (size_t)ng * sizeof(T));
    copy_in<T>(lbt, g.lbt + g0, (size_t)ng * sizeof(T));
    copy_in<T>(ubt, g.ubt + g0, (size_t)ng * sizeof(T));
    copy_in<T>(uloc, u_glob + u0, (size_t)nu * sizeof(T));
    copy_in<T>(cdst, g.cdst + u0, (size_t)nu * sizeof(int));
    copy_in<T>(recip, g.recip, 256 * sizeof(T));
    copy_in<T>(xrg, g.xr + g0, (size_t)ng * sizeof(double));
    copy_in<T>(cg64, g.c64 + g0, (size_t)ng * sizeof(double));
    copy_in<T>(lrs, g.lamr + k0, (size_t)nk * sizeof(double));
    for (int k = threadIdx.x; k < nk; k += blockDim.x) xrs[k] = g.xr[g.gk[k0 + k]];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) { vbx[i] = (T)0; vbw[i] = (T)0; }
    if (threadIdx.x == 0) *stop = 0;
    __syncthreads();
    const T rho = g.rho, inv_rho = g.inv_rho;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const int mt = meta[k];
        vbw[srec[mt >> 8].y + (mt & 255)] = mu[k] * inv_rho;
    }
    cl.sync();   // every CTA staged before the first remote store
    T *u_prev = u_glob + L;
    int it = 0;
    for (it = 0; it < n_iters; ++it) {
        const bool chk = ((it + 1) % check_every) == 0 || it == n_iters - 1;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        // A: owner global update, x to every copy
        for (int i = threadIdx.x; i < ng; i += blockDim.x) {
            const int sp = gsegp[i];
            const int p0 = sp >> 8, cnt = sp & 255;
            T sigma = 0;
            for (int q = 0; q < cnt; ++q) sigma += uloc[p0 + q];
            T x = (sigma - ct[i]) * recip[cnt];
            const T lo = lbt[i], hi = ubt[i];
            if (x < lo) x = lo;
            if (x > hi) x = hi;
            for (int q = 0; q < cnt; ++q) {
                const int d = cdst[p0 + q];
                const int r = d >> 24, pos = d & 0xffffff;
                T *dst = (r == rank) ? vbx : cl.map_shared_rank(vbx, r);
                dst[pos] = x;
            }
            if (chk) {
                for (int q = 0; q < cnt; ++q) u_prev[u0 + p0 + q] = uloc[p0 + q];
                const double xd = xrg[i] + (double)x;
                acc[2] += (double)cnt * xd * xd;
                acc[5] += cg64[i] * xd;
            }
        }
        cl.sync();
        // B: t = F^T (x + w) per factor column
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            const int itm = items[j];
            const int4 r = srec[itm >> 8];
            const int c = itm & 255, npad = (r.w >> 1) & 0x1ff;
            tb[r.z + c] = dot_padded2<T>(F + r.x + c * npad, vbx + r.y, vbw + r.y, npad);
        }
        __syncthreads();
        // C: projection, dual update, u to the owner
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int mt = meta[k];
            const int4 r = srec[mt >> 8];
            const int row = mt & 255;
            const int f = r.w >> 10, npad = (r.w >> 1) & 0x1ff, mode = r.w & 1;
            const T *Fr = F + r.x + row;
            const T *tt = tb + r.z;
            T y0 = 0, y1 = 0;
            int c = 0;
            for (; c + 1 < f; c += 2) {
                y0 += Fr[c * npad] * tt[c];
                y1 += Fr[(c + 1) * npad] * tt[c + 1];
            }
            if (c < f) y0 += Fr[c * npad] * tt[c];
            const int pos = r.y + row;
            const T x = vbx[pos];
            const T v = x + vbw[pos];
            const T xm = (mode ? (y0 + y1) : v - (y0 + y1)) + bt[k];
            const T res = x - xm;
            const T mu_new = mu[k] + rho * res;
            const T d_old = ds[k];
            ds[k] = xm;
            mu[k] = mu_new;
            vbw[pos] = mu_new * inv_rho;
            const int d = udst[k];
            const int ro = d >> 24, up = d & 0xffffff;
            T *ud = (ro == rank) ? uloc : cl.map_shared_rank(uloc, ro);
            ud[up] = rho * xm - mu_new;
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
        cl.sync();
        if (chk) {
            __shared__ double bred[32][6];
            block_sum6(acc, bred);
            if (threadIdx.x == 0) {
                double *dst = cl.map_shared_rank(red, 0);
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[rank * 6 + q] = acc[q];
            }
            cl.sync();
            if (rank == 0 && threadIdx.x == 0) {
                double s6[6] = {0, 0, 0, 0, 0, 0};
                for (int r = 0; r < P; ++r)
#pragma unroll
                    for (int q = 0; q < 6; ++q) s6[q] += red[r * 6 + q];
                const int since = ((it + 1) % check_every) == 0 ? check_every : ((it + 1) % check_every);
                apply_test(st, s6, rho_d, since);
                *stop = st->done;
            }
            cl.sync();
            const int halt = *cl.map_shared_rank(stop, 0);
            if (halt) break;
        }
    }
    // write back: slots' mu and x_s, the owner's u (the previous u was saved on the last tested iteration)
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        g.mu[k0 + k] = mu[k];
        g.ds[k0 + k] = ds[k];
    }
    for (int p = threadIdx.x; p < nu; p += blockDim.x) u_glob[u0 + p] = uloc[p];
    cl.sync();   // no CTA exits while others may still read its shared memory
    if (use_cond && rank == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, *stop ? 0u : 1u);
}

// ============================================================ warp engine
// Persistent engine for instances of at most 16 x 12 subsystems: a cluster of
// P CTAs, one warp per subsystem for the whole solve (the plan's warp map
// spreads the sizes over the CTAs), or two warps for a large one, each owning
// half of its rows; lane l owns the warp's rows r0 + l and r0 + l + 32.
// In FP32 a subsystem with n <= 32 keeps its factor F in registers (lane c:
// column c for t = F^T v; lane r: row r for y = F t), so both mat-vecs are
// chains of warp shuffles and FMAs; a larger one (n <= 64) reads F from shared
// memory.  In FP64 every factor is read from shared memory (two copies,
// column- and row-major), t = F^T v splits the rows over 2 or 4 lane groups
// when f <= 16 and y = F t the columns when the warp has at most 16 rows: a
// warp FP64 instruction occupies the FP64 pipe the same whatever its active
// lanes, so the count of them on the slowest warp sets the time.  The two
// warps of a split subsystem add their halves of t through shared memory
// behind a two-warp named barrier.  For one iteration:
//   x = clip((sum of u over the global's copies - c~) / (rho N), lb~, ub~)   (Eq. closed_1)
//   v = x + mu / rho;  t = F^T v;  y = F t
//   x_s = (v - y or y) + bbar~  (Eq. closed_2),  mu += rho (x - x_s) (Eq. ADMM-3)
//   u = rho x_s - mu stored into every replica of the global's u (each CTA
//   keeps one for each global it has copies of; other CTAs through
//   distributed shared memory, double-buffered by iteration parity)
// followed by one barrier (cluster-wide, or __syncthreads when P = 1).
constexpr int WE_WARPS = 12;
constexpr int WE_NREG = 32;   // factor rows held in registers (n <= 32)
constexpr int WE_FREG = 16;   // factor columns held in registers
constexpr int WE_DREG = 4;    // u destinations held in registers

__device__ __forceinline__ void we_barrier(cg::cluster_group &cl, int P) {
    if (P == 1) __syncthreads();
    else cl.sync();
}

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(32 * WE_WARPS, 1)
k_warp_engine(IterArgs<T> g, WarpLayout lay, const int *pr, T *u_glob, int n_iters, int check_every,
              DevStatus *st, double rho_d, cudaGraphConditionalHandle cond, int use_cond) {
    constexpr bool REG = sizeof(T) == 4;   // register-resident factors (FP32 only)
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int P = lay.P, P1 = P + 1;
    const int rank = (int)cl.block_rank();
    if (st->done) {
        if (use_cond && rank == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const int kb = pr[PR_K * P1 + rank];                                              // local slots
    const int fb0 = pr[PR_F * P1 + rank], nfb = pr[PR_F * P1 + rank + 1] - fb0;       // shared-memory factors
    const int db0 = pr[PR_J * P1 + rank], ndb = pr[PR_J * P1 + rank + 1] - db0;       // u destinations
    const int rb0 = pr[PR_V * P1 + rank], nrb = pr[PR_V * P1 + rank + 1] - rb0;       // replica segments
    T *ubuf[2] = {reinterpret_cast<T *>(sm + lay.off_useg),
                  reinterpret_cast<T *>(sm + lay.off_useg) + lay.useg_len};           // read t % 2, write the other
    int *dd = reinterpret_cast<int *>(sm + lay.off_dd);
    T *Fbig = reinterpret_cast<T *>(sm + lay.off_fbig);
    T *vbig = reinterpret_cast<T *>(sm + lay.off_vbig);    // 64 entries per warp
    T *tpart = reinterpret_cast<T *>(sm + lay.off_tpart);  // per warp pair: its two halves of t
    double *red = reinterpret_cast<double *>(sm + lay.off_red);
    int *stop = reinterpret_cast<int *>(sm + lay.off_red + 16 * 6 * sizeof(double));
    copy_in<T>(dd, g.wdd + db0, (size_t)ndb * sizeof(int));
    copy_in<T>(Fbig, g.F2 + fb0, (size_t)nfb * sizeof(T));
    for (int i = threadIdx.x; i < nrb; i += blockDim.x) {
        const int3 r = g.wrep[rb0 + i];
        for (int q = 0; q < r.z; ++q) ubuf[0][r.x + q] = u_glob[r.y + q];
    }
    if (threadIdx.x == 0) *stop = 0;
    __syncthreads();   // the factors copied in by the whole CTA are read per warp below
    const T rho = g.rho, inv_rho = g.inv_rho;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // ---- per-warp subsystem, its rows [r0, r0 + nr) and per-lane row state (registers)
    const int wm = g.wmap[rank * lay.warps + warp];
    const int s = wm >= 0 ? (wm >> 8) : lay.S;
    const int part = (wm >> 4) & 15, nparts = wm & 15;   // nparts 2: rows split with warp slot warp ^ 1
    const bool have = wm >= 0 && s < lay.S;
    int n = 0, f = 0, mode = 0, soff = 0, big = 0, npad = 0, r0 = 0, nr = 0;
    const T *Fs = nullptr;
    T *Frm = nullptr;
    T Fc[REG ? WE_NREG : 1], Fr[REG ? WE_FREG : 1];
#pragma unroll
    for (int r = 0; r < (REG ? WE_NREG : 1); ++r) Fc[r] = T(0);
#pragma unroll
    for (int c = 0; c < (REG ? WE_FREG : 1); ++c) Fr[c] = T(0);
    T bt[2] = {0, 0}, ds[2] = {0, 0}, mu[2] = {0, 0}, ct[2] = {0, 0}, lo[2] = {0, 0}, hi[2] = {0, 0};
    T rcp[2] = {0, 0};
    int rseg[2] = {0, 0}, dsp[2] = {0, 0}, qk[2] = {0, 0}, pk[2] = {0, 0};
    int ndr = 0;
    T *dptr[WE_DREG];
#pragma unroll
    for (int e = 0; e < WE_DREG; ++e) dptr[e] = nullptr;
    if (have) {
        const int4 h = g.sub[s], q = g.sub2[s];
        soff = h.x; n = h.y; f = h.z; mode = h.w;
        npad = q.y;
        const int hn = (n + 1) >> 1;
        r0 = (nparts == 2 && part) ? hn : 0;
        nr = nparts == 2 ? (part ? n - hn : hn) : n;
        big = REG ? (n > 32 || nparts == 2) : 1;
        if (!big) {
            if constexpr (REG) {
                const T *Fg = g.F + q.x;
#pragma unroll
                for (int r = 0; r < WE_NREG; ++r)
                    if (lane < f && r < n) Fc[r] = Fg[lane * npad + r];
#pragma unroll
                for (int c = 0; c < WE_FREG; ++c)
                    if (c < f && lane < n) Fr[c] = Fg[c * npad + lane];
            }
        } else {
            Fs = Fbig + (g.fbig[s] - fb0);                      // column-major, column stride npad
            Frm = Fbig + lay.fbig_len + (g.fbig[s] - fb0);      // row-major copy, row stride f
            for (int i = r0 * f + lane; i < (r0 + nr) * f; i += 32) {   // this warp's rows
                const int r = i / f, c = i - r * f;
                Frm[i] = Fs[c * npad + r];
            }
        }
        const int kl0 = g.klb[s];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int lr = lane + 32 * j, row = r0 + lr;
            if (lr < nr) {
                const int kg = soff + row;
                const int gi = g.gk[kg];
                bt[j] = g.bt[kg];
                ds[j] = g.ds[kg];
                mu[j] = g.mu[kg];
                ct[j] = g.ct[gi];
                lo[j] = g.lbt[gi];
                hi[j] = g.ubt[gi];
                const int sp = g.segp[kg];
                rcp[j] = g.recip[sp & 255];
                pk[j] = g.pk[kg];
                qk[j] = pk[j] - (sp >> 8);
                rseg[j] = g.wrseg[kb + kl0 + row];
                dsp[j] = g.wdsp[kb + kl0 + row];
            }
        }
        // first row: up to WE_DREG destinations resolved to pointers (buffer 0;
        // the parity offset is added per iteration)
        if (lane < nr) {
            const int d0 = dsp[0] >> 8, nd = dsp[0] & 255;
            ndr = nd < WE_DREG ? nd : WE_DREG;
#pragma unroll
            for (int e = 0; e < WE_DREG; ++e)
                if (e < ndr) {
                    const int d = g.wdd[db0 + d0 + e];
                    const int ro = d >> 24, up = d & 0xffffff;
                    dptr[e] = (ro == rank ? ubuf[0] : cl.map_shared_rank(ubuf[0], ro)) + up;
                }
        }
    }
    __syncthreads();
    if (P > 1) cl.sync();
    int par = 0;
    for (int it = 0; it < n_iters; ++it) {
        const bool chk = ((it + 1) % check_every) == 0 || it == n_iters - 1;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const T *useg = ubuf[par];
        const int nxt = (par ^ 1) * lay.useg_len;      // offset of the buffer written this iteration
        if (have) {
            T x[2] = {0, 0}, v[2] = {0, 0};
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int lr = lane + 32 * j, row = r0 + lr;
                if (lr < nr) {
                    const int base = rseg[j] >> 8, cnt = rseg[j] & 255;
                    T sum;
                    if constexpr (REG) {   // four chains for latency
                        T sg[4] = {0, 0, 0, 0};
#pragma unroll
                        for (int qq = 0; qq < 8; ++qq)
                            if (qq < cnt) sg[qq & 3] += useg[base + qq];
                        for (int qq = 8; qq < cnt; ++qq) sg[qq & 3] += useg[base + qq];
                        sum = (sg[0] + sg[1]) + (sg[2] + sg[3]);
                    } else {               // FP64: cnt - 1 adds, no padding adds on the FP64 pipe
                        sum = useg[base];
                        for (int qq = 1; qq < cnt; ++qq) sum += useg[base + qq];
                    }
                    T xv = (sum - ct[j]) * rcp[j];
                    if (xv < lo[j]) xv = lo[j];
                    if (xv > hi[j]) xv = hi[j];
                    x[j] = xv;
                    v[j] = xv + mu[j] * inv_rho;
                    if (chk) {   // FP64 data of the test read from global memory
                        g.u_prev_out[pk[j]] = useg[base + qk[j]];
                        const int gi = g.gk[soff + row];
                        const double xd = g.xr[gi] + (double)xv;
                        acc[2] += xd * xd;
                        if (qk[j] == 0) acc[5] += g.c64[gi] * xd;
                    }
                }
            }
            T t = 0, y[2] = {0, 0};
            if (!big) {
                if constexpr (REG) {
                    // t_c (lane c) = sum_r F[r][c] v_r, then y_r (lane r) = sum_c F[r][c] t_c;
                    // warp-uniform bounds: n shuffles for t and f for y
                    T t1 = 0;
#pragma unroll
                    for (int r = 0; r < WE_NREG; r += 2) {
                        if (r >= n) break;
                        t = fma_t(Fc[r], __shfl_sync(0xffffffffu, v[0], r), t);
                        t1 = fma_t(Fc[r + 1], __shfl_sync(0xffffffffu, v[0], r + 1), t1);
                    }
                    t += t1;
                    T y1 = 0;
#pragma unroll
                    for (int c = 0; c < WE_FREG; c += 2) {
                        if (c >= f) break;
                        y[0] = fma_t(Fr[c], __shfl_sync(0xffffffffu, t, c), y[0]);
                        y1 = fma_t(Fr[c + 1], __shfl_sync(0xffffffffu, t, c + 1), y1);
                    }
                    y[0] += y1;
                }
            } else {
                T *vb = vbig + warp * 64;   // indexed by subsystem row; this warp's rows only
                if (lane < nr) vb[r0 + lane] = v[0];
                if (lane + 32 < nr) vb[r0 + lane + 32] = v[1];
                __syncwarp();
                if (!REG && f <= 16) {
                    // FP64: G = 2 or 4 lane groups; group h sums rows h, h + G, ...
                    // of column c = lane % (32 / G), then the groups are added
                    const int lg = f <= 8 ? 3 : 4, G = 32 >> lg;
                    const int c = lane & ((1 << lg) - 1), h = lane >> lg;
                    T a0 = 0, a1 = 0;
                    if (c < f) {
                        const int re = r0 + nr;
                        int r = r0 + h;
                        for (; r + G < re; r += 2 * G) {
                            a0 = fma_t(Frm[r * f + c], vb[r], a0);
                            a1 = fma_t(Frm[(r + G) * f + c], vb[r + G], a1);
                        }
                        for (; r < re; r += G) a0 = fma_t(Frm[r * f + c], vb[r], a0);
                    }
                    t = a0 + a1;
                    for (int o = 1 << lg; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                } else if (lane < f) {
                    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
                    const int re = r0 + nr;
                    int r = r0;
                    for (; r + 3 < re; r += 4) {
                        a0 = fma_t(Frm[(r + 0) * f + lane], vb[r + 0], a0);
                        a1 = fma_t(Frm[(r + 1) * f + lane], vb[r + 1], a1);
                        a2 = fma_t(Frm[(r + 2) * f + lane], vb[r + 2], a2);
                        a3 = fma_t(Frm[(r + 3) * f + lane], vb[r + 3], a3);
                    }
                    for (; r < re; ++r) a0 = fma_t(Frm[r * f + lane], vb[r], a0);
                    t = (a0 + a1) + (a2 + a3);
                }
                __syncwarp();
                if (nparts == 2) {
                    // the pair's halves of t, added in the same order by both warps
                    T *tp = tpart + (warp >> 1) * 64;
                    if (lane < f) tp[part * 32 + lane] = t;
                    asm volatile("bar.sync %0, 64;" ::"r"(1 + (warp >> 1)) : "memory");
                    if (lane < f) t = tp[lane] + tp[32 + lane];
                }
                if (!REG && nr <= 16) {
                    // FP64: G = 2 or 4 lane groups; group h sums columns h, h + G, ...
                    // for row r0 + lane % (32 / G), then the groups are added
                    const int lg = nr <= 8 ? 3 : 4, G = 32 >> lg;
                    const int rl = lane & ((1 << lg) - 1), h = lane >> lg;
                    const int rr = r0 + rl < npad ? r0 + rl : 0;
                    const int nc = (f + G - 1) / G;
                    T b0 = 0;
                    for (int i = 0; i < nc; ++i) {
                        const int c = i * G + h;
                        const T tc = __shfl_sync(0xffffffffu, t, c < f ? c : 0);
                        if (c < f) b0 = fma_t(Fs[c * npad + rr], tc, b0);
                    }
                    for (int o = 1 << lg; o < 32; o <<= 1) b0 += __shfl_xor_sync(0xffffffffu, b0, o);
                    y[0] = b0;
                } else {
                    const bool two = nr > 32;   // a second row per lane (only when r0 = 0)
                    const int r1 = r0 + lane < npad ? r0 + lane : 0;     // stays inside the column
                    const int r2 = lane + 32 < npad ? lane + 32 : lane;
                    T b0 = 0, b1 = 0, e0 = 0, e1 = 0;
                    int c = 0;
                    for (; c + 1 < f; c += 2) {
                        const T ta = __shfl_sync(0xffffffffu, t, c);
                        const T tb2 = __shfl_sync(0xffffffffu, t, c + 1);
                        b0 = fma_t(Fs[c * npad + r1], ta, b0);
                        b1 = fma_t(Fs[(c + 1) * npad + r1], tb2, b1);
                        if (two) {
                            e0 = fma_t(Fs[c * npad + r2], ta, e0);
                            e1 = fma_t(Fs[(c + 1) * npad + r2], tb2, e1);
                        }
                    }
                    if (c < f) {
                        const T ta = __shfl_sync(0xffffffffu, t, c);
                        b0 = fma_t(Fs[c * npad + r1], ta, b0);
                        if (two) e0 = fma_t(Fs[c * npad + r2], ta, e0);
                    }
                    y[0] = b0 + b1;
                    y[1] = e0 + e1;   // used only when lane + 32 < n
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int lr = lane + 32 * j, row = r0 + lr;
                if (lr < nr) {
                    const T xm = (mode ? y[j] : v[j] - y[j]) + bt[j];
                    const T res = x[j] - xm;
                    const T mu_new = mu[j] + rho * res;
                    const T d_old = ds[j];
                    ds[j] = xm;
                    mu[j] = mu_new;
                    const T un = rho * xm - mu_new;
                    const int d0 = dsp[j] >> 8, nd = dsp[j] & 255;
                    int e0 = 0;
                    if (j == 0) {
#pragma unroll
                        for (int e = 0; e < WE_DREG; ++e)
                            if (e < ndr) dptr[e][nxt] = un;
                        e0 = ndr;
                    }
                    for (int e = e0; e < nd; ++e) {
                        const int d = dd[d0 + e];
                        const int ro = d >> 24, up = d & 0xffffff;
                        T *ud = (ro == rank) ? ubuf[par ^ 1] : cl.map_shared_rank(ubuf[par ^ 1], ro);
                        ud[up] = un;
                    }
                    if (chk) {
                        const int kg = soff + row;
                        const double xsd = g.xr[g.gk[kg]] + (double)xm;
                        const double dd2 = (double)xm - (double)d_old;
                        acc[0] += (double)res * (double)res;
                        acc[1] += dd2 * dd2;
                        acc[3] += xsd * xsd;
                        const double lamd = g.lamr[kg] + (double)mu_new;
                        acc[4] += lamd * lamd;
                    }
                }
            }
        }
        par ^= 1;
        we_barrier(cl, P);
        if (chk) {
            __shared__ double bred[32][6];
            block_sum6(acc, bred);
            if (threadIdx.x == 0) {
                double *dst = P > 1 ? cl.map_shared_rank(red, 0) : red;
#pragma unroll
                for (int q = 0; q < 6; ++q) dst[rank * 6 + q] = acc[q];
            }
            we_barrier(cl, P);
            if (rank == 0 && threadIdx.x == 0) {
                double s6[6] = {0, 0, 0, 0, 0, 0};
                for (int r = 0; r < P; ++r)
#pragma unroll
                    for (int q = 0; q < 6; ++q) s6[q] += red[r * 6 + q];
                const int since = ((it + 1) % check_every) == 0 ? check_every : ((it + 1) % check_every);
                apply_test(st, s6, rho_d, since);
                *stop = st->done;
            }
            we_barrier(cl, P);
            if (*(P > 1 ? cl.map_shared_rank(stop, 0) : stop)) break;
        }
    }
    // write back the slots' mu, x_s and current u (each copy by its slot)
    if (have) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int lr = lane + 32 * j, row = r0 + lr;
            if (lr < nr) {
                g.mu[soff + row] = mu[j];
                g.ds[soff + row] = ds[j];
                u_glob[pk[j]] = ubuf[par][(rseg[j] >> 8) + qk[j]];
            }
        }
    }
    if (P > 1) cl.sync();
    if (use_cond && rank == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, *stop ? 0u : 1u);
}

template <typename T>
int prepare_warp_engine(unsigned bytes) {
    if (cudaFuncSetAttribute(k_warp_engine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return -1;
    if (cudaFuncSetAttribute(k_warp_engine<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    return 0;
}

static void fill_cluster_cfg(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *attr, int P, int threads,
                             unsigned bytes, cudaStream_t s) {
    memset(cfg, 0, sizeof(*cfg));
    cfg->gridDim = dim3(P, 1, 1);
    cfg->blockDim = dim3(threads, 1, 1);
    cfg->dynamicSmemBytes = bytes;
    cfg->stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg->attrs = attr;
    cfg->numAttrs = 1;
}

template <typename T>
int launch_warp_engine(const IterArgs<T> &g, const WarpLayout &lay, const int *pr, T *u_glob, int n_iters,
                       int check_every, DevStatus *st, double rho, cudaGraphConditionalHandle cond, int use_cond,
                       cudaStream_t s) {
    if (lay.warps < 1 || lay.warps > WE_WARPS) return -1;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    fill_cluster_cfg(&cfg, attr, lay.P, 32 * lay.warps, lay.bytes, s);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_warp_engine<T>, g, lay, pr, u_glob, n_iters, check_every, st, rho,
                                       cond, use_cond);
    return e == cudaSuccess ? 0 : -1;
}

template <typename T>
int warp_engine_occupancy(const WarpLayout &lay) {
    if (lay.warps < 1 || lay.warps > WE_WARPS) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    fill_cluster_cfg(&cfg, attr, lay.P, 32 * lay.warps, lay.bytes, 0);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_warp_engine<T>, &cfg) != cudaSuccess) return 0;
    return n;
}

template int prepare_warp_engine<float>(unsigned);
template int prepare_warp_engine<double>(unsigned);
template int launch_warp_engine<float>(const IterArgs<float> &, const WarpLayout &, const int *, float *, int, int,
                                       DevStatus *, double, cudaGraphConditionalHandle, int, cudaStream_t);
template int launch_warp_engine<double>(const IterArgs<double> &, const WarpLayout &, const int *, double *, int,
                                        int, DevStatus *, double, cudaGraphConditionalHandle, int, cudaStream_t);
template int warp_engine_occupancy<float>(const WarpLayout &);
template int warp_engine_occupancy<double>(const WarpLayout &);

// ============================================================ small kernels
// u[pk[k]] = rho * ds[k] - mu[k]
template <typename T>
__global__ void k_make_u(int L, const int *pk, const T *ds, const T *mu, T rho, T *u,
                         const DevStatus *st) {
    if (st && st->done) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x)
        u[pk[k]] = rho * ds[k] - mu[k];
}

// Global x_i = x_ref_i + clip((sum_seg u - c~_i) / (rho N_i), lb~, ub~) and
// per-block partial of c^T x.
template <typename T>
__global__ void k_global_x(int G, const int2 *gseg, const T *u, const T *ct, const T *lbt,
                           const T *ubt, const double *xr, const double *c64, T rho,
                           double *x, double *obj_part, const DevStatus *st) {
    __shared__ double red[256];
    if (st && st->done) return;
    double o = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        const int2 sg = gseg[i];
        T sigma = 0;
        for (int q = 0; q < sg.y; ++q) sigma += u[sg.x + q];
        T xh = (sigma - ct[i]) / (rho * (T)sg.y);
        if (xh < lbt[i]) xh = lbt[i];
        if (xh > ubt[i]) xh = ubt[i];
        const double xv = xr[i] + (double)xh;
        x[i] = xv;
        o += c64[i] * xv;
    }
    red[threadIdx.x] = o;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) obj_part[blockIdx.x] = red[0];
}

// Start point of Sec. V-A: every copy of global i at x0_i, lambda = 0.
template <typename T>
__global__ void k_init_state(int L, const int *gk, const double *x0, T *ds, T *mu) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
        ds[k] = (T)x0[gk[k]];
        mu[k] = (T)0;
    }
}

template <typename A, typename B>
__global__ void k_cast(long long n, const A *src, B *dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}

__global__ void k_copy_if_running(long long n, const double *src, double *dst, const DevStatus *st) {
    if (st && st->done) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// x_s = x_ref[g] + d, lambda = lambda_ref + mu in FP64 (leaves the shifted frame)
template <typename T>
__global__ void k_unshift(int L, const int *gk, const double *xr, const double *lamr, const T *ds,
                          const T *mu, double *ds64, double *mu64) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
        ds64[k] = xr[gk[k]] + (double)ds[k];
        mu64[k] = lamr[k] + (double)mu[k];
    }
}

// entering the shifted frame: d = x_s - x_ref[g] (rounded once), lambda_ref = lambda, mu = 0
__global__ void k_enter_shift(int L, const int *gk, const double *xr, const double *ds64,
                              const double *mu64, float *ds32, float *mu32, double *lamr) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
        ds32[k] = (float)(ds64[k] - xr[gk[k]]);
        mu32[k] = 0.0f;
        lamr[k] = mu64[k];
    }
}

// ---- re-centring (OPF_PREC_MIXED): all FP64
// slot k: d_new = d + x_ref_old[g] - x_ref_new[g];  lambda_ref += mu;  mu = 0
template <typename T>
__global__ void k_recenter_slots(int L, const int *gk, const double *xr_old, const double *xr_new,
                                 T *ds, T *mu, double *lamr, const DevStatus *st) {
    if (st && st->done) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
        const int g = gk[k];
        ds[k] = (T)((double)ds[k] + xr_old[g] - xr_new[g]);
        lamr[k] += (double)mu[k];
        mu[k] = (T)0;
    }
}

// per global: c~ = c + sum over its slots of lambda_ref, bounds - x_ref
template <typename T>
__global__ void k_recenter_globals(int G, const int2 *gseg, const int *uslot, const double *lamr,
                                   const double *c64, const double *lb, const double *ub,
                                   const double *xr, T *ct, T *lbt, T *ubt, const DevStatus *st) {
    if (st && st->done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        const int2 sg = gseg[i];
        double s = c64[i];
        for (int q = 0; q < sg.y; ++q) s += lamr[uslot[sg.x + q]];
        ct[i] = (T)s;
        lbt[i] = (T)(lb[i] - xr[i]);
        ubt[i] = (T)(ub[i] - xr[i]);
    }
}

// per subsystem (one warp): bbar~ = M (x_ref[g] + lambda_ref / rho) + bbar - x_ref[g]
template <typename T>
__global__ void __launch_bounds__(128) k_recenter_bbar(int S, const int4 *sub, const int4 *sub2,
                                                       const double *F, const int *gk, const double *xr,
                                                       const double *lamr, const double *bbar,
                                                       double rho, T *bt, const DevStatus *st) {
    __shared__ double buf[4][2][OPF_MAX_NS];
    if (st && st->done) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * 4 + w;
    if (s >= S) return;
    const int4 h = sub[s], q = sub2[s];
    const int so = h.x, n = h.y, f = h.z, mode = h.w, npad = q.y;
    const double *Fs = F + q.x;
    double *v = buf[w][0], *t = buf[w][1];
    for (int r = lane; r < n; r += 32) v[r] = xr[gk[so + r]] + lamr[so + r] / rho;
    __syncwarp();
    for (int c = lane; c < f; c += 32) {
        double acc = 0.0;
        for (int r = 0; r < n; ++r) acc += Fs[(long long)c * npad + r] * v[r];
        t[c] = acc;
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
        double y = 0.0;
        for (int c = 0; c < f; ++c) y += Fs[(long long)c * npad + r] * t[c];
        const double mv = mode ? y : v[r] - y;
        bt[so + r] = (T)(mv + bbar[so + r] - xr[gk[so + r]]);
    }
}

// ============================================================ launchers
static inline int nblocks(long long n, int t) {
    long long b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

int launch_precompute(const PreArgs &a, cudaStream_t st) {
    const int big = a.sh_m > a.sh_n ? a.sh_m : a.sh_n;
    const size_t shm = sizeof(double) * ((size_t)a.sh_m * a.sh_n + (size_t)a.sh_n * a.sh_n +
                                         33 * (size_t)big + (size_t)a.sh_m + 2);
    if (cudaFuncSetAttribute(k_precompute, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
        return -1;
    k_precompute<<<a.S, 32, shm, st>>>(a);
    return 0;
}

void launch_pack_factors(int S, const int4 *sub, const int4 *sub2, const long long *cap_off,
                         const double *src, double *dst64, float *dst32, cudaStream_t st) {
    k_pack_factors<<<S, 128, 0, st>>>(S, sub, sub2, cap_off, src, dst64, dst32);
}

template <typename T>
void launch_iterate(const IterArgs<T> &a, const T *u_in, T *u_out, double *partials,
                    const DevStatus *st, bool check, int n_tiles, int block, int xcap, int vcap,
                    int tcap, cudaStream_t s) {
    const size_t shm = ((size_t)xcap + vcap + tcap) * sizeof(T);
    if (check) k_tile_iter<T, true><<<n_tiles, block, shm, s>>>(a, u_in, u_out, partials, st, xcap, vcap);
    else k_tile_iter<T, false><<<n_tiles, block, shm, s>>>(a, u_in, u_out, partials, st, xcap, vcap);
}

void launch_check(const double *partials, int nblk, DevStatus *st, double rho, int add,
                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
    k_check<<<1, 256, 0, s>>>(partials, nblk, st, rho, add, cond, use_cond);
}

void launch_copy_if_running(long long n, const double *src, double *dst, const DevStatus *st,
                            cudaStream_t s) {
    k_copy_if_running<<<nblocks(n, 256), 256, 0, s>>>(n, src, dst, st);
}

void launch_add_iters(DevStatus *st, long long n, cudaStream_t s) { k_add_iters<<<1, 32, 0, s>>>(st, n); }

void launch_enter_shift(int L, const int *gk, const double *xr, const double *ds64,
                        const double *mu64, float *ds32, float *mu32, double *lamr, cudaStream_t s) {
    k_enter_shift<<<nblocks(L, 256), 256, 0, s>>>(L, gk, xr, ds64, mu64, ds32, mu32, lamr);
}

template <typename T>
int prepare_cluster_engine(unsigned bytes, int P) {
    if (cudaFuncSetAttribute(k_cluster_engine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return -1;
    if (P > 8 && cudaFuncSetAttribute(k_cluster_engine<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return -1;
    return 0;
}

template <typename T>
int launch_cluster_engine(const IterArgs<T> &g, const ClusterLayout &lay, const int *pr, T *u_glob,
                          int n_iters, int check_every, DevStatus *st, double rho,
                          cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(lay.P, 1, 1);
    cfg.blockDim = dim3(lay.threads, 1, 1);
    cfg.dynamicSmemBytes = lay.bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = lay.P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster_engine<T>, g, lay, pr, u_glob, n_iters, check_every, st,
                                       rho, cond, use_cond);
    return e == cudaSuccess ? 0 : -1;
}

// Largest cluster of P CTAs with `bytes` of shared memory each that can be
// resident (0 if none).
template <typename T>
int cluster_occupancy(const ClusterLayout &lay) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(lay.P, 1, 1);
    cfg.blockDim = dim3(lay.threads, 1, 1);
    cfg.dynamicSmemBytes = lay.bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = lay.P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_cluster_engine<T>, &cfg) != cudaSuccess) return 0;
    return n;
}

template <typename T>
void launch_make_u(int L, const int *pk, const T *ds, const T *mu, T rho, T *u, const DevStatus *st,
                   cudaStream_t s) {
    k_make_u<T><<<nblocks(L, 256), 256, 0, s>>>(L, pk, ds, mu, rho, u, st);
}

template <typename T>
int launch_global_x(int G, const int2 *gseg, const T *u, const T *ct, const T *lbt, const T *ubt,
                    const double *xr, const double *c64, T rho, double *x, double *obj_part,
                    const DevStatus *st, cudaStream_t s) {
    const int b = nblocks(G, 256);
    k_global_x<T><<<b, 256, 0, s>>>(G, gseg, u, ct, lbt, ubt, xr, c64, rho, x, obj_part, st);
    return b;
}

template <typename T>
void launch_unshift(int L, const int *gk, const double *xr, const double *lamr, const T *ds,
                    const T *mu, double *ds64, double *mu64, cudaStream_t s) {
    k_unshift<T><<<nblocks(L, 256), 256, 0, s>>>(L, gk, xr, lamr, ds, mu, ds64, mu64);
}

template <typename T>
void launch_init_state(int L, const int *gk, const double *x0, T *ds, T *mu, cudaStream_t s) {
    k_init_state<T><<<nblocks(L, 256), 256, 0, s>>>(L, gk, x0, ds, mu);
}

template <typename A, typename B>
void launch_cast(long long n, const A *src, B *dst, cudaStream_t s) {
    k_cast<A, B><<<nblocks(n, 256), 256, 0, s>>>(n, src, dst);
}

template <typename T>
void launch_recenter(int L, int G, int S, const int *gk, const double *xr_old, const double *xr_new,
                     T *ds, T *mu, double *lamr, const int2 *gseg, const int *uslot,
                     const double *c64, const double *lb, const double *ub, T *ct, T *lbt, T *ubt,
                     const int4 *sub, const int4 *sub2, const double *F64, const double *bbar,
                     double rho, T *bt, const DevStatus *st, cudaStream_t s) {
    k_recenter_slots<T><<<nblocks(L, 256), 256, 0, s>>>(L, gk, xr_old, xr_new, ds, mu, lamr, st);
    k_recenter_globals<T><<<nblocks(G, 256), 256, 0, s>>>(G, gseg, uslot, lamr, c64, lb, ub, xr_new,
                                                          ct, lbt, ubt, st);
    k_recenter_bbar<T><<<(S + 3) / 4, 128, 0, s>>>(S, sub, sub2, F64, gk, xr_new, lamr, bbar, rho, bt, st);
}

#define OPF_INST(T)                                                                                   \
    template void launch_iterate<T>(const IterArgs<T> &, const T *, T *, double *, const DevStatus *, \
                                    bool, int, int, int, int, int, cudaStream_t);                     \
    template int prepare_cluster_engine<T>(unsigned, int);                                            \
    template int launch_cluster_engine<T>(const IterArgs<T> &, const ClusterLayout &, const int *, T *,\
                                          int, int, DevStatus *, double, cudaGraphConditionalHandle,  \
                                          int, cudaStream_t);                                         \
    template int cluster_occupancy<T>(const ClusterLayout &);                                         \
    template void launch_make_u<T>(int, const int *, const T *, const T *, T, T *, const DevStatus *, \
                                   cudaStream_t);                                                     \
    template int launch_global_x<T>(int, const int2 *, const T *, const T *, const T *, const T *,    \
                                    const double *, const double *, T, double *, double *,            \
                                    const DevStatus *, cudaStream_t);                                 \
    template void launch_init_state<T>(int, const int *, const double *, T *, T *, cudaStream_t);     \
    template void launch_unshift<T>(int, const int *, const double *, const double *, const T *,      \
                                    const T *, double *, double *, cudaStream_t);                     \
    template void launch_recenter<T>(int, int, int, const int *, const double *, const double *, T *, \
                                     T *, double *, const int2 *, const int *, const double *,        \
                                     const double *, const double *, T *, T *, T *, const int4 *,     \
                                     const int4 *, const double *, const double *, double, T *,       \
                                     const DevStatus *, cudaStream_t);
OPF_INST(double)
OPF_INST(float)
template void launch_cast<double, float>(long long, const double *, float *, cudaStream_t);
template void launch_cast<float, double>(long long, const float *, double *, cudaStream_t);

}  // namespace opf
