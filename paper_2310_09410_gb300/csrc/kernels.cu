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
//  k_iterate      one ADMM iteration of Algorithm 1 over all subsystems:
//                 global update (Eq. closed_1) recomputed per slot from the
//                 slot's segment of u = rho x_s - lambda of the previous
//                 iteration, local update (Eq. closed_2) x_s = M_s v + bbar_s
//                 with v = x_g + lambda/rho, dual update (Eq. ADMM-3), and on
//                 tested iterations the Sec. III-C sums in FP64.
//  k_cta_engine   the same iteration run by one CTA for many iterations with
//                 the whole instance resident in shared memory.
//
// Every quantity may be shifted by an FP64 reference point (x_ref per global,
// lambda_ref per slot): the kernels iterate on d = x_s - x_ref[g] and
// mu = lambda - lambda_ref with shifted data c~ = c + sum lambda_ref,
// bounds - x_ref and bbar~ = M (x_ref[g] + lambda_ref/rho) + bbar - x_ref[g].
// This is the same algorithm after a change of variables; with a zero
// reference it is plain ADMM.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "opf_internal.h"

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

__global__ void __launch_bounds__(128) k_precompute(PreArgs a) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.S) return;
    const int s = warp;
    const int m = a.sm[s], n = a.sn[s];
    const int T = (n + 31) >> 5;   // entries per lane (n <= 256 -> T <= 8)
    double *Aw = a.W + a.aoff[s];
    double *bw = a.Bw + a.boff[s];
    double bmax = 0.0;
    for (int j = lane; j < m; j += 32) bmax = fmax(bmax, fabs(bw[j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    int r = 0, bad = 0;
    for (int j = 0; j < m; ++j) {
        double v[RMAX];
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
            int c = lane + 32 * t;
            v[t] = (t < T && c < n) ? Aw[(long long)j * n + c] : 0.0;
        }
        double bj = bw[j];
        double n0 = 0.0;
#pragma unroll
        for (int t = 0; t < RMAX; ++t) n0 += v[t] * v[t];
        n0 = sqrt(warp_sum(n0));
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < r; ++k) {
                const double *q = Aw + (long long)k * n;
                double d = 0.0;
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    int c = lane + 32 * t;
                    if (t < T && c < n) d += q[c] * v[t];
                }
                d = warp_sum(d);
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    int c = lane + 32 * t;
                    if (t < T && c < n) v[t] -= d * q[c];
                }
                bj -= d * bw[k];
            }
        }
        double nr = 0.0;
#pragma unroll
        for (int t = 0; t < RMAX; ++t) nr += v[t] * v[t];
        nr = sqrt(warp_sum(nr));
        __syncwarp();
        if (n0 > 0.0 && nr > 1e-10 * n0) {
            double inv = 1.0 / nr;
#pragma unroll
            for (int t = 0; t < RMAX; ++t) {
                int c = lane + 32 * t;
                if (t < T && c < n) Aw[(long long)r * n + c] = v[t] * inv;
            }
            __syncwarp();
            if (lane == 0) bw[r] = bj * inv;
            __syncwarp();
            ++r;
        } else if (fabs(bj) > 1e-9 * (1.0 + bmax)) {
            bad = 1;
        }
    }
    __syncwarp();
    // bbar = sum_k beta_k q_k
    const int so = a.soff[s];
    for (int c = lane; c < n; c += 32) {
        double acc = 0.0;
        for (int k = 0; k < r; ++k) acc += bw[k] * Aw[(long long)k * n + c];
        a.bbar[so + c] = acc;
    }
    double *F = a.F + a.foff[s];
    if (r <= n - r) {
        // mode 0: F = Q^T, column k of F = row k of Q
        for (int k = 0; k < r; ++k)
            for (int c = lane; c < n; c += 32) F[(long long)k * n + c] = Aw[(long long)k * n + c];
        if (lane == 0) { a.sf[s] = r; a.smode[s] = 0; }
    } else {
        // mode 1: orthonormal basis of null(A_s) from pivoted Gram-Schmidt on
        // the columns of P = I - Q^T Q (column-major n x n in scratch)
        double *P = a.P + a.poff[s];
        for (int col = 0; col < n; ++col) {
            for (int c = lane; c < n; c += 32) {
                double acc = (c == col) ? 1.0 : 0.0;
                for (int k = 0; k < r; ++k) acc -= Aw[(long long)k * n + col] * Aw[(long long)k * n + c];
                P[(long long)col * n + c] = acc;
            }
        }
        __syncwarp();
        const int nf = n - r;
        for (int t = 0; t < nf; ++t) {
            // pivot: column of largest remaining norm
            double best = -1.0;
            int bc = 0;
            for (int col = 0; col < n; ++col) {
                double nn = 0.0;
                for (int c = lane; c < n; c += 32) { double x = P[(long long)col * n + c]; nn += x * x; }
                nn = warp_sum(nn);
                if (nn > best) { best = nn; bc = col; }
            }
            double v[RMAX];
#pragma unroll
            for (int q = 0; q < RMAX; ++q) {
                int c = lane + 32 * q;
                v[q] = (q < T && c < n) ? P[(long long)bc * n + c] : 0.0;
            }
            // re-orthogonalise against the null vectors found so far and Q
            for (int pass = 0; pass < 2; ++pass) {
                for (int k = 0; k < t; ++k) {
                    const double *q = F + (long long)k * n;
                    double d = 0.0;
#pragma unroll
                    for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) d += q[c] * v[qq]; }
                    d = warp_sum(d);
#pragma unroll
                    for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) v[qq] -= d * q[c]; }
                }
                for (int k = 0; k < r; ++k) {
                    const double *q = Aw + (long long)k * n;
                    double d = 0.0;
#pragma unroll
                    for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) d += q[c] * v[qq]; }
                    d = warp_sum(d);
#pragma unroll
                    for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) v[qq] -= d * q[c]; }
                }
            }
            double nn = 0.0;
#pragma unroll
            for (int qq = 0; qq < RMAX; ++qq) nn += v[qq] * v[qq];
            nn = sqrt(warp_sum(nn));
            double inv = nn > 0.0 ? 1.0 / nn : 0.0;
#pragma unroll
            for (int qq = 0; qq < RMAX; ++qq) {
                int c = lane + 32 * qq;
                if (qq < T && c < n) { v[qq] *= inv; F[(long long)t * n + c] = v[qq]; }
            }
            __syncwarp();
            // remove the new direction from every column of P
            for (int col = 0; col < n; ++col) {
                double d = 0.0;
#pragma unroll
                for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) d += v[qq] * P[(long long)col * n + c]; }
                d = warp_sum(d);
#pragma unroll
                for (int qq = 0; qq < RMAX; ++qq) { int c = lane + 32 * qq; if (qq < T && c < n) P[(long long)col * n + c] -= d * v[qq]; }
            }
            __syncwarp();
        }
        if (lane == 0) { a.sf[s] = nf; a.smode[s] = 1; }
    }
    if (lane == 0) a.status[s] = bad;
}

// ============================================================ iteration
// One warp task: up to 32/W subsystems, W lanes each, R rows per lane.
// sv: per-warp shared scratch of 2 * vstride T values.
template <typename T, bool CHECK, bool SMEM>
__device__ __forceinline__ void run_task(const IterArgs<T> &a, int task, int lane,
                                         const T *__restrict__ u_in, T *__restrict__ u_out,
                                         T *sv, int vstride, double acc[6]) {
    const int4 tk = ld<SMEM>(a.tasks + task);
    const int W = tk.z, R = tk.w;
    const int grp = lane / W, gl = lane - grp * W;
    const bool act = grp < tk.y;
    const int s = tk.x + (act ? grp : 0);
    const int n = act ? ld<SMEM>(a.sn + s) : 0;
    const int f = act ? ld<SMEM>(a.sf + s) : 0;
    const int mode = act ? ld<SMEM>(a.smode + s) : 0;
    const int so = act ? ld<SMEM>(a.soff + s) : 0;
    const long long fo = act ? ld<SMEM>(a.sfoff + s) : 0;
    T *vb = sv + grp * W * R;
    T *tb = sv + vstride + grp * W * R;
    T v[RMAX], xg[RMAX];
    // global update of each row's global (Eq. closed_1), then v = x_g + mu / rho
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        const int r = gl + W * j;
        if (j < R && r < n) {
            const int k = so + r;
            const int2 sg = ld<SMEM>(a.seg + k);
            T sigma = 0;
            for (int q = 0; q < sg.y; ++q) sigma += u_in[sg.x + q];
            const int g = ld<SMEM>(a.gk + k);
            T xh = (sigma - ld<SMEM>(a.ct + g)) / (a.rho * (T)sg.y);
            const T lo = ld<SMEM>(a.lbt + g), hi = ld<SMEM>(a.ubt + g);
            if (xh < lo) xh = lo;
            if (xh > hi) xh = hi;
            xg[j] = xh;
            v[j] = xh + a.mu[k] * a.inv_rho;
            vb[r] = v[j];
        }
    }
    __syncwarp();
    // t = F^T v  (column c per lane)
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        const int c = gl + W * j;
        if (j < R && c < f) {
            const T *Fc = a.F + fo + (long long)c * n;
            T t = 0;
            for (int r = 0; r < n; ++r) t += ld<SMEM>(Fc + r) * vb[r];
            tb[c] = t;
        }
    }
    __syncwarp();
    // y = F t ;  x_s = M v + bbar ;  lambda += rho (x_g - x_s) ; u = rho x_s - lambda
#pragma unroll
    for (int j = 0; j < RMAX; ++j) {
        const int r = gl + W * j;
        if (j < R && r < n) {
            const int k = so + r;
            T y = 0;
            const T *Fr = a.F + fo + r;
            for (int c = 0; c < f; ++c) y += ld<SMEM>(Fr + (long long)c * n) * tb[c];
            const T xm = (mode ? y : v[j] - y) + ld<SMEM>(a.bt + k);
            const T res = xg[j] - xm;
            const T mu_old = a.mu[k];
            const T mu_new = mu_old + a.rho * res;
            const T d_old = a.ds[k];
            a.mu[k] = mu_new;
            a.ds[k] = xm;
            const int pos = ld<SMEM>(a.pk + k);
            u_out[pos] = a.rho * xm - mu_new;
            if constexpr (CHECK) {
                const int g = ld<SMEM>(a.gk + k);
                const double xr = a.xr[g];
                const double xgd = xr + (double)xg[j];
                const double xsd = xr + (double)xm;
                const double dd = (double)xm - (double)d_old;
                acc[0] += (double)res * (double)res;
                acc[1] += dd * dd;
                acc[2] += xgd * xgd;
                acc[3] += xsd * xsd;
                const double lamd = a.lamr[k] + (double)mu_new;
                acc[4] += lamd * lamd;
                const int2 sg = ld<SMEM>(a.seg + k);
                if (pos == sg.x) acc[5] += a.c64[g] * xgd;
            }
        }
    }
    __syncwarp();
}

template <typename T, bool CHECK>
__global__ void __launch_bounds__(256) k_iterate(IterArgs<T> a, const T *__restrict__ u_in,
                                                 T *__restrict__ u_out, int vstride,
                                                 double *partials, const DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (st->done) return;
    T *sv = reinterpret_cast<T *>(smem_raw) + (threadIdx.x >> 5) * 2 * vstride;
    const int task = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (task < a.n_tasks) run_task<T, CHECK, false>(a, task, lane, u_in, u_out, sv, vstride, acc);
    if constexpr (CHECK) {
        __shared__ double red[8][6];
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
        const int w = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 6; ++q) red[w][q] = acc[q];
        __syncthreads();
        if (threadIdx.x < 6) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q][threadIdx.x];
            partials[blockIdx.x * 6 + threadIdx.x] = t;
        }
    }
}

// Stopping test of Sec. III-C (plus the absolute gate on pres).
__device__ void apply_test(DevStatus *st, const double s[6], double rho, long long add_iters) {
    const double pres = sqrt(s[0]);
    const double dres = rho * sqrt(s[1]);
    const double eprim = fmax(sqrt(s[2]), sqrt(s[3]));
    const double edual = sqrt(s[4]);
    st->iter += add_iters;
    st->pres = pres;
    st->dres = dres;
    st->eprim = eprim;
    st->edual = edual;
    st->obj = s[5];
    bool finite = true;
    for (int q = 0; q < 6; ++q) finite = finite && isfinite(s[q]);
    st->numeric = finite ? 0 : 1;
    st->converged = (finite && pres <= st->eps_rel * eprim && dres <= st->eps_rel * edual &&
                     pres <= st->eps_abs_pres) ? 1 : 0;
    if (st->converged || st->numeric || st->iter >= st->max_iter) st->done = 1;
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

// ============================================================ CTA engine
// Whole instance in shared memory; one CTA runs up to n_iters iterations,
// testing every check_every.  Layout offsets in bytes inside dynamic smem.

template <typename T>
__device__ void copy_in(void *dst, const void *src, size_t bytes) {
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    const size_t n4 = bytes / 16;
    for (size_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
    const unsigned char *sb = reinterpret_cast<const unsigned char *>(src);
    unsigned char *db = reinterpret_cast<unsigned char *>(dst);
    for (size_t i = n4 * 16 + threadIdx.x; i < bytes; i += blockDim.x) db[i] = sb[i];
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_cta_engine(IterArgs<T> g, CtaLayout lay, T *u_glob,
                                                        int n_iters, int check_every, DevStatus *st,
                                                        double rho_d, cudaGraphConditionalHandle cond,
                                                        int use_cond) {
    extern __shared__ __align__(16) unsigned char sm[];
    if (st->done) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    // stage the instance into shared memory (16-byte aligned regions)
    copy_in<T>(sm + lay.off_F, g.F, lay.nF * sizeof(T));
    copy_in<T>(sm + lay.off_bt, g.bt, (size_t)lay.L * sizeof(T));
    copy_in<T>(sm + lay.off_mu, g.mu, (size_t)lay.L * sizeof(T));
    copy_in<T>(sm + lay.off_ds, g.ds, (size_t)lay.L * sizeof(T));
    copy_in<T>(sm + lay.off_u0, u_glob, (size_t)lay.L * sizeof(T));
    copy_in<T>(sm + lay.off_ct, g.ct, (size_t)lay.G * sizeof(T));
    copy_in<T>(sm + lay.off_lbt, g.lbt, (size_t)lay.G * sizeof(T));
    copy_in<T>(sm + lay.off_ubt, g.ubt, (size_t)lay.G * sizeof(T));
    copy_in<T>(sm + lay.off_seg, g.seg, (size_t)lay.L * sizeof(int2));
    copy_in<T>(sm + lay.off_gk, g.gk, (size_t)lay.L * sizeof(int));
    copy_in<T>(sm + lay.off_pk, g.pk, (size_t)lay.L * sizeof(int));
    copy_in<T>(sm + lay.off_soff, g.soff, (size_t)lay.S * sizeof(int));
    copy_in<T>(sm + lay.off_sn, g.sn, (size_t)lay.S * sizeof(int));
    copy_in<T>(sm + lay.off_sf, g.sf, (size_t)lay.S * sizeof(int));
    copy_in<T>(sm + lay.off_smode, g.smode, (size_t)lay.S * sizeof(int));
    copy_in<T>(sm + lay.off_sfoff, g.sfoff, (size_t)lay.S * sizeof(long long));
    copy_in<T>(sm + lay.off_tasks, g.tasks, (size_t)lay.n_tasks * sizeof(int4));
    __syncthreads();
    IterArgs<T> a = g;
    a.F = reinterpret_cast<const T *>(sm + lay.off_F);
    a.bt = reinterpret_cast<const T *>(sm + lay.off_bt);
    a.mu = reinterpret_cast<T *>(sm + lay.off_mu);
    a.ds = reinterpret_cast<T *>(sm + lay.off_ds);
    a.ct = reinterpret_cast<const T *>(sm + lay.off_ct);
    a.lbt = reinterpret_cast<const T *>(sm + lay.off_lbt);
    a.ubt = reinterpret_cast<const T *>(sm + lay.off_ubt);
    a.seg = reinterpret_cast<const int2 *>(sm + lay.off_seg);
    a.gk = reinterpret_cast<const int *>(sm + lay.off_gk);
    a.pk = reinterpret_cast<const int *>(sm + lay.off_pk);
    a.soff = reinterpret_cast<const int *>(sm + lay.off_soff);
    a.sn = reinterpret_cast<const int *>(sm + lay.off_sn);
    a.sf = reinterpret_cast<const int *>(sm + lay.off_sf);
    a.smode = reinterpret_cast<const int *>(sm + lay.off_smode);
    a.sfoff = reinterpret_cast<const long long *>(sm + lay.off_sfoff);
    a.tasks = reinterpret_cast<const int4 *>(sm + lay.off_tasks);
    T *ub[2] = {reinterpret_cast<T *>(sm + lay.off_u0), reinterpret_cast<T *>(sm + lay.off_u1)};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    T *sv = reinterpret_cast<T *>(sm + lay.off_sv) + warp * 2 * lay.vstride;
    __shared__ double red[32][6];
    __shared__ int stop;
    if (threadIdx.x == 0) stop = 0;
    int par = 0, it = 0;
    __syncthreads();
    for (it = 0; it < n_iters; ++it) {
        const bool chk = ((it + 1) % check_every) == 0 || it == n_iters - 1;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if (chk) {
            for (int t = warp; t < lay.n_tasks; t += nw)
                run_task<T, true, true>(a, t, lane, ub[par], ub[par ^ 1], sv, lay.vstride, acc);
        } else {
            for (int t = warp; t < lay.n_tasks; t += nw)
                run_task<T, false, true>(a, t, lane, ub[par], ub[par ^ 1], sv, lay.vstride, acc);
        }
        par ^= 1;
        if (chk) {
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[q] = warp_sum(acc[q]);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 6; ++q) red[warp][q] = acc[q];
            __syncthreads();
            if (threadIdx.x == 0) {
                double s[6] = {0, 0, 0, 0, 0, 0};
                for (int w = 0; w < nw; ++w)
                    for (int q = 0; q < 6; ++q) s[q] += red[w][q];
                const int since = ((it + 1) % check_every) == 0 ? check_every : ((it + 1) % check_every);
                apply_test(st, s, rho_d, since);
                stop = st->done;
            }
        }
        __syncthreads();
        if (stop) { ++it; break; }
    }
    // write back the iterate; u of the last iteration goes to u_glob and the
    // u that produced its global update to u_glob + L (parity kept by caller)
    for (int i = threadIdx.x; i < lay.L; i += blockDim.x) {
        g.mu[i] = a.mu[i];
        g.ds[i] = a.ds[i];
        u_glob[i] = ub[par][i];
        u_glob[lay.L + i] = ub[par ^ 1][i];
    }
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

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
__global__ void __launch_bounds__(128) k_recenter_bbar(int S, const int *soff, const int *sn,
                                                       const int *sf, const int *smode,
                                                       const long long *sfoff, const double *F,
                                                       const int *gk, const double *xr,
                                                       const double *lamr, const double *bbar,
                                                       double rho, T *bt, const DevStatus *st) {
    __shared__ double buf[4][2][OPF_MAX_NS];
    if (st && st->done) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * 4 + w;
    if (s >= S) return;
    const int n = sn[s], f = sf[s], mode = smode[s], so = soff[s];
    const double *Fs = F + sfoff[s];
    double *v = buf[w][0], *t = buf[w][1];
    for (int r = lane; r < n; r += 32) v[r] = xr[gk[so + r]] + lamr[so + r] / rho;
    __syncwarp();
    for (int c = lane; c < f; c += 32) {
        double acc = 0.0;
        for (int r = 0; r < n; ++r) acc += Fs[(long long)c * n + r] * v[r];
        t[c] = acc;
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
        double y = 0.0;
        for (int c = 0; c < f; ++c) y += Fs[(long long)c * n + r] * t[c];
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

void launch_precompute(const PreArgs &a, cudaStream_t st) {
    const int warps = 4;
    k_precompute<<<(a.S + warps - 1) / warps, 32 * warps, 0, st>>>(a);
}

template <typename T>
void launch_iterate(const IterArgs<T> &a, const T *u_in, T *u_out, int vstride, double *partials,
                    const DevStatus *st, bool check, cudaStream_t s) {
    const int blocks = (a.n_tasks + 7) / 8;
    const size_t shm = 8 * 2 * (size_t)vstride * sizeof(T);
    if (check) k_iterate<T, true><<<blocks, 256, shm, s>>>(a, u_in, u_out, vstride, partials, st);
    else k_iterate<T, false><<<blocks, 256, shm, s>>>(a, u_in, u_out, vstride, partials, st);
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
int prepare_cta_engine(unsigned bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_cta_engine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    return e == cudaSuccess ? 0 : -1;
}

template <typename T>
void launch_cta_engine(const IterArgs<T> &g, const CtaLayout &lay, T *u_glob, int n_iters,
                       int check_every, DevStatus *st, double rho, cudaGraphConditionalHandle cond,
                       int use_cond, cudaStream_t s) {
    k_cta_engine<T><<<1, 1024, lay.bytes, s>>>(g, lay, u_glob, n_iters, check_every, st, rho, cond,
                                               use_cond);
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
                     const int *soff, const int *sn, const int *sf, const int *smode,
                     const long long *sfoff, const double *F64, const double *bbar, double rho,
                     T *bt, const DevStatus *st, cudaStream_t s) {
    k_recenter_slots<T><<<nblocks(L, 256), 256, 0, s>>>(L, gk, xr_old, xr_new, ds, mu, lamr, st);
    k_recenter_globals<T><<<nblocks(G, 256), 256, 0, s>>>(G, gseg, uslot, lamr, c64, lb, ub, xr_new,
                                                          ct, lbt, ubt, st);
    k_recenter_bbar<T><<<(S + 3) / 4, 128, 0, s>>>(S, soff, sn, sf, smode, sfoff, F64, gk, xr_new,
                                                   lamr, bbar, rho, bt, st);
}

#define OPF_INST(T)                                                                                   \
    template void launch_iterate<T>(const IterArgs<T> &, const T *, T *, int, double *,               \
                                    const DevStatus *, bool, cudaStream_t);                           \
    template int prepare_cta_engine<T>(unsigned);                                                     \
    template void launch_cta_engine<T>(const IterArgs<T> &, const CtaLayout &, T *, int, int,         \
                                       DevStatus *, double, cudaGraphConditionalHandle, int,          \
                                       cudaStream_t);                                                 \
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
                                     const double *, const double *, T *, T *, T *, const int *,      \
                                     const int *, const int *, const int *, const long long *,        \
                                     const double *, const double *, double, T *, const DevStatus *,  \
                                     cudaStream_t);
OPF_INST(double)
OPF_INST(float)
template void launch_cast<double, float>(long long, const double *, float *, cudaStream_t);
template void launch_cast<float, double>(long long, const float *, double *, cudaStream_t);

}  // namespace opf
