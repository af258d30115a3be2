// Batched ADMM (Algorithm 1) over many instances of one model: every instance
// shares A_s, c and the bounds (so M_s = -Abar_s and its factor F) and has its
// own right-hand side b, hence its own bbar = A_s^+ b.
//
//  k_batch_engine  n_iters iterations of Algorithm 1 for the K instances of
//                  one CTA, all resident: factors, u = rho x_s - lambda and
//                  rho x in shared memory; lambda and bbar~ in tensor memory
//                  (FP32 plans) or streamed from L2 as 16-byte vectors, the
//                  test data from L2.  Per iteration:
//                    G. per (global, instance): Eq. closed_1 as a fixed-order
//                       sum over the global's copies of u, rho x stored into
//                       the copies' slots (a global with one copy and no
//                       bounds needs none: with c~ = 0 its rho x is the u of
//                       its slot);
//                    -- CTA barrier --
//                    L. per warp task: J member subsystems x K instances,
//                       in units of rho (no multiplies): V = rho x_g + lambda
//                       (= rho v), rho x_s = M V + rho bbar~ as one pass over
//                       the factor rows (w_r = <F_r, V>, y += w_r F_r),
//                       lambda <- V - rho x_s (Eq. ADMM-3 with
//                       rho x_g = V - lambda), u = rho x_s - lambda;
//                    -- CTA barrier --
//                  and every check_every iterations the Sec. III-C sums per
//                  instance in FP64 and the test; finished instances freeze.
//  k_bref_*        FP64 re-centring: x_ref = next global update of the FP64
//                  state, lambda_ref = lambda (less delta at unbounded
//                  globals, so that their shifted cost is zero), shifted data
//                  written in the engine layout (the engine iterates on
//                  x_s - x_ref[g] and lambda - lambda_ref, the change of
//                  variables of the single-instance engines).
//  k_bunshift_*    back to the unshifted FP64 state.
//  k_bbar          bbar = A_s^+ b per instance and subsystem (Sec. III-B).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "opf_internal.h"
#include "test_rule.cuh"
#include "tmem.cuh"

namespace opf {

namespace {

template <typename T>
struct Q4 {
    T v[4];
};

__device__ __forceinline__ Q4<float> ld4(const float *p) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Q4<double> ld4(const double *p) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float *p, const Q4<float> &q) {
    *reinterpret_cast<float4 *>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ void st4(double *p, const Q4<double> &q) {
    *reinterpret_cast<double2 *>(p) = make_double2(q.v[0], q.v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(q.v[2], q.v[3]);
}

template <typename T>
__device__ __forceinline__ T clampT(T x, T lo, T hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

}  // namespace

// ============================================================ engine
// K-wide register rows: K consecutive values moved with the widest aligned
// vector loads/stores (the offsets used are multiples of K elements).
template <typename T, int K>
struct RowK {
    T v[K];
};

template <typename T, int K, bool L2ONLY>
__device__ __forceinline__ void load_row(RowK<T, K> &r, const T *p) {
    if constexpr (K * sizeof(T) >= 16) {
#pragma unroll
        for (int i = 0; i < K; i += 16 / sizeof(T)) {
            if constexpr (sizeof(T) == 4) {
                const float4 t = L2ONLY ? __ldcg(reinterpret_cast<const float4 *>(p + i))
                                        : *reinterpret_cast<const float4 *>(p + i);
                r.v[i] = t.x; r.v[i + 1] = t.y; r.v[i + 2] = t.z; r.v[i + 3] = t.w;
            } else {
                const double2 t = L2ONLY ? __ldcg(reinterpret_cast<const double2 *>(p + i))
                                         : *reinterpret_cast<const double2 *>(p + i);
                r.v[i] = t.x; r.v[i + 1] = t.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) r.v[i] = L2ONLY ? __ldcg(p + i) : p[i];
    }
}

template <typename T, int K>
__device__ __forceinline__ void store_row(T *p, const RowK<T, K> &r) {
    if constexpr (K * sizeof(T) >= 16) {
#pragma unroll
        for (int i = 0; i < K; i += 16 / sizeof(T)) {
            if constexpr (sizeof(T) == 4)
                *reinterpret_cast<float4 *>(p + i) = make_float4(r.v[i], r.v[i + 1], r.v[i + 2], r.v[i + 3]);
            else
                *reinterpret_cast<double2 *>(p + i) = make_double2(r.v[i], r.v[i + 1]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) p[i] = r.v[i];
    }
}

__device__ __forceinline__ Q4<float> ld4cg(const float *p) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    return {{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Q4<double> ld4cg(const double *p) {
    const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcg(reinterpret_cast<const double2 *>(p + 2));
    return {{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4cg(float *p, const Q4<float> &q) {
    __stcg(reinterpret_cast<float4 *>(p), make_float4(q.v[0], q.v[1], q.v[2], q.v[3]));
}
__device__ __forceinline__ void st4cg(double *p, const Q4<double> &q) {
    __stcg(reinterpret_cast<double2 *>(p), make_double2(q.v[0], q.v[1]));
    __stcg(reinterpret_cast<double2 *>(p + 2), make_double2(q.v[2], q.v[3]));
}

// One warp task with exactly NQT chunks per position.  chg holds g * K per
// slot (-1: padding); bt holds +bbar~ for members with M = F^T F and -bbar~
// for M = I - F^T F, so that y = bt + F^T w gives x_s = y or v - y.
// Shared-memory slot array: chunk ch, slot e, column sc at
// (ch * 4 + (e ^ (ch & 3))) * K + sc.  Between the two phases of an
// iteration it holds, at every slot, x of the slot's global (written there by
// the global update); otherwise u = rho x_s - lambda of the slot.  The
// swizzle e ^ (ch & 3) puts the four member positions of a warp (consecutive
// chunks) on distinct banks.  Padding slots hold 0.
template <int K>
__device__ __forceinline__ int upos(int ch, int e, int sc) {
    return (ch * 4 + (e ^ (ch & 3))) * K + sc;
}

// ---- tensor memory (tcgen05, tmem.cuh): lambda and bbar~ of the tasks,
// 32-bit columns.
// 8 consecutive columns of the lane: lambda (4) then bbar~ (4) of one chunk
__device__ __forceinline__ void tm_ld8(unsigned taddr, Q4<float> &m, Q4<float> &b) {
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        m.v[e] = __uint_as_float(r[e]);
        b.v[e] = __uint_as_float(r[4 + e]);
    }
}
__device__ __forceinline__ void tm_st8(unsigned taddr, const Q4<float> &m, const Q4<float> &b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(m.v[0])), "r"(__float_as_uint(m.v[1])), "r"(__float_as_uint(m.v[2])),
                 "r"(__float_as_uint(m.v[3])), "r"(__float_as_uint(b.v[0])), "r"(__float_as_uint(b.v[1])),
                 "r"(__float_as_uint(b.v[2])), "r"(__float_as_uint(b.v[3]))
                 : "memory");
}
__device__ __forceinline__ void tm_st4(unsigned taddr, const Q4<float> &m) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(__float_as_uint(m.v[0])), "r"(__float_as_uint(m.v[1])), "r"(__float_as_uint(m.v[2])),
                 "r"(__float_as_uint(m.v[3]))
                 : "memory");
}
__device__ __forceinline__ void tm_ld4(unsigned taddr, Q4<float> &m) {
    unsigned r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int e = 0; e < 4; ++e) m.v[e] = __uint_as_float(r[e]);
}

// Tensor-memory staging of one task (TMTASK): at the start of a launch
// lambda and bbar~ from the engine arrays into the task's columns; at a
// freeze or the end lambda back to the engine array for the columns flagged
// in `wcols` (bit sc), after the lanes' own loads.
template <int K, int NQT>
__device__ __forceinline__ void tm_stage_in(const BatchTask &tk, unsigned tl, const float *mu_c, const float *bt_c,
                                            int jpos, int sc, float rho) {
    constexpr int J = 32 / K;
    const unsigned col = (unsigned)(tk.tm >> 2);
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
        const int off = ((tk.ch0 + jpos + q * J) * K + sc) * 4;
        Q4<float> b = ld4cg(bt_c + off);
#pragma unroll
        for (int e = 0; e < 4; ++e) b.v[e] *= rho;     // rho bbar~
        tm_st8(tl + col + 8 * q, ld4cg(mu_c + off), b);
    }
}
template <int K, int NQT>
__device__ __forceinline__ void tm_stage_out(const BatchTask &tk, unsigned tl, float *mu_c, int jpos, int sc,
                                             bool write) {
    constexpr int J = 32 / K;
    const unsigned col = (unsigned)(tk.tm >> 2);
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
        Q4<float> m;
        tm_ld4(tl + col + 8 * q, m);
        tm_wait_ld();
        if (write) st4cg(mu_c + ((tk.ch0 + jpos + q * J) * K + sc) * 4, m);
    }
}

// The slot array holds rho x_g at every slot when the task starts (the global
// update wrote it; a one-copy unbounded global's slot holds its u, which is
// that value) and gets u at the end; y starts at +-rho bbar~ (tensor-memory
// plans stage it scaled, the others scale it on load).
template <typename T, int K, int NQT, bool TM>
__device__ __forceinline__ void batch_task(const BatchTask &tk, const T *Fs, T *us, T *mu_c, const T *bt_c,
                                           T *ds_c, const T *lr_c, const T *xr_c, const int4 *chg, int jpos,
                                           int sc, T rho, T inv_rho, bool check, bool act, bool wds,
                                           double *redw, unsigned tl) {
    constexpr int J = 32 / K;
    const int mode1 = (tk.modes >> (jpos >> tk.lp)) & 1;
    T v[4 * NQT], y[4 * NQT];
    double c0 = 0.0, c1 = 0.0, c3 = 0.0, c4 = 0.0;
    // FP32 plans: a lane's test terms (FP32 already) summed over the task's
    // chunks in FP32 and added to the FP64 sums once per task (FP64 adds
    // cost this part 64 FP32 ones)
    float f0 = 0.f, f1 = 0.f, f3 = 0.f, f4 = 0.f;
    const int ch0 = tk.ch0 + jpos;
    const unsigned tcol = tl + (unsigned)(tk.tm >> 2);
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
        const int ch = ch0 + q * J;
        const int off = (ch * K + sc) * 4;
        Q4<T> m4, b4;
        if constexpr (TM) {
            tm_ld8(tcol + 8 * q, m4, b4);
            tm_wait_ld();
        } else {
            m4 = ld4cg(mu_c + off);
            b4 = ld4cg(bt_c + off);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            y[4 * q + e] = TM ? b4.v[e] : rho * b4.v[e];
            v[4 * q + e] = us[upos<K>(ch, e, sc)] + m4.v[e];
        }
    }
    // rho x_s = M V + rho bbar~ over the factor rows, two rows per step
    const int rstride = NQT * J * 4;
    const T *F0 = Fs + tk.foff + jpos * 4;
    const int red_top = tk.p * K;
    // (the task's row count is even: a member's missing rows are zero)
    for (int r = 0; r < tk.f; r += 2, F0 += 2 * rstride) {
        const T *F1 = F0 + rstride;
        // one accumulation chain per row (four partial sums and their adds
        // measured 4.5 % slower per launch: more instructions)
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int q = 0; q < NQT; ++q) {
            const Q4<T> f0 = ld4(F0 + q * J * 4);
            const Q4<T> f1 = ld4(F1 + q * J * 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                s0 += f0.v[e] * v[4 * q + e];
                s1 += f1.v[e] * v[4 * q + e];
            }
        }
        for (int o = K; o < red_top; o <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
#pragma unroll
        for (int q = 0; q < NQT; ++q) {
            const Q4<T> f0 = ld4(F0 + q * J * 4);
            const Q4<T> f1 = ld4(F1 + q * J * 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                y[4 * q + e] += f0.v[e] * s0;
                y[4 * q + e] += f1.v[e] * s1;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NQT; ++q) {
        const int ch = ch0 + q * J;
        const int off = (ch * K + sc) * 4;
        Q4<T> x4, m4, u4, r4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const T vv = v[4 * q + e];
            const T rx = mode1 ? y[4 * q + e] : vv - y[4 * q + e];     // rho x_s
            const T mun = vv - rx;
            r4.v[e] = rx;
            m4.v[e] = mun;
            u4.v[e] = rx - mun;
        }
        // x_s~ (written on wds iterations, test terms); computed on every
        // iteration: a branch here measured 6 % slower per launch
#pragma unroll
        for (int e = 0; e < 4; ++e) x4.v[e] = r4.v[e] * inv_rho;
        if (check) {
            const int4 g4 = __ldg(chg + ch);
            const int gg[4] = {g4.x, g4.y, g4.z, g4.w};
            const Q4<T> o4 = ld4cg(ds_c + off);
            const Q4<T> l4 = ld4cg(lr_c + off);
            T t0 = T(0), t1 = T(0), t3 = T(0), t4 = T(0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (gg[e] < 0) continue;
                const T d0 = (us[upos<K>(ch, e, sc)] - r4.v[e]) * inv_rho, d1 = x4.v[e] - o4.v[e];
                const T xa = x4.v[e] + __ldcg(xr_c + gg[e]);
                const T la = m4.v[e] + l4.v[e];
                t0 += d0 * d0;
                t1 += d1 * d1;
                t3 += xa * xa;
                t4 += la * la;
            }
            if constexpr (sizeof(T) == 4) {
                f0 += t0;
                f1 += t1;
                f3 += t3;
                f4 += t4;
            } else {
                c0 += (double)t0;
                c1 += (double)t1;
                c3 += (double)t3;
                c4 += (double)t4;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) us[upos<K>(ch, e, sc)] = u4.v[e];
        if constexpr (TM) {
            // every lane (a frozen column keeps iterating in tensor memory;
            // its lambda went to the engine array when it froze)
            tm_st4(tcol + 8 * q, m4);
            if (act && wds) st4cg(ds_c + off, x4);
        } else if (act) {
            st4cg(mu_c + off, m4);
            if (wds) st4cg(ds_c + off, x4);
        }
    }
    if (check) {
        if constexpr (sizeof(T) == 4) {
            c0 = (double)f0;
            c1 = (double)f1;
            c3 = (double)f3;
            c4 = (double)f4;
        }
        // per instance column: sum over the J member positions, in lane order
        for (int o = K; o < 32; o <<= 1) {
            c0 += __shfl_xor_sync(0xffffffffu, c0, o);
            c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            c3 += __shfl_xor_sync(0xffffffffu, c3, o);
            c4 += __shfl_xor_sync(0xffffffffu, c4, o);
        }
        if (jpos == 0) {
            redw[sc * 6 + 0] += c0;
            redw[sc * 6 + 1] += c1;
            redw[sc * 6 + 3] += c3;
            redw[sc * 6 + 4] += c4;
        }
    }
}

// K: instance columns per CTA (compile time), J = 32 / K member positions.
// NQ: chunks of 4 slots a lane can hold (registers v and y: 2 * 4 * NQ).
// FG: factors read from global memory (L1/L2) instead of shared memory.
// TM (FP32 only): lambda and bbar~ of the tasks in tensor memory for the
// launch instead of streamed from L2; the tasks of lane quadrant q run on the
// warps w with w % 4 == q (a dynamic schedule per quadrant).
template <typename T, int K, int NQ, bool FG, bool TM>
__global__ void __launch_bounds__(512, 1)
    k_batch_engine(BatchArgs<T> a, int n_iters, int check_every) {
    constexpr int J = 32 / K;
    constexpr int KS = K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : K == 16 ? 4 : 5;
    constexpr int KQ = K < 4 ? K : 4;          // columns per global-update item
    constexpr int NQD = K / KQ;                  // items per global
    constexpr int QS = NQD == 1 ? 0 : NQD == 2 ? 1 : NQD == 4 ? 2 : 3;
    // global-update items per thread taken together (their loads in flight
    // together): 1 in FP32 (on the 1024 x 123-bus batch, with the first two
    // copies' rows in the table entry and c~ in shared memory, 1 to 4 items
    // gave 12.89, 12.97, 13.30 and 12.98 ms per launch of 2000 iterations;
    // with the copy rows looked up in a second table and c~ read from L2, 2
    // had been fastest: more items cost predicated instructions and
    // registers the rest of the iteration needs), 4 for FP64 rows of 4
    constexpr int GB = (sizeof(T) == 8 && KQ == 4) ? 4 : 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Fsm = reinterpret_cast<T *>(smraw);
    const T *Fs = FG ? a.Fpk : Fsm;
    T *us = reinterpret_cast<T *>(smraw + a.off_u);
    int4 *gts = reinterpret_cast<int4 *>(smraw + a.off_gt);      // [Gs] (row0, row1, copies | first extra << 8, bounded index)
    T *rcs = reinterpret_cast<T *>(smraw + a.off_rc);            // 1 / N by copy count N
    BatchTask *tks = reinterpret_cast<BatchTask *>(smraw + a.off_task);   // the warp tasks
    int *usg = reinterpret_cast<int *>(smraw + a.off_useg);      // slot-array rows of the third and later copies
    T *bnd = reinterpret_cast<T *>(smraw + a.off_bnd);           // [NB][3][K]: rho (bounds - x_ref), c~
    double *red = reinterpret_cast<double *>(smraw + a.off_red);
    int *flags = reinterpret_cast<int *>(smraw + a.off_flag);    // [0,K) running, [K,2K) just finished
    int *tnext = flags + 2 * K;                                    // next task of the dynamic schedule (per quadrant)
    __shared__ unsigned tm_base;                                   // tensor-memory address of the allocation
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nthr = blockDim.x;
    const int c = blockIdx.x;
    if (tid < K) {
        const int in = a.inst[c * K + tid];
        flags[tid] = (in >= 0 && !a.st[in].done) ? 1 : 0;
        flags[K + tid] = 0;
    }
    __syncthreads();
    {
        int any = 0;
        for (int q = 0; q < K; ++q) any |= flags[q];
        if (!any) return;
    }
    // factors and the global-update tables into shared memory (nF is a multiple of 4)
    if (!FG)
        for (int i = tid * 4; i < a.nF; i += nthr * 4) st4(Fsm + i, ld4(a.Fpk + i));
    for (int j = tid; j < a.Gs; j += nthr) gts[j] = __ldg(a.gtab + j);
    // 1 / N by copy count N: the global update stores rho x = (sum u - c~) / N
    for (int i = tid; i < kBatchRecip; i += nthr) rcs[i] = i ? (T)(1.0 / (double)i) : T(0);
    for (int i = tid; i < a.n_tasks; i += nthr) tks[i] = a.tasks[i];
    for (int k = tid; k < a.n_uxt; k += nthr) usg[k] = __ldg(a.uxt + k);
    const size_t sb = (size_t)c * a.NCH * K * 4;     // this CTA's slot arrays
    const size_t gb = (size_t)c * a.G * K;           // global arrays
    const size_t bb = (size_t)c * a.NB * K;          // bounded-global arrays
    for (int idx = tid; idx < a.NB * K; idx += nthr) {
        const int b = idx >> KS, col = idx & (K - 1);
        bnd[(b * 3) * K + col] = a.rho * __ldcg(a.lbt + bb + idx);         // rho (bounds - x_ref)
        bnd[(b * 3 + 1) * K + col] = a.rho * __ldcg(a.ubt + bb + idx);
        bnd[(b * 3 + 2) * K + col] = __ldcg(a.cbt + bb + idx);              // c~
    }
    T *mu_c = a.mu + sb, *ds_c = a.ds + sb;
    const T *bt_c = a.bt + sb, *lr_c = a.lref + sb;
    // u = rho d - mu into the swizzled slot array
    for (int idx = tid; idx < a.NCH * K; idx += nthr) {
        const int ch = idx >> KS, col = idx & (K - 1);
        const Q4<T> d = ld4cg(ds_c + (size_t)idx * 4), m = ld4cg(mu_c + (size_t)idx * 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) us[upos<K>(ch, e, col)] = a.rho * d.v[e] - m.v[e];
    }
    const int sc = tid & (K - 1);
    const int jpos = lane >> KS;
    const int n_warps = nthr >> 5;
    const int qd = w & 3, wq = w >> 2, nwq = n_warps >> 2;     // quadrant, warp in it, warps per quadrant
    unsigned tl = 0;                                             // this warp's tensor-memory lane base
    if constexpr (TM) {
        if (w == 0) tm_alloc(&tm_base, a.tm_cols);
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        tl = tm_base + ((unsigned)(32 * qd) << 16);
        for (int t = a.qstart[qd] + wq; t < a.qstart[qd + 1]; t += nwq) {
            const BatchTask tk = a.tasks[t];
            switch (tk.nq) {
                case 1: tm_stage_in<K, 1>(tk, tl, mu_c, bt_c, jpos, sc, a.rho); break;
                case 2: tm_stage_in<K, 2>(tk, tl, mu_c, bt_c, jpos, sc, a.rho); break;
                case 3: tm_stage_in<K, 3>(tk, tl, mu_c, bt_c, jpos, sc, a.rho); break;
                default: tm_stage_in<K, 4>(tk, tl, mu_c, bt_c, jpos, sc, a.rho); break;
            }
        }
        tm_wait_st();
        tm_fence_before();
    }
    __syncthreads();
    if constexpr (TM) tm_fence_after();
    const T *xr_c = a.xrf + gb + sc;
    const T rho = a.rho, inv_rho = a.inv_rho;
    double *redw = red + (size_t)w * K * 6;      // this warp's test sums per column
    int last_check = 0;
    bool all_done = false;
    const int GK = a.G * K;
    const int GQ = a.Gs * NQD;       // the globals the global update computes (the table's first Gs)
    for (int it = 0; it < n_iters; ++it) {
        const bool check = check_every > 0 && ((it + 1) % check_every == 0);
        const bool last = it == n_iters - 1;
        const bool wds = check || last || (check_every > 0 && ((it + 2) % check_every == 0));
        const bool act = flags[sc] != 0;
        if (check && lane < K)
#pragma unroll
            for (int q = 0; q < 6; ++q) redw[lane * 6 + q] = 0.0;
        if constexpr (TM) {
            if (tid < 4) tnext[tid] = a.qstart[tid] + nwq;
        } else if (tid == 0) {
            *tnext = n_warps;
        }
        // ---- G: global update (Eq. closed_1).  An item is one global and KQ of
        // its columns: sum of u over the copies, shift by c~ (bounded globals,
        // whose table entry names their bounded index; elsewhere c~ = 0),
        // 1 / N, clip to rho (bounds - x_ref), and rho x stored into every
        // copy's slot; GB items per thread
        for (int b0 = tid; b0 < GQ; b0 += GB * nthr) {
            // the GB items of this thread advance stage by stage, so that the
            // loads of one stage are in flight together: the table entries
            // (with the first two copies' rows), their u; further copies
            // (vertices of degree > 1) one by one; then the update
            RowK<T, KQ> sum[GB];
            int4 gtj[GB];
            int row0[GB], row1[GB];
#pragma unroll
            for (int j = 0; j < GB; ++j) {
                const int item = b0 + j * nthr;
                gtj[j] = make_int4(0, 0, 0, -1);
                if (item < GQ) gtj[j] = gts[item >> QS];
                const int hq = (item & (NQD - 1)) * KQ;
                row0[j] = gtj[j].x + hq;
                row1[j] = gtj[j].y + hq;
            }
#pragma unroll
            for (int j = 0; j < GB; ++j) {
                const int cnt = gtj[j].z & 0xff;
#pragma unroll
                for (int k = 0; k < KQ; ++k) sum[j].v[k] = T(0);
                if (cnt > 0) {
                    RowK<T, KQ> u0;
                    load_row<T, KQ, false>(u0, us + row0[j]);
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] += u0.v[k];
                }
                if (cnt > 1) {
                    RowK<T, KQ> u1;
                    load_row<T, KQ, false>(u1, us + row1[j]);
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] += u1.v[k];
                }
            }
#pragma unroll
            for (int j = 0; j < GB; ++j) {
                const int item = b0 + j * nthr;
                if (item >= GQ) continue;
                const int h = item & (NQD - 1);
                const int4 gt = gtj[j];
                const int cnt = gt.z & 0xff, st0 = (gt.z >> 8) - 2;    // usg[st0 + q]: copy q >= 2
                for (int q = 2; q < cnt; ++q) {
                    RowK<T, KQ> uq;
                    load_row<T, KQ, false>(uq, us + usg[st0 + q] + h * KQ);
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] += uq.v[k];
                }
                const T rcp = rcs[cnt];
                if (gt.w >= 0) {
                    RowK<T, KQ> lo, hi, cr;
                    load_row<T, KQ, false>(cr, bnd + (gt.w * 3 + 2) * K + h * KQ);
                    load_row<T, KQ, false>(lo, bnd + (gt.w * 3) * K + h * KQ);
                    load_row<T, KQ, false>(hi, bnd + (gt.w * 3 + 1) * K + h * KQ);
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] = (sum[j].v[k] - cr.v[k]) * rcp;
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] = clampT(sum[j].v[k], lo.v[k], hi.v[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < KQ; ++k) sum[j].v[k] *= rcp;
                }
                if (cnt > 0) store_row<T, KQ>(us + row0[j], sum[j]);
                if (cnt > 1) store_row<T, KQ>(us + row1[j], sum[j]);
                for (int q = 2; q < cnt; ++q) store_row<T, KQ>(us + usg[st0 + q] + h * KQ, sum[j]);
            }
        }
        __syncthreads();
        if (check || last) {
            // x of each global (rho x at its first copy): objective and
            // ||B x||^2 per column on test iterations, and x~ of the running
            // instances for their results (thread column sc = tid % K)
            // (FP32 plans: x_ref + x~ and the thread's partial sums in FP32,
            // FP64 from the warp sums on; FP64 plans: FP64 throughout)
            double c2 = 0.0, c5 = 0.0;
            T p2 = T(0), p5 = T(0);
            for (int item = tid; item < GK; item += nthr) {
                const int j = item >> KS;
                const int2 gt = make_int2(__ldg(a.gx + j), 0);   // first copy's row | copies << 24
                const int i = __ldg(a.gperm + j);
                const size_t gi = gb + (size_t)i * K + sc;
                const T xv = us[(gt.x & 0xffffff) + sc] * a.inv_rho;
                if (flags[sc]) a.xo[gi] = xv;
                if (check) {
                    if constexpr (sizeof(T) == 4) {
                        const T xa = xv + __ldcg(a.xrf + gi);
                        p2 += (T)((unsigned)gt.x >> 24) * xa * xa;
                        p5 += __ldg(a.cost + i) * xa;
                    } else {
                        const double xa = (double)xv + (double)__ldcg(a.xrf + gi);
                        c2 += (double)((unsigned)gt.x >> 24) * xa * xa;
                        c5 += (double)__ldg(a.cost + i) * xa;
                    }
                }
            }
            if constexpr (sizeof(T) == 4) {
                c2 = (double)p2;
                c5 = (double)p5;
            }
            if (check) {
                for (int o = K; o < 32; o <<= 1) {
                    c2 += __shfl_xor_sync(0xffffffffu, c2, o);
                    c5 += __shfl_xor_sync(0xffffffffu, c5, o);
                }
                if (lane < K) {
                    redw[lane * 6 + 2] += c2;
                    redw[lane * 6 + 5] += c5;
                }
            }
            __syncthreads();      // the slots still hold x: read before phase L overwrites them
        }
        // ---- L: local update (Eq. closed_2) and dual update (Eq. ADMM-3)
        // tasks in decreasing cost; warps take the next one as they finish
        // (test iterations: task t on warp t % n_warps, a fixed summation order)
        {
            // each warp's first task is its own (the counter starts at
            // n_warps); the next task's index is claimed at the start of a
            // task and read at its end, so the atomic's latency is hidden
            // (tensor-memory plans: the same within the warp's quadrant)
            int t = TM ? a.qstart[qd] + wq : w;
            const int t_end = TM ? a.qstart[qd + 1] : a.n_tasks;
            const int t_step = TM ? nwq : n_warps;
            int *cnt = TM ? tnext + qd : tnext;
            while (t < t_end) {
                int claim = 0;
                if (!check && lane == 0) claim = atomicAdd(cnt, 1);
                const BatchTask tk = tks[t];
                switch (tk.nq) {
                    case 1: batch_task<T, K, 1, TM>(tk, Fs, us, mu_c, bt_c, ds_c, lr_c, xr_c, a.chg, jpos, sc, rho,
                                                    inv_rho, check, act, wds, redw, tl); break;
                    case 2: if constexpr (NQ >= 2) batch_task<T, K, 2, TM>(tk, Fs, us, mu_c, bt_c, ds_c, lr_c, xr_c,
                                                                           a.chg, jpos, sc, rho, inv_rho, check, act,
                                                                           wds, redw, tl); break;
                    case 3: if constexpr (NQ >= 3) batch_task<T, K, 3, TM>(tk, Fs, us, mu_c, bt_c, ds_c, lr_c, xr_c,
                                                                           a.chg, jpos, sc, rho, inv_rho, check, act,
                                                                           wds, redw, tl); break;
                    default: if constexpr (NQ >= 4) batch_task<T, K, 4, TM>(tk, Fs, us, mu_c, bt_c, ds_c, lr_c, xr_c,
                                                                            a.chg, jpos, sc, rho, inv_rho, check, act,
                                                                            wds, redw, tl); break;
                }
                t = check ? t + t_step : __shfl_sync(0xffffffffu, claim, 0);
            }
            if constexpr (TM) {
                tm_wait_st();
                tm_fence_before();
            }
        }
        if (check) {
            __syncthreads();
            if constexpr (TM) tm_fence_after();
            // one thread per (column, quantity) sums the warps' parts in warp
            // order into warp 0's slot, then one thread per column tests
            if (tid < 6 * K) {
                const int col = tid / 6, q = tid - 6 * col;
                double sum = 0.0;
                for (int ww = 0; ww < n_warps; ++ww) sum += red[((size_t)ww * K + col) * 6 + q];
                red[col * 6 + q] = sum;
            }
            __syncthreads();
            if (tid < K) {
                flags[K + tid] = 0;
                if (flags[tid]) {
                    const int in = a.inst[c * K + tid];
                    double s6[6];
#pragma unroll
                    for (int q = 0; q < 6; ++q) s6[q] = red[tid * 6 + q];
                    apply_test(&a.st[in], s6, a.rho_d, check_every);
                    if (a.st[in].done) {
                        flags[tid] = 0;
                        flags[K + tid] = 1;
                    }
                }
            }
            __syncthreads();
            last_check = it + 1;
            if constexpr (TM) {
                // lambda of the columns that just finished, to the engine array
                int fin = 0;
                for (int q = 0; q < K; ++q) fin |= flags[K + q];
                if (fin)
                    for (int t = a.qstart[qd] + wq; t < a.qstart[qd + 1]; t += nwq) {
                        const BatchTask tk = tks[t];
                        const bool wr = flags[K + sc] != 0;
                        switch (tk.nq) {
                            case 1: tm_stage_out<K, 1>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                            case 2: tm_stage_out<K, 2>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                            case 3: tm_stage_out<K, 3>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                            default: tm_stage_out<K, 4>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                        }
                    }
            }
            int any = 0;
            for (int q = 0; q < K; ++q) any |= flags[q];
            if (!any) {
                all_done = true;
                break;
            }
        } else {
            __syncthreads();
            if constexpr (TM) tm_fence_after();
        }
    }
    if (!all_done && tid < K && flags[tid]) a.st[a.inst[c * K + tid]].iter += n_iters - last_check;
    if constexpr (TM) {
        // lambda of the columns still running, then the allocation is freed
        if (!all_done)
            for (int t = a.qstart[qd] + wq; t < a.qstart[qd + 1]; t += nwq) {
                const BatchTask tk = tks[t];
                const bool wr = flags[sc] != 0;
                switch (tk.nq) {
                    case 1: tm_stage_out<K, 1>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                    case 2: tm_stage_out<K, 2>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                    case 3: tm_stage_out<K, 3>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                    default: tm_stage_out<K, 4>(tk, tl, (float *)mu_c, jpos, sc, wr); break;
                }
            }
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (w == 0) tm_dealloc(tm_base, a.tm_cols);
    }
}

// ============================================================ per-instance data
// Engine column of an instance: ipos[inst] = c * K + sc (-1: not placed).

// Start point of Sec. V-A for instances [i0, i0 + cnt): x_s = x0[g], lambda = 0.
__global__ void k_binit(int i0, int cnt, int L, const int *gk, const double *x0, double *xs, double *lam,
                        DevStatus *st, long long max_iter, double eps_rel, double eps_abs) {
    const long long n = (long long)cnt * L;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = i0 + (int)(t / L), k = (int)(t % L);
        xs[(size_t)in * L + k] = x0[gk[k]];
        lam[(size_t)in * L + k] = 0.0;
        if (k == 0) {
            DevStatus z;
            memset(&z, 0, sizeof(z));
            z.max_iter = max_iter;
            z.eps_rel = eps_rel;
            z.eps_abs_pres = eps_abs;
            st[in] = z;
        }
    }
}

// Warm start of instances [i0, i0 + cnt): x_s and lambda copied from one
// start state (device slot order), e.g. a converged base-load solution.
__global__ void k_bwarm(int i0, int cnt, int L, const double *xs0, const double *lam0, double *xs, double *lam) {
    const long long n = (long long)cnt * L;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = i0 + (int)(t / L), k = (int)(t % L);
        xs[(size_t)in * L + k] = xs0[k];
        lam[(size_t)in * L + k] = lam0[k];
    }
}

__global__ void k_bfill(int cnt, int nrows, const double *b0, double *rhs) {
    const long long n = (long long)cnt * nrows;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        rhs[t] = b0[t % nrows];
}

// rhs in device row order from canonical rows, or from load values.
__global__ void k_brhs_perm(int i0, int cnt, int nrows, const int *c2d, const double *src, double *rhs) {
    const long long n = (long long)cnt * nrows;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / nrows), r = (int)(t % nrows);
        rhs[(size_t)(i0 + j) * nrows + c2d[r]] = src[t];
    }
}

__global__ void k_brhs_loads(int i0, int cnt, int nrows, int nload, const int *rsrc, const double *rcoef,
                             const double *b0, const double *lp, const double *lq, double *rhs) {
    const long long n = (long long)cnt * nrows;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / nrows), r = (int)(t % nrows);
        const int s = rsrc[r];
        double v = b0[r];
        if (s >= 0) {
            const double *src = (s & 1) ? lq : lp;
            v = rcoef[r] * src[(size_t)j * nload * 3 + (s >> 1)];
        }
        rhs[(size_t)(i0 + j) * nrows + r] = v;
    }
}

// bbar = A_s^+ b per (instance, slot): slot k of device subsystem d = meta >> 8
// at position meta & 255.
__global__ void k_bbar(int i0, int cnt, int L, const int *meta, const int *sm, const int *boff,
                       const long long *pioff, const double *pinv, int nrows, const double *rhs,
                       double *bbar) {
    const long long n = (long long)cnt * L;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = i0 + (int)(t / L), k = (int)(t % L);
        const int d = meta[k] >> 8, cpos = meta[k] & 255, m = sm[d];
        const double *P = pinv + pioff[d] + (long long)cpos * m;
        const double *b = rhs + (size_t)in * nrows + boff[d];
        double acc = 0.0;
        for (int i = 0; i < m; ++i) acc += P[i] * b[i];
        bbar[(size_t)in * L + k] = acc;
    }
}

// Consistency of A_s x = b_s per instance: every rejected-row combination
// must annihilate b_s (relative to the largest |b| of the subsystem).
__global__ void k_bconsistent(int i0, int cnt, int S, const int *sm, const int *boff, const long long *toff,
                              const int *nrej, const double *Tw, int nrows, const double *rhs, int *bad) {
    const long long n = (long long)cnt * S;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = i0 + (int)(t / S), d = (int)(t % S);
        const int m = sm[d], nr = nrej[d];
        if (nr == 0) continue;
        const double *b = rhs + (size_t)in * nrows + boff[d];
        double bmax = 0.0;
        for (int i = 0; i < m; ++i) bmax = fmax(bmax, fabs(b[i]));
        const double *Tr = Tw + toff[d] + (long long)m * m;
        for (int q = 0; q < nr; ++q) {
            double acc = 0.0;
            for (int i = 0; i < m; ++i) acc += Tr[(long long)q * m + i] * b[i];
            if (!(fabs(acc) <= 1e-9 * (1.0 + bmax))) bad[in] = 1;
        }
    }
}

// ============================================================ re-centring
// Per (instance, global), instances still running: x_ref = clip((sum over the
// copies of rho x_s - lambda) - c) / (rho N)) in FP64 (the next global
// update), c~ = c + sum lambda_ref, bounds - x_ref, all in the engine layout.
// The change of variables is exact for any reference dual; at an unbounded
// global i it is lambda_ref_k = lambda_k - delta_i with delta_i = (c_i + sum
// over the copies of lambda) / N_i (FP64, kept in dref), which makes c~_i
// zero (up to rounding), and delta_i is itself small near a solution (the
// stationarity of Eq. closed_1 makes c_i + sum lambda = rho sum (x_k - x_i)).
// At a bounded global lambda_ref = lambda (delta = 0): there c~ is the bound's
// multiplier, which the clip of the global update removes, and a copy of it in
// every lambda~ would cost the FP32 iterations their small values.  c~ of the
// bounded globals also goes to cbt, in the layout of the bounds.
template <typename T>
__global__ void k_bref_globals(int n_inst, int G, int L, int K, int kshift, int NB, const int *ipos,
                               const int2 *gseg, const int *uslot, const int *bidx, const double *c64,
                               const double *lb, const double *ub, double rho, const double *xsv,
                               const double *lam, DevStatus *st, double *xref, double *dref, T *ct, T *xrf,
                               T *lbt, T *ubt, T *cbt) {
    const long long n = (long long)n_inst * G;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = (int)(t / G), i = (int)(t % G);
        if (st[in].done || ipos[in] < 0) continue;
        const int2 sg = gseg[i];
        const double *xi = xsv + (size_t)in * L, *li = lam + (size_t)in * L;
        double s = 0.0, ls = 0.0;
        for (int q = 0; q < sg.y; ++q) {
            const int k = uslot[sg.x + q];
            s += rho * xi[k] - li[k];
            ls += li[k];
        }
        double x = (s - c64[i]) / (rho * sg.y);
        x = fmin(fmax(x, lb[i]), ub[i]);
        xref[(size_t)in * G + i] = x;
        const int b = bidx[i];
        const double delta = b >= 0 ? 0.0 : (c64[i] + ls) / sg.y;
        dref[(size_t)in * G + i] = delta;
        const int pos = ipos[in], cc = pos >> kshift, sc = pos & (K - 1);
        const size_t e = ((size_t)cc * G + i) * K + sc;
        const double cs = c64[i] + (ls - sg.y * delta);
        ct[e] = (T)cs;
        xrf[e] = (T)x;
        if (b >= 0) {
            const size_t eb = ((size_t)cc * NB + b) * K + sc;
            lbt[eb] = (T)(lb[i] - x);
            ubt[eb] = (T)(ub[i] - x);
            cbt[eb] = (T)cs;
        }
        if (i == 0) st[in].pad = 1;     // shifted: unshift after the engine
    }
}

// Per (subsystem, instance), one warp: bbar~ = M (x_ref[g] + lambda_ref / rho)
// + bbar - x_ref[g], d = x_s - x_ref[g], mu = lambda - lambda_ref, lambda_ref,
// in the engine layout (lambda_ref = lambda - delta[g]).
// One subsystem of one instance by `nl` lanes starting at lane `l0` of the
// warp (v and t staged in v[], tt[]): the two FP64 products of the shifted
// bbar, written in the engine layout.
template <typename T>
__device__ __forceinline__ void bref_one(int in, bool valid, int d, int l0, int nl, int lane, const int4 h,
                                         const int4 q2, const double *F64, const int *ipos, const int *gk,
                                         const int *sch, double rho, const double *xref, const double *dref,
                                         const double *xsv, const double *lam, const double *bbar, int G, int L,
                                         int K, int kshift, int NCH, double *v, double *tt, T *bt, T *ds, T *mu,
                                         T *lref) {
    const int so = h.x, n = h.y, f = h.z, mode = h.w, npad = q2.y;
    const double *Fs = F64 + q2.x;
    const int ll = lane - l0;
    const double *xr = xref + (size_t)in * G, *dr = dref + (size_t)in * G;
    const double *xi = xsv + (size_t)in * L, *li = lam + (size_t)in * L, *bi = bbar + (size_t)in * L;
    if (valid)
        for (int r = ll; r < n; r += nl) v[r] = xr[gk[so + r]] + (li[so + r] - dr[gk[so + r]]) / rho;
    __syncwarp();
    if (valid)
        for (int cc = ll; cc < f; cc += nl) {
            double acc = 0.0;
            for (int r = 0; r < n; ++r) acc += Fs[(long long)cc * npad + r] * v[r];
            tt[cc] = acc;
        }
    __syncwarp();
    if (!valid) return;
    const int pos = ipos[in], cta = pos >> kshift, sc = pos & (K - 1);
    for (int r = ll; r < n; r += nl) {
        double yv = 0.0;
        for (int cc = 0; cc < f; ++cc) yv += Fs[(long long)cc * npad + r] * tt[cc];
        const double mv = mode ? yv : v[r] - yv;
        const int k = so + r;
        const double xg = xr[gk[k]];
        const int p = sch[k];
        const size_t e = (((size_t)cta * NCH + (p >> 2)) * K + sc) * 4 + (p & 3);
        const double btv = mv + bi[k] - xg;
        const double dg = dr[gk[k]];
        bt[e] = (T)(mode ? btv : -btv);      // the engine starts y at this value
        ds[e] = (T)(xi[k] - xg);
        mu[e] = (T)dg;
        lref[e] = (T)(li[k] - dg);
    }
}

// Per (subsystem, pair of instances), running instances only: bbar~ =
// M (x_ref[g] + lambda_ref / rho) + bbar - x_ref[g], d = x_s - x_ref[g],
// mu = 0, lambda_ref, in the engine layout.  A subsystem with at most 16
// slots and 16 factor columns takes a half-warp per instance (the FP64 pipe
// issues a warp instruction at the same cost however many lanes are active),
// a larger one the whole warp for each instance in turn.
template <typename T>
__global__ void __launch_bounds__(128) k_bref_slots(int S, int n_inst, int G, int L, int K, int kshift, int NCH,
                                                    const int *ipos, const int4 *sub, const int4 *sub2,
                                                    const double *F64, const int *gk, const int *sch,
                                                    double rho, const double *xref, const double *dref,
                                                    const double *xsv, const double *lam, const double *bbar,
                                                    const DevStatus *st, T *bt, T *ds, T *mu, T *lref) {
    __shared__ double buf[4][2][OPF_MAX_NS];
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long task = (long long)blockIdx.x * 4 + wl;
    const int npair = (n_inst + 1) / 2;
    if (task >= (long long)S * npair) return;
    const int pair = (int)(task / S), d = (int)(task % S);
    const int4 h = sub[d], q2 = sub2[d];
    if (h.y <= 16 && h.z <= 16) {
        const int half = lane >> 4, in = 2 * pair + half;
        const bool valid = in < n_inst && !st[in].done && ipos[in] >= 0;
        bref_one<T>(in, valid, d, half * 16, 16, lane, h, q2, F64, ipos, gk, sch, rho, xref, dref, xsv, lam, bbar,
                    G, L, K, kshift, NCH, buf[wl][0] + half * 128, buf[wl][1] + half * 128, bt, ds, mu, lref);
    } else {
        for (int q = 0; q < 2; ++q) {
            const int in = 2 * pair + q;
            if (in >= n_inst) break;
            const bool valid = !st[in].done && ipos[in] >= 0;
            bref_one<T>(in, valid, d, 0, 32, lane, h, q2, F64, ipos, gk, sch, rho, xref, dref, xsv, lam, bbar, G,
                        L, K, kshift, NCH, buf[wl][0], buf[wl][1], bt, ds, mu, lref);
            __syncwarp();
        }
    }
}

// Back to the unshifted FP64 state for instances that ran (status pad = 1):
// x_s = x_ref[g] + d, lambda = lambda_ref + mu = lambda - delta[g] + mu.
template <typename T>
__global__ void k_bunshift_slots(int n_inst, int G, int L, int K, int kshift, int NCH, const int *ipos,
                                 const int *gk, const int *sch, const double *xref, const double *dref,
                                 const T *ds, const T *mu, const DevStatus *st, double *xsv, double *lam) {
    const long long n = (long long)n_inst * L;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = (int)(t / L), k = (int)(t % L);
        if (!st[in].pad || ipos[in] < 0) continue;
        const int pos = ipos[in], cta = pos >> kshift, sc = pos & (K - 1);
        const int p = sch[k];
        const size_t e = (((size_t)cta * NCH + (p >> 2)) * K + sc) * 4 + (p & 3);
        const size_t gi = (size_t)in * G + gk[k];
        xsv[(size_t)in * L + k] = xref[gi] + (double)ds[e];
        lam[(size_t)in * L + k] = (lam[(size_t)in * L + k] - dref[gi]) + (double)mu[e];
    }
}

template <typename T>
__global__ void k_bunshift_globals(int n_inst, int G, int K, int kshift, const int *ipos, const double *xref,
                                   const T *xo, const DevStatus *st, double *x) {
    const long long n = (long long)n_inst * G;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int in = (int)(t / G), i = (int)(t % G);
        if (!st[in].pad || ipos[in] < 0) continue;
        const int pos = ipos[in], cta = pos >> kshift, sc = pos & (K - 1);
        x[(size_t)in * G + i] = xref[(size_t)in * G + i] + (double)xo[((size_t)cta * G + i) * K + sc];
    }
}

// Clears the shifted marks of the plan's instances (ipos >= 0); flag = 1
// while one of them still runs (and the graph condition, when a conditional
// node drives the loop).
__global__ void k_bany(int n_inst, const int *ipos, DevStatus *st, int *flag, cudaGraphConditionalHandle cond,
                       int use_cond) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int mine = 0;
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        if (ipos[i] < 0) continue;
        st[i].pad = 0;
        mine |= st[i].done ? 0 : 1;
    }
    if (mine) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        *flag = any;
        if (use_cond) cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
}

// Objective c^T x per instance (one warp each, fixed order).
__global__ void k_bobjective(int n_inst, int G, const double *c64, const double *x, double *obj) {
    const int wg = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (wg >= n_inst) return;
    double s = 0.0;
    for (int i = lane; i < G; i += 32) s += c64[i] * x[(size_t)wg * G + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) obj[wg] = s;
}

// Prepares the polish: instances that stopped without a numeric failure run again.
__global__ void k_brestart(int n_inst, DevStatus *st, long long add_max) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
        if (st[i].numeric) continue;
        st[i].done = 0;
        st[i].converged = 0;
        if (st[i].max_iter < st[i].iter + add_max) st[i].max_iter = st[i].iter + add_max;
    }
}

// Factors packed per task: element (r, q, jpos, e) of task t from the FP64
// factor of member mb = jpos >> lp (memb[t * J + mb], -1: none), slot
// c = ((jpos & (p-1)) * nq + q) * 4 + e.
template <typename T>
__global__ void k_bpack(int n_tasks, int J, const BatchTask *tasks, const int *memb, const int4 *sub,
                        const int4 *sub2, const double *F64, T *dst) {
    const int t = blockIdx.x;
    if (t >= n_tasks) return;
    const BatchTask tk = tasks[t];
    const int n = tk.f * tk.nq * J * 4;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const int e = x & 3, jpos = (x >> 2) % J, q = (x / (4 * J)) % tk.nq, r = x / (4 * J * tk.nq);
        const int mb = jpos >> tk.lp, part = jpos & (tk.p - 1);
        const int d = memb[t * J + mb];
        double v = 0.0;
        if (d >= 0) {
            const int4 h = sub[d], q2 = sub2[d];
            const int cpos = (part * tk.nq + q) * 4 + e;
            if (r < h.z && cpos < h.y) v = F64[q2.x + (long long)r * q2.y + cpos];
        }
        dst[tk.foff + x] = (T)v;
    }
}

// ============================================================ launchers
static inline int bl(long long n, int t) {
    long long b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

// Instantiated shapes: FP32 with factors in shared memory (K = 2, 4, 8; NQ = 4),
// lambda and bbar~ in tensor memory or streamed from L2; FP64 (NQ = 2,
// K = 1, 2, 4) with factors in shared or global memory.
template <typename T>
static const void *engine_fn(int K, int nq, bool fg, bool tm) {
    if constexpr (sizeof(T) == 4) {
        if (fg || nq != 4) return nullptr;
        if (K == 2) return tm ? (const void *)k_batch_engine<float, 2, 4, false, true>
                              : (const void *)k_batch_engine<float, 2, 4, false, false>;
        if (K == 4) return tm ? (const void *)k_batch_engine<float, 4, 4, false, true>
                              : (const void *)k_batch_engine<float, 4, 4, false, false>;
        if (K == 8) return tm ? (const void *)k_batch_engine<float, 8, 4, false, true>
                              : (const void *)k_batch_engine<float, 8, 4, false, false>;
    } else {
        if (nq != 2 || tm) return nullptr;
        if (K == 1) return fg ? (const void *)k_batch_engine<double, 1, 2, true, false> : (const void *)k_batch_engine<double, 1, 2, false, false>;
        if (K == 2) return fg ? (const void *)k_batch_engine<double, 2, 2, true, false> : (const void *)k_batch_engine<double, 2, 2, false, false>;
        if (K == 4) return fg ? (const void *)k_batch_engine<double, 4, 2, true, false> : (const void *)k_batch_engine<double, 4, 2, false, false>;
    }
    return nullptr;
}

template <typename T>
int batch_engine_prepare(int K, int nq, bool fg, bool tm, unsigned bytes) {
    const void *fn = engine_fn<T>(K, nq, fg, tm);
    if (!fn) return -1;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess ? 0 : -1;
}

template <typename T>
int batch_engine_launch(const BatchArgs<T> &a, int nq, bool fg, int ctas, int threads, unsigned bytes, int n_iters,
                        int check_every, cudaStream_t s) {
    const void *fn = engine_fn<T>(a.K, nq, fg, a.tm != 0);
    if (!fn) return -1;
    BatchArgs<T> aa = a;
    void *args[] = {(void *)&aa, (void *)&n_iters, (void *)&check_every};
    return cudaLaunchKernel(fn, dim3(ctas), dim3(threads), args, bytes, s) == cudaSuccess ? 0 : -1;
}

template <typename T>
int batch_engine_max_ctas_per_sm(int K, int nq, bool fg, bool tm, int threads, unsigned bytes) {
    const void *fn = engine_fn<T>(K, nq, fg, tm);
    if (!fn) return -1;
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, bytes) == cudaSuccess ? n : -1;
}

template int batch_engine_prepare<float>(int, int, bool, bool, unsigned);
template int batch_engine_prepare<double>(int, int, bool, bool, unsigned);
template int batch_engine_launch<float>(const BatchArgs<float> &, int, bool, int, int, unsigned, int, int,
                                        cudaStream_t);
template int batch_engine_launch<double>(const BatchArgs<double> &, int, bool, int, int, unsigned, int, int,
                                         cudaStream_t);
template int batch_engine_max_ctas_per_sm<float>(int, int, bool, bool, int, unsigned);
template int batch_engine_max_ctas_per_sm<double>(int, int, bool, bool, int, unsigned);

void launch_binit(int i0, int cnt, int L, const int *gk, const double *x0, double *xs, double *lam,
                  DevStatus *st, long long max_iter, double eps_rel, double eps_abs, cudaStream_t s) {
    k_binit<<<bl((long long)cnt * L, 256), 256, 0, s>>>(i0, cnt, L, gk, x0, xs, lam, st, max_iter, eps_rel, eps_abs);
}

void launch_bwarm(int i0, int cnt, int L, const double *xs0, const double *lam0, double *xs, double *lam,
                  cudaStream_t s) {
    k_bwarm<<<bl((long long)cnt * L, 256), 256, 0, s>>>(i0, cnt, L, xs0, lam0, xs, lam);
}

void launch_bfill(int cnt, int nrows, const double *b0, double *rhs, cudaStream_t s) {
    k_bfill<<<bl((long long)cnt * nrows, 256), 256, 0, s>>>(cnt, nrows, b0, rhs);
}

void launch_brhs_perm(int i0, int cnt, int nrows, const int *c2d, const double *src, double *rhs, cudaStream_t s) {
    k_brhs_perm<<<bl((long long)cnt * nrows, 256), 256, 0, s>>>(i0, cnt, nrows, c2d, src, rhs);
}

void launch_brhs_loads(int i0, int cnt, int nrows, int nload, const int *rsrc, const double *rcoef,
                       const double *b0, const double *lp, const double *lq, double *rhs, cudaStream_t s) {
    k_brhs_loads<<<bl((long long)cnt * nrows, 256), 256, 0, s>>>(i0, cnt, nrows, nload, rsrc, rcoef, b0, lp, lq, rhs);
}

void launch_bbar(int i0, int cnt, int L, const int *meta, const int *sm, const int *boff, const long long *pioff,
                 const double *pinv, int nrows, const double *rhs, double *bbar, cudaStream_t s) {
    k_bbar<<<bl((long long)cnt * L, 256), 256, 0, s>>>(i0, cnt, L, meta, sm, boff, pioff, pinv, nrows, rhs, bbar);
}

void launch_bconsistent(int i0, int cnt, int S, const int *sm, const int *boff, const long long *toff,
                        const int *nrej, const double *Tw, int nrows, const double *rhs, int *bad, cudaStream_t s) {
    k_bconsistent<<<bl((long long)cnt * S, 128), 128, 0, s>>>(i0, cnt, S, sm, boff, toff, nrej, Tw, nrows, rhs, bad);
}

template <typename T>
void launch_bref(int n_inst, int S, int G, int L, int K, int kshift, int NCH, int NB, const int *ipos,
                 const int2 *gseg, const int *uslot, const int *bidx, const double *c64, const double *lb,
                 const double *ub, double rho, const double *xsv, const double *lam, DevStatus *st,
                 double *xref, double *dref, T *ct, T *xrf, T *lbt, T *ubt, T *cbt, const int4 *sub,
                 const int4 *sub2, const double *F64, const int *gk, const int *sch, const double *bbar, T *bt,
                 T *ds, T *mu, T *lref, cudaStream_t s) {
    k_bref_globals<T><<<bl((long long)n_inst * G, 256), 256, 0, s>>>(n_inst, G, L, K, kshift, NB, ipos, gseg, uslot,
                                                                    bidx, c64, lb, ub, rho, xsv, lam, st, xref,
                                                                    dref, ct, xrf, lbt, ubt, cbt);
    const long long warps = (long long)S * ((n_inst + 1) / 2);
    k_bref_slots<T><<<(int)((warps + 3) / 4), 128, 0, s>>>(S, n_inst, G, L, K, kshift, NCH, ipos, sub, sub2, F64,
                                                           gk, sch, rho, xref, dref, xsv, lam, bbar, st, bt, ds, mu,
                                                           lref);
}

template <typename T>
void launch_bunshift(int n_inst, int G, int L, int K, int kshift, int NCH, const int *ipos, const int *gk,
                     const int *sch, const double *xref, const double *dref, const T *ds, const T *mu, const T *xo,
                     const DevStatus *st, double *xsv, double *lam, double *x, cudaStream_t s) {
    k_bunshift_slots<T><<<bl((long long)n_inst * L, 256), 256, 0, s>>>(n_inst, G, L, K, kshift, NCH, ipos, gk, sch,
                                                                      xref, dref, ds, mu, st, xsv, lam);
    k_bunshift_globals<T><<<bl((long long)n_inst * G, 256), 256, 0, s>>>(n_inst, G, K, kshift, ipos, xref, xo, st, x);
}

template void launch_bref<float>(int, int, int, int, int, int, int, int, const int *, const int2 *, const int *,
                                 const int *, const double *, const double *, const double *, double,
                                 const double *, const double *, DevStatus *, double *, double *, float *,
                                 float *, float *, float *, float *, const int4 *, const int4 *, const double *,
                                 const int *, const int *, const double *, float *, float *, float *, float *,
                                 cudaStream_t);
template void launch_bref<double>(int, int, int, int, int, int, int, int, const int *, const int2 *, const int *,
                                  const int *, const double *, const double *, const double *, double,
                                  const double *, const double *, DevStatus *, double *, double *, double *,
                                  double *, double *, double *, double *, const int4 *, const int4 *, const double *,
                                  const int *, const int *, const double *, double *, double *, double *,
                                  double *, cudaStream_t);
template void launch_bunshift<float>(int, int, int, int, int, int, const int *, const int *, const int *,
                                     const double *, const double *, const float *, const float *, const float *,
                                     const DevStatus *, double *, double *, double *, cudaStream_t);
template void launch_bunshift<double>(int, int, int, int, int, int, const int *, const int *, const int *,
                                      const double *, const double *, const double *, const double *,
                                      const double *, const DevStatus *, double *, double *, double *,
                                      cudaStream_t);

void launch_bany(int n_inst, const int *ipos, DevStatus *st, int *flag, cudaGraphConditionalHandle cond,
                 int use_cond, cudaStream_t s) {
    k_bany<<<1, 1024, 0, s>>>(n_inst, ipos, st, flag, cond, use_cond);
}

void launch_bobjective(int n_inst, int G, const double *c64, const double *x, double *obj, cudaStream_t s) {
    k_bobjective<<<bl((long long)n_inst * 32, 256), 256, 0, s>>>(n_inst, G, c64, x, obj);
}

void launch_brestart(int n_inst, DevStatus *st, long long add_max, cudaStream_t s) {
    k_brestart<<<bl(n_inst, 256), 256, 0, s>>>(n_inst, st, add_max);
}

template <typename T>
void launch_bpack(int n_tasks, int J, const BatchTask *tasks, const int *memb, const int4 *sub, const int4 *sub2,
                  const double *F64, T *dst, cudaStream_t s) {
    if (n_tasks > 0) k_bpack<T><<<n_tasks, 256, 0, s>>>(n_tasks, J, tasks, memb, sub, sub2, F64, dst);
}
template void launch_bpack<float>(int, int, const BatchTask *, const int *, const int4 *, const int4 *,
                                  const double *, float *, cudaStream_t);
template void launch_bpack<double>(int, int, const BatchTask *, const int *, const int4 *, const int4 *,
                                   const double *, double *, cudaStream_t);

}  // namespace opf
