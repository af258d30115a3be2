// Batched ADMM (Algorithm 1) with the instances in the lanes of a warp.
//
// Every instance of a batch shares the model, so the subsystem loops, the
// factor entries and every table index are the same for the 32 instances of
// a warp: a lane runs one instance and the warp's control flow, the factor
// reads (shared-memory broadcasts) and the index arithmetic are spent once
// for 32 instances.  A tile of 128 instances (lane quadrant q of the
// tensor memory = instances 32 q .. 32 q + 31) runs on a cluster of C CTAs;
// CTA r holds part r of the subsystems (a run of the subsystem graph in
// depth-first order) with, for its slots and all 128 instances:
//   lambda~ and bbar~       tensor memory (columns p and nslm + p),
//   u = rho x_s - lambda    shared memory U[p][128] (x of the slot's global
//                           between the global and the local update),
//   u of exchanged slots    shared memory X[2][row][128] (slots whose global
//                           has copies in other parts; double-buffered by
//                           iteration parity, read by those parts through
//                           distributed shared memory).
// Per iteration (the shifted FP32 frame of the batched engine):
//   G. per global of the part's slots and instance: Eq. closed_1 as a
//      fixed-order sum over all copies of u (own part: U, other parts: their
//      X), x written into the own copies' rows of U.  A global with copies in
//      several parts is computed by each of them, identically;
//   L. per subsystem (one warp, 32 instances): v = x + lambda / rho,
//      t = F^T v, x_s = M v + bbar~ (y = bt + F t; M = F F^T or I - F F^T),
//      lambda <- rho (v - x_s) (Eq. ADMM-3), u = rho x_s - lambda;
//   -- cluster barrier (split: the globals with all copies in the own part
//      are updated between its arrive and its wait) --
// and every check_every iterations the Sec. III-C sums per instance (FP32
// partials per thread, FP64 across warps and CTAs), the test by CTA 0 and
// the result broadcast to the cluster; finished instances freeze (their
// lambda goes back to the engine array, their lanes keep computing).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "opf_internal.h"
#include "test_rule.cuh"
#include "tmem.cuh"

namespace opf {

namespace {

namespace cg = cooperative_groups;

__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ void ld4cg(const float *p, float (&v)[4]) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4cg(float *p, const float (&v)[4]) {
    __stcg(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}

// Per-thread view of the launch: the tile's arrays at this thread's instance.
struct LaneCtx {
    int rank, inst;
    size_t gbase, bbase;        // [G][128] and [NB][128] arrays of the tile, + inst
    const float *rcs;
    float rho, inv_rho;
};

// G for global items [j0, j1) of the part (one instance per thread); x into
// the own copies' rows of U; test terms 2 and 5 (owner part only) into p2,
// p5; x~ to xo on test and last iterations of running instances.  GB items
// at a time, so that their L2 loads (c~, bounds) and the loads of their
// first SEGW copies are in flight together; further copies one by one.
__device__ __forceinline__ void lane_g(const LaneArgs &a, const LaneCtx &c, cg::cluster_group &cl, int j0, int j1,
                                       const int4 *gis, const int *cps, float *U, const float *Xin, bool check,
                                       bool wx, float &p2, float &p5) {
    constexpr int GB = 4, SEGW = 4;
    for (int jb = j0; jb < j1; jb += GB) {
        int4 gr[GB];
        float ctv[GB], lo[GB], hi[GB], s[GB];
#pragma unroll
        for (int e = 0; e < GB; ++e) {
            gr[e] = jb + e < j1 ? gis[jb + e] : make_int4(0, -1, 0, 0);
            ctv[e] = jb + e < j1 ? __ldcg(a.ct + c.gbase + (size_t)gr[e].x * kLaneInst) : 0.f;
            lo[e] = hi[e] = 0.f;
            if (gr[e].y >= 0) {
                lo[e] = __ldcg(a.lbt + c.bbase + (size_t)gr[e].y * kLaneInst);
                hi[e] = __ldcg(a.ubt + c.bbase + (size_t)gr[e].y * kLaneInst);
            }
        }
        float v[GB][SEGW];
#pragma unroll
        for (int e = 0; e < GB; ++e) {
            const int N = gr[e].w & 0xffff;
#pragma unroll
            for (int q = 0; q < SEGW; ++q) {
                v[e][q] = 0.f;
                if (q < N) {
                    const int cp = cps[gr[e].z + q];
                    const int r = cp >> 24, row = cp & 0xffffff;
                    const float *src = (r == c.rank) ? U : cl.map_shared_rank(Xin, r);
                    v[e][q] = src[row * kLaneInst + c.inst];
                }
            }
        }
#pragma unroll
        for (int e = 0; e < GB; ++e) {
            const int N = gr[e].w & 0xffff;
            s[e] = 0.f;
#pragma unroll
            for (int q = 0; q < SEGW; ++q)
                if (q < N) s[e] += v[e][q];
            for (int q = SEGW; q < N; ++q) {
                const int cp = cps[gr[e].z + q];
                const int r = cp >> 24, row = cp & 0xffffff;
                const float *src = (r == c.rank) ? U : cl.map_shared_rank(Xin, r);
                s[e] += src[row * kLaneInst + c.inst];
            }
        }
#pragma unroll
        for (int e = 0; e < GB; ++e) {
            const int N = gr[e].w & 0xffff;
            if (N == 0) continue;
            const int i = gr[e].x;
            float x = (s[e] - ctv[e]) * c.rcs[N];
            if (gr[e].y >= 0) x = x < lo[e] ? lo[e] : (x > hi[e] ? hi[e] : x);
            for (int q = 0; q < N; ++q) {
                const int cp = cps[gr[e].z + q];
                if ((cp >> 24) == c.rank) U[(cp & 0xffffff) * kLaneInst + c.inst] = x;
            }
            if ((gr[e].w >> 16) != 0) {
                if (check) {
                    const float xa = x + __ldcg(a.xrf + c.gbase + (size_t)i * kLaneInst);
                    p2 += (float)N * xa * xa;
                    p5 += __ldg(a.cost + i) * xa;
                }
                if (wx) a.xo[c.gbase + (size_t)i * kLaneInst] = x;
            }
        }
    }
}

// Test-iteration terms of one thread (its instance, its warp's subsystems).
struct LaneTerms {
    float f0, f1, f3, f4;
};

// L for one subsystem and this thread's instance.  sr = (first local slot p0,
// rows n, factor offset, mode | has-exchange-rows << 1 | F4 << 8); rows in
// blocks of 4 (p0 is a multiple of 4, so each block is one 4-column
// tensor-memory access and one engine-array chunk).
template <int F4>
__device__ __forceinline__ void lane_sub(const LaneArgs &a, const LaneCtx &c, const int4 sr, float *U, float *Xout,
                                         const int *uxm, const int *gkm, const float *Fs, unsigned tl, bool check,
                                         bool wds, bool act, float *ds_t, const float *lr_t, LaneTerms &tt) {
    constexpr int FW = 4 * F4;
    const int p0 = sr.x, n = sr.y;
    const float *F = Fs + sr.z;
    const bool mode1 = (sr.w & 1) != 0, hasx = (sr.w & 2) != 0;
    const float rho = c.rho, inv_rho = c.inv_rho;
    float t[FW];
#pragma unroll
    for (int k = 0; k < FW; ++k) t[k] = 0.f;
    // t = F^T v, v = x + lambda / rho
    for (int r = 0; r < n; r += 4) {
        float l4[4];
        tm_ld4(tl + (unsigned)(p0 + r), l4);
        tm_wait_ld();
        const float *ur = U + (p0 + r) * kLaneInst + c.inst;
        if (r + 4 <= n) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = fmaf(l4[e], inv_rho, ur[e * kLaneInst]);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 *Fr = reinterpret_cast<const float4 *>(F + (r + e) * FW);
#pragma unroll
                for (int q = 0; q < F4; ++q) {
                    const float4 f = Fr[q];
                    t[4 * q] = fmaf(f.x, v[e], t[4 * q]);
                    t[4 * q + 1] = fmaf(f.y, v[e], t[4 * q + 1]);
                    t[4 * q + 2] = fmaf(f.z, v[e], t[4 * q + 2]);
                    t[4 * q + 3] = fmaf(f.w, v[e], t[4 * q + 3]);
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                if (e >= n - r) break;
                const float v = fmaf(l4[e], inv_rho, ur[e * kLaneInst]);
                const float4 *Fr = reinterpret_cast<const float4 *>(F + (r + e) * FW);
#pragma unroll
                for (int q = 0; q < F4; ++q) {
                    const float4 f = Fr[q];
                    t[4 * q] = fmaf(f.x, v, t[4 * q]);
                    t[4 * q + 1] = fmaf(f.y, v, t[4 * q + 1]);
                    t[4 * q + 2] = fmaf(f.z, v, t[4 * q + 2]);
                    t[4 * q + 3] = fmaf(f.w, v, t[4 * q + 3]);
                }
            }
        }
    }
    // x_s = (y or v - y), y = bt + F t; dual update; u
    for (int r = 0; r < n; r += 4) {
        float l4[4], b4[4];
        tm_ld4(tl + (unsigned)(p0 + r), l4);
        tm_ld4(tl + (unsigned)(a.nslm + p0 + r), b4);
        tm_wait_ld();
        float *ur = U + (p0 + r) * kLaneInst + c.inst;
        const int ne = n - r < 4 ? n - r : 4;
        float m4[4] = {0.f, 0.f, 0.f, 0.f}, x4[4] = {0.f, 0.f, 0.f, 0.f}, xg[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e < ne) {
                const float x = ur[e * kLaneInst];
                const float v = fmaf(l4[e], inv_rho, x);
                const float4 *Fr = reinterpret_cast<const float4 *>(F + (r + e) * FW);
                float y0 = b4[e], y1 = 0.f;
#pragma unroll
                for (int q = 0; q < F4; ++q) {
                    const float4 f = Fr[q];
                    y0 = fmaf(f.x, t[4 * q], y0);
                    y1 = fmaf(f.y, t[4 * q + 1], y1);
                    y0 = fmaf(f.z, t[4 * q + 2], y0);
                    y1 = fmaf(f.w, t[4 * q + 3], y1);
                }
                const float y = y0 + y1;
                const float xs = mode1 ? y : v - y;
                const float mun = rho * (v - xs);
                const float u = fmaf(rho, xs, -mun);
                ur[e * kLaneInst] = u;
                if (hasx) {
                    const int ux = uxm[p0 + r + e];
                    if (ux >= 0) Xout[ux * kLaneInst + c.inst] = u;
                }
                m4[e] = mun;
                x4[e] = xs;
                xg[e] = x;
            }
        }
        tm_st4(tl + (unsigned)(p0 + r), m4);
        float *dsc = ds_t + (size_t)((p0 + r) >> 2) * (4 * kLaneInst);
        if (check) {
            float o4[4], lr4[4];
            ld4cg(dsc, o4);
            ld4cg(lr_t + (size_t)((p0 + r) >> 2) * (4 * kLaneInst), lr4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e < ne) {
                    const float d0 = xg[e] - x4[e], d1 = x4[e] - o4[e];
                    const float xa = x4[e] + __ldcg(a.xrf + c.gbase + (size_t)gkm[p0 + r + e] * kLaneInst);
                    const float la = m4[e] + lr4[e];
                    tt.f0 += d0 * d0;
                    tt.f1 += d1 * d1;
                    tt.f3 += xa * xa;
                    tt.f4 += la * la;
                }
            }
        }
        if (wds && act) st4cg(dsc, x4);
    }
}

// lane_sub for the subsystem's factor width (F4 <= kLaneMaxF4).
__device__ __forceinline__ void lane_sub_any(const LaneArgs &a, const LaneCtx &c, const int4 sr, float *U,
                                             float *Xout, const int *uxm, const int *gkm, const float *Fs,
                                             unsigned tl, bool check, bool wds, bool act, float *ds_t,
                                             const float *lr_t, LaneTerms &tt) {
    switch ((sr.w >> 8) & 15) {
        case 1: lane_sub<1>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
        case 2: lane_sub<2>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
        case 3: lane_sub<3>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
        case 4: lane_sub<4>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
        case 5: lane_sub<5>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
        default: lane_sub<6>(a, c, sr, U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt); break;
    }
}

// n_iters iterations of the tile blockIdx.x / C on its cluster.  Every
// decision that changes the cluster's barrier sequence (the early return,
// the stop) is taken on data all CTAs of the cluster see alike: the status
// read before the first cluster barrier, and the flags CTA 0 broadcasts.
__global__ void __launch_bounds__(512, 1) k_lane_engine(LaneArgs a, int n_iters, int check_every) {
    extern __shared__ __align__(16) unsigned char sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tile = blockIdx.x / a.C;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nthr = blockDim.x;
    const int q = w & 3, g = w >> 2, WG = a.WG;
    const int inst = q * 32 + lane;
    float *U = reinterpret_cast<float *>(sm + a.off_U);
    float *X = reinterpret_cast<float *>(sm + a.off_X);
    float *Fs = reinterpret_cast<float *>(sm + a.off_F);
    int4 *subs = reinterpret_cast<int4 *>(sm + a.off_sub);
    int4 *gis = reinterpret_cast<int4 *>(sm + a.off_gi);
    int *cps = reinterpret_cast<int *>(sm + a.off_cp);
    int *uxm = reinterpret_cast<int *>(sm + a.off_ux);
    int *gkm = reinterpret_cast<int *>(sm + a.off_gk);
    float *rcs = reinterpret_cast<float *>(sm + a.off_rc);
    double *red = reinterpret_cast<double *>(sm + a.off_red);     // [WG][6][128]
    double *part = reinterpret_cast<double *>(sm + a.off_part);   // [6][128]: this CTA's sums
    int *flags = reinterpret_cast<int *>(sm + a.off_flag);        // [0,128) running, [128,256) just finished
    __shared__ unsigned tm_base;
    __shared__ LanePart P;
    if (tid == 0) P = a.parts[rank];
    if (tid < kLaneInst) {
        const int in = a.inst[tile * kLaneInst + tid];
        flags[tid] = (in >= 0 && !a.st[in].done) ? 1 : 0;
        flags[kLaneInst + tid] = 0;
    }
    __syncthreads();
    {
        int any = 0;
        for (int k = 0; k < kLaneInst; ++k) any |= flags[k];
        if (!any) return;
    }
    for (int k = tid; k < P.nsub; k += nthr) subs[k] = a.sub[P.sub0 + k];
    for (int k = tid * 4; k < P.nF; k += nthr * 4)
        *reinterpret_cast<float4 *>(Fs + k) = __ldg(reinterpret_cast<const float4 *>(a.F + P.F0 + k));
    for (int k = tid; k < P.ng; k += nthr) gis[k] = a.gi[P.g0 + k];
    for (int k = tid; k < P.ncp; k += nthr) cps[k] = a.cp[P.cp0 + k];
    for (int k = tid; k < P.nslot; k += nthr) {
        uxm[k] = a.ux[4 * P.cb + k];
        gkm[k] = a.gk[4 * P.cb + k];
    }
    for (int k = tid; k < kBatchRecip; k += nthr) rcs[k] = __ldg(a.recip + k);
    if (w == 0) tm_alloc(&tm_base, a.tm_cols);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const unsigned tl = tm_base + ((unsigned)(32 * q) << 16);
    const size_t sbase = ((size_t)(tile * a.NCH + P.cb) * kLaneInst + inst) * 4;    // chunk 0 of the part
    float *mu_t = a.mu + sbase, *ds_t = a.ds + sbase;
    const float *bt_t = a.bt + sbase, *lr_t = a.lref + sbase;
    const float rho = a.rho, inv_rho = a.inv_rho;
    // lambda~ and bbar~ into tensor memory; u = rho d - mu into U and X[0]
    for (int ch = g; ch < (P.nslot >> 2); ch += WG) {
        float m[4], bb[4], d[4];
        ld4cg(mu_t + (size_t)ch * 4 * kLaneInst, m);
        ld4cg(bt_t + (size_t)ch * 4 * kLaneInst, bb);
        ld4cg(ds_t + (size_t)ch * 4 * kLaneInst, d);
        tm_st4(tl + (unsigned)(4 * ch), m);
        tm_st4(tl + (unsigned)(a.nslm + 4 * ch), bb);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float u = fmaf(rho, d[e], -m[e]);
            U[(4 * ch + e) * kLaneInst + inst] = u;
            const int ux = uxm[4 * ch + e];
            if (ux >= 0) X[ux * kLaneInst + inst] = u;
        }
    }
    tm_wait_st();
    tm_fence_before();
    cl.sync();
    tm_fence_after();
    LaneCtx c;
    c.rank = rank;
    c.inst = inst;
    c.gbase = (size_t)tile * a.G * kLaneInst + inst;
    c.bbase = (size_t)tile * a.NB * kLaneInst + inst;
    c.rcs = rcs;
    c.rho = rho;
    c.inv_rho = inv_rho;
    const size_t xstride = (size_t)a.maxux * kLaneInst;
    int last_check = 0;
    bool all_done = false, pre = false;
    float p2 = 0.f, p5 = 0.f;
    for (int it = 0; it < n_iters; ++it) {
        const bool check = check_every > 0 && ((it + 1) % check_every == 0);
        const bool last = it == n_iters - 1;
        const bool wds = check || last || (check_every > 0 && ((it + 2) % check_every == 0));
        const bool act = flags[inst] != 0;
        const float *Xin = X + (size_t)(it & 1) * xstride;
        float *Xout = X + (size_t)((it + 1) & 1) * xstride;
        // G (the part's own globals ran during the last barrier unless pre is false)
        if (!pre) {
            p2 = p5 = 0.f;
            lane_g(a, c, cl, P.gint[g], P.gint[g + 1], gis, cps, U, Xin, check, (check || last) && act, p2, p5);
        }
        lane_g(a, c, cl, P.gcut[g], P.gcut[g + 1], gis, cps, U, Xin, check, (check || last) && act, p2, p5);
        __syncthreads();
        tm_fence_after();
        // L
        LaneTerms tt = {0.f, 0.f, 0.f, 0.f};
        for (int k = P.gsub[g]; k < P.gsub[g + 1]; ++k)
            lane_sub_any(a, c, subs[k], U, Xout, uxm, gkm, Fs, tl, check, wds, act, ds_t, lr_t, tt);
        if (check) {
            double *rw = red + (size_t)g * 6 * kLaneInst + inst;
            rw[0 * kLaneInst] = (double)tt.f0;
            rw[1 * kLaneInst] = (double)tt.f1;
            rw[2 * kLaneInst] = (double)p2;
            rw[3 * kLaneInst] = (double)tt.f3;
            rw[4 * kLaneInst] = (double)tt.f4;
            rw[5 * kLaneInst] = (double)p5;
        }
        tm_wait_st();
        tm_fence_before();
        __syncthreads();
        if (check) {
            // this CTA's sums per (quantity, instance) over the item groups in
            // order; CTA 0 adds the CTAs' sums in rank order and tests
            for (int idx = tid; idx < 6 * kLaneInst; idx += nthr) {
                double s = 0.0;
                for (int gg = 0; gg < WG; ++gg) s += red[(size_t)gg * 6 * kLaneInst + idx];
                part[idx] = s;
            }
            cl_arrive();
            cl_wait();
            if (rank == 0 && tid < kLaneInst) {
                int run = flags[tid], fin = 0;
                if (run) {
                    double s6[6];
#pragma unroll
                    for (int qq = 0; qq < 6; ++qq) s6[qq] = 0.0;
                    for (int r = 0; r < a.C; ++r) {
                        const double *pr = cl.map_shared_rank(part, r);
#pragma unroll
                        for (int qq = 0; qq < 6; ++qq) s6[qq] += pr[qq * kLaneInst + tid];
                    }
                    DevStatus *st = a.st + a.inst[tile * kLaneInst + tid];
                    apply_test(st, s6, a.rho_d, check_every);
                    if (st->done) {
                        run = 0;
                        fin = 1;
                    }
                }
                for (int r = 0; r < a.C; ++r) {
                    int *fr = cl.map_shared_rank(flags, r);
                    fr[tid] = run;
                    fr[kLaneInst + tid] = fin;
                }
            }
            cl_arrive();
            cl_wait();
            tm_fence_after();
            last_check = it + 1;
            int anyfin = 0, anyrun = 0;
            for (int k = 0; k < kLaneInst; ++k) {
                anyfin |= flags[kLaneInst + k];
                anyrun |= flags[k];
            }
            if (anyfin) {
                // lambda of the instances that just finished, to the engine array
                const bool wr = flags[kLaneInst + inst] != 0;
                for (int ch = g; ch < (P.nslot >> 2); ch += WG) {
                    float m[4];
                    tm_ld4(tl + (unsigned)(4 * ch), m);
                    tm_wait_ld();
                    if (wr) st4cg(mu_t + (size_t)ch * 4 * kLaneInst, m);
                }
                tm_fence_before();
            }
            pre = false;
            if (!anyrun) {
                all_done = true;
                break;
            }
        } else if (!last) {
            // split barrier: the own globals of the next iteration meanwhile
            cl_arrive();
            const bool check1 = check_every > 0 && ((it + 2) % check_every == 0);
            const bool last1 = it + 1 == n_iters - 1;
            p2 = p5 = 0.f;
            lane_g(a, c, cl, P.gint[g], P.gint[g + 1], gis, cps, U, Xout, check1, (check1 || last1) && act, p2,
                   p5);
            pre = true;
            cl_wait();
            tm_fence_after();
        }
    }
    if (!all_done && rank == 0 && tid < kLaneInst && flags[tid])
        a.st[a.inst[tile * kLaneInst + tid]].iter += n_iters - last_check;
    // lambda of the instances still running, then the allocation is freed
    if (!all_done) {
        tm_fence_after();
        const bool wr = flags[inst] != 0;
        for (int ch = g; ch < (P.nslot >> 2); ch += WG) {
            float m[4];
            tm_ld4(tl + (unsigned)(4 * ch), m);
            tm_wait_ld();
            if (wr) st4cg(mu_t + (size_t)ch * 4 * kLaneInst, m);
        }
    }
    tm_fence_before();
    cl.sync();        // no CTA leaves while another may read its shared memory
    tm_fence_after();
    if (w == 0) tm_dealloc(tm_base, a.tm_cols);
}

}  // namespace

namespace {

// Factors of the lane engine: record t = (device subsystem d, first float,
// F4) gets rows k < n of 4 F4 floats, F[k][c] = c-th factor vector at slot k
// (zero for c >= f).
__global__ void k_lpack(int nrec, const int4 *desc, const int4 *sub, const int4 *sub2, const double *F64,
                        float *dst) {
    const int t = blockIdx.x;
    if (t >= nrec) return;
    const int4 ds = desc[t];
    const int4 h = sub[ds.x], q2 = sub2[ds.x];
    const int FW = 4 * ds.z, n = h.y, f = h.z;
    for (int x = threadIdx.x; x < n * FW; x += blockDim.x) {
        const int k = x / FW, cc = x - k * FW;
        dst[ds.y + x] = cc < f ? (float)F64[q2.x + (long long)cc * q2.y + k] : 0.f;
    }
}

}  // namespace

int lane_engine_prepare(int C, unsigned bytes) {
    if (cudaFuncSetAttribute(k_lane_engine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return -1;
    if (C > 8 && cudaFuncSetAttribute(k_lane_engine, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                     cudaSuccess)
        return -1;
    return 0;
}

static void lane_config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr, int tiles, int C, int threads,
                        unsigned bytes, cudaStream_t s) {
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(tiles * C), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

// Clusters of C CTAs of this shape that the device holds at once (0: none).
int lane_engine_max_clusters(int C, int threads, unsigned bytes) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    lane_config(cfg, attr, 1, C, threads, bytes, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_lane_engine, &cfg) != cudaSuccess) return 0;
    return n;
}

// CTAs of this shape one SM holds (0: none).
int lane_engine_ctas_per_sm(int threads, unsigned bytes) {
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_lane_engine, threads, bytes) != cudaSuccess) return 0;
    return m;
}

int lane_engine_launch(const LaneArgs &a, int tiles, int threads, unsigned bytes, int n_iters, int check_every,
                       cudaStream_t s) {
    if (tiles < 1) return 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    lane_config(cfg, attr, tiles, a.C, threads, bytes, s);
    return cudaLaunchKernelEx(&cfg, k_lane_engine, a, n_iters, check_every) == cudaSuccess ? 0 : -1;
}

void launch_lpack(int nrec, const int4 *desc, const int4 *sub, const int4 *sub2, const double *F64, float *dst,
                  cudaStream_t s) {
    if (nrec > 0) k_lpack<<<nrec, 128, 0, s>>>(nrec, desc, sub, sub2, F64, dst);
}

}  // namespace opf
