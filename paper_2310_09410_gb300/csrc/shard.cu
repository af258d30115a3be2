// Sharded single instance (C ABI opf_partition, opf_shard_*): the
// subsystems of one feeder split over several GPUs by subtree, the exchange
// of Algorithm 1's global update reduced to the globals whose copies lie on
// more than one shard (the cut).
//
// Partition: the buses in depth-first order from the substation, cut into
// contiguous ranges of balanced work (sum of n_s^2 of the subsystems anchored
// at a bus: a bus subsystem at its bus, a line subsystem, merged leaf
// included, at its to-bus), so a part is a run of whole subtrees and the cut
// is the handful of lines between runs.
//
// Shard: the part's subsystems as an instance of their own (a handle over
// the globals they touch, in ascending global order).  One FP64 iteration:
//   1. opf_shard_partial: per cut global i, the local part of
//      sigma_i = sum over copies of (rho x_k - lambda_k) (Eq. closed_1);
//   2. the caller adds the parts over all shards (an all-reduce over the cut);
//   3. opf_shard_step: the global update of Eq. closed_1 with the summed sigma
//      and the total copy count for cut globals (the local ones as in one
//      instance), then the local update (Eq. closed_2) and the dual update
//      (Eq. ADMM-3) of the shard's subsystems; on tested iterations the
//      shard's part of the Sec. III-C sums (the objective counted by the
//      owner of each global only), which the caller adds over the shards
//      before the test (opf_test_rule).
// The iterates equal those of the whole instance: every shard computes the
// same x_i for a cut global from the same sigma_i and N_i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "handle.h"
#include "opf_internal.h"

namespace opf {
template <typename T>
void launch_make_u(int L, const int *pk, const T *ds, const T *mu, T rho, T *u, const DevStatus *st,
                   cudaStream_t s);
}

using namespace opf;

struct opf_shard {
    opf_handle *h = nullptr;
    int part = 0, n_parts = 0;
    int G = 0, n_cut = 0, n_tiles = 0;
    std::vector<int> global_of_local;     // local global -> global index of the whole instance
    std::vector<int> cut_global;          // cut j -> global index (the cut of all shards, ascending)
    std::vector<int> cut_local;           // cut j -> local global on this shard, or -1
    int *d_cutj = nullptr;                // per local global: cut index or -1
    double *d_ntot = nullptr;             // per local global: copies over all shards
    unsigned char *d_own = nullptr;       // per local global: 1 if this shard counts it in the objective
    int *d_cut_local = nullptr;
    double *d_x = nullptr;                // x per local global after the last step
    double *d_part = nullptr;             // per tile: 6 partial sums (n_tiles known after the precompute)
    int part_cap = 0;                     // tiles d_part holds
    int parity = 0;                       // u of the last iteration at d_u64 + parity * L
    bool started = false;
    double rho = -1.0;
};

namespace {

// This shard's part of sigma for every cut global from u of the last
// iteration (0 for cut globals it holds no copy of).
__global__ void k_shard_partial(int n_cut, const int *cut_local, const int2 *gseg, const double *u, double *sig) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_cut) return;
    const int l = cut_local[j];
    double s = 0.0;
    if (l >= 0) {
        const int2 sg = gseg[l];
        for (int q = 0; q < sg.y; ++q) s += u[sg.x + q];
    }
    sig[j] = s;
}

// One FP64 iteration of the shard's tiles (the whole-grid engine's three
// phases with the cut globals' sigma and copy count from all shards).
template <bool CHECK>
__global__ void __launch_bounds__(256) k_shard_iter(IterArgs<double> a, const double *__restrict__ u_in,
                                                    double *__restrict__ u_out, const int *cutj,
                                                    const double *ntot, const unsigned char *own,
                                                    const double *sig_tot, double *xg, double *partials,
                                                    int xcap, int vcap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *vb = reinterpret_cast<double *>(smem_raw);
    double *xb = vb + vcap;
    double *tb = xb + xcap;
    const int s0 = a.tile_s0[blockIdx.x], s1 = a.tile_s0[blockIdx.x + 1];
    const int4 h0 = a.sub[s0], h1 = a.sub[s1];
    const int4 q0 = a.sub2[s0];
    const int k0 = h0.x, k1 = h1.x;
    const int v0 = q0.z, j0 = q0.w, j1 = a.sub2[s1].w;
    // phase 0: global update per slot, v = x + lambda / rho
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
        const int mt = a.meta[k];
        const int s = mt >> 8, r = mt & 255;
        const int sp = a.segp[k];
        const int us = sp >> 8, cnt = sp & 255;
        const int g = a.gk[k];
        const int j = cutj[g];
        double sigma = 0.0, n = (double)cnt;
        if (j >= 0) {
            sigma = sig_tot[j];
            n = ntot[g];
        } else {
            for (int q = 0; q < cnt; ++q) sigma += u_in[us + q];
        }
        double x = (sigma - a.ct[g]) / (a.rho * n);
        if (x < a.lbt[g]) x = a.lbt[g];
        if (x > a.ubt[g]) x = a.ubt[g];
        xb[k - k0] = x;
        if (a.pk[k] == us) xg[g] = x;
        const int4 q2 = a.sub2[s];
        double *vs = vb + (q2.z - v0);
        vs[r] = x + a.mu[k] * a.inv_rho;
        if (r == 0)
            for (int p = a.sub[s].y; p < q2.y; ++p) vs[p] = 0.0;
    }
    __syncthreads();
    // phase 1: t = F^T v per factor column
    for (int jj = j0 + (int)threadIdx.x; jj < j1; jj += blockDim.x) {
        const int it = a.items[jj];
        const int s = it >> 8, c = it & 255;
        const int4 q2 = a.sub2[s];
        const double *f = a.F + q2.x + (long long)c * q2.y;
        const double *v = vb + (q2.z - v0);
        double acc = 0.0;
        for (int r = 0; r < q2.y; ++r) acc = fma(f[r], v[r], acc);
        tb[q2.w - j0 + c] = acc;
    }
    __syncthreads();
    // phase 2: local update, dual update, u; the test sums
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
        const int mt = a.meta[k];
        const int s = mt >> 8, r = mt & 255;
        const int4 h = a.sub[s];
        const int4 q2 = a.sub2[s];
        const double *Fr = a.F + q2.x + r;
        const double *tt = tb + (q2.w - j0);
        double y = 0.0;
        for (int c = 0; c < h.z; ++c) y = fma(Fr[(long long)c * q2.y], tt[c], y);
        const double v = vb[q2.z - v0 + r];
        const double x = xb[k - k0];
        const double xm = (h.w ? y : v - y) + a.bt[k];
        const double res = x - xm;
        const double mu_new = a.mu[k] + a.rho * res;
        const double d_old = a.ds[k];
        a.mu[k] = mu_new;
        a.ds[k] = xm;
        const int pos = a.pk[k];
        u_out[pos] = a.rho * xm - mu_new;
        if (CHECK) {
            const int g = a.gk[k];
            const double dd = xm - d_old;
            acc[0] += res * res;
            acc[1] += dd * dd;
            acc[2] += x * x;
            acc[3] += xm * xm;
            acc[4] += mu_new * mu_new;
            if (pos == (a.segp[k] >> 8) && own[g]) acc[5] += a.c64[g] * x;
        }
    }
    if (CHECK) {
        __shared__ double red[8][6];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int q = 0; q < 6; ++q)
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
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
            for (int q = 0; q < 6; ++q) partials[blockIdx.x * 6 + q] = t[q];
        }
    }
}

// The tiles' partial sums in tile order (fixed, deterministic).
__global__ void k_shard_sum(int n_tiles, const double *partials, double *sums) {
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int b = 0; b < n_tiles; ++b) s += partials[b * 6 + threadIdx.x];
        sums[threadIdx.x] = s;
    }
}

int fail(int code, const std::string &msg) {
    set_last_error(msg);
    return code;
}

#define SH_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));        \
            return e_ == cudaErrorMemoryAllocation ? OPF_E_OOM : OPF_E_CUDA;           \
        }                                                                              \
    } while (0)

// Anchor bus of each subsystem in canonical order: the non-leaf buses in bus
// order (bus subsystems), then every line's to-bus (line subsystems, a leaf
// bus merged into its line).
std::vector<int> subsystem_anchors(const opf_feeder *f) {
    const int nb = f->n_bus, nl = f->n_line;
    std::vector<char> has_child(nb, 0);
    for (int e = 0; e < nl; ++e) has_child[f->line_from[e]] = 1;
    std::vector<int> anchor;
    for (int i = 0; i < nb; ++i)
        if (i == 0 || has_child[i]) anchor.push_back(i);
    for (int e = 0; e < nl; ++e) anchor.push_back(f->line_to[e]);
    return anchor;
}

}  // namespace

extern "C" {

int opf_partition(const opf_feeder *f, int32_t n_parts, int32_t *sub_part, int32_t n_sub) {
    if (!f || !sub_part || n_parts < 1) return fail(OPF_E_INVALID, "partition: need a feeder, n_parts >= 1");
    HostModel M;
    std::string err;
    int rc = build_feeder_model(f, &M, &err);
    if (rc != OPF_OK) return fail(rc, "partition: " + err);
    const int S = (int)M.subs.size();
    if (n_sub != S) return fail(OPF_E_INVALID, "partition: sub_part needs " + std::to_string(S) + " entries");
    const std::vector<int> anchor = subsystem_anchors(f);
    if ((int)anchor.size() != S) return fail(OPF_E_INVALID, "partition: subsystem count does not match the feeder");
    const int nb = f->n_bus;
    std::vector<double> work(nb, 0.0);
    for (int s = 0; s < S; ++s) work[anchor[s]] += (double)M.subs[s].n * M.subs[s].n;
    // depth-first order from the substation (children in line order)
    std::vector<std::vector<int>> child(nb);
    for (int e = 0; e < f->n_line; ++e) child[f->line_from[e]].push_back(f->line_to[e]);
    std::vector<int> order, stack = {0};
    while (!stack.empty()) {
        const int i = stack.back();
        stack.pop_back();
        order.push_back(i);
        for (int q = (int)child[i].size() - 1; q >= 0; --q) stack.push_back(child[i][q]);
    }
    double total = 0.0;
    for (double w : work) total += w;
    std::vector<int> bus_part(nb, 0);
    double run = 0.0;
    int p = 0;
    for (int i : order) {
        // the range of part p ends where its share of the work is reached
        if (p < n_parts - 1 && run >= total * (p + 1) / n_parts) ++p;
        bus_part[i] = p;
        run += work[i];
    }
    for (int s = 0; s < S; ++s) sub_part[s] = bus_part[anchor[s]];
    return OPF_OK;
}

int opf_shard_create(const opf_feeder *f, const int32_t *sub_part, int32_t n_sub, int32_t part,
                     const opf_options *o, opf_shard **out) {
    if (!f || !sub_part || !out || part < 0) return fail(OPF_E_INVALID, "shard: bad arguments");
    *out = nullptr;
    HostModel M;
    std::string err;
    int rc = build_feeder_model(f, &M, &err);
    if (rc != OPF_OK) return fail(rc, "shard: " + err);
    const int S = (int)M.subs.size(), Gall = M.n;
    if (n_sub != S) return fail(OPF_E_INVALID, "shard: sub_part needs " + std::to_string(S) + " entries");
    int n_parts = 0;
    for (int s = 0; s < S; ++s) {
        if (sub_part[s] < 0) return fail(OPF_E_INVALID, "shard: negative part");
        n_parts = std::max(n_parts, sub_part[s] + 1);
    }
    if (part >= n_parts) return fail(OPF_E_INVALID, "shard: no subsystem in this part");
    // copies per global over all parts and on this part; owner = lowest part
    std::vector<int> ntot(Gall, 0), nloc(Gall, 0), owner(Gall, n_parts);
    for (int s = 0; s < S; ++s)
        for (int g : M.subs[s].vars) {
            ++ntot[g];
            if (sub_part[s] == part) ++nloc[g];
            owner[g] = std::min(owner[g], (int)sub_part[s]);
        }
    std::vector<int> loc(Gall, -1);
    opf_shard *sh = new opf_shard();
    sh->part = part;
    sh->n_parts = n_parts;
    for (int g = 0; g < Gall; ++g)
        if (nloc[g] > 0) {
            loc[g] = (int)sh->global_of_local.size();
            sh->global_of_local.push_back(g);
        }
    const int G = (int)sh->global_of_local.size();
    sh->G = G;
    // the part's subsystems over its globals (ascending global order is kept)
    std::vector<double> c(G), lb(G), ub(G), A, b;
    std::vector<uint8_t> volt(G);
    std::vector<int> ms, ns, idx;
    for (int l = 0; l < G; ++l) {
        const int g = sh->global_of_local[l];
        c[l] = M.c[g]; lb[l] = M.lb[g]; ub[l] = M.ub[g]; volt[l] = M.volt[g];
    }
    for (int s = 0; s < S; ++s) {
        if (sub_part[s] != part) continue;
        const HostSub &hs = M.subs[s];
        ms.push_back(hs.m);
        ns.push_back(hs.n);
        A.insert(A.end(), hs.A.begin(), hs.A.end());
        b.insert(b.end(), hs.b.begin(), hs.b.end());
        for (int g : hs.vars) idx.push_back(loc[g]);
    }
    if (ms.empty()) { delete sh; return fail(OPF_E_INVALID, "shard: no subsystem in this part"); }
    rc = opf_create_generic(G, c.data(), lb.data(), ub.data(), volt.data(), (int)ms.size(), ms.data(), ns.data(),
                            A.data(), b.data(), idx.data(), o, &sh->h);
    if (rc != OPF_OK) { delete sh; return rc; }
    // the cut: globals with copies on more than one part, ascending (the same
    // list and order on every shard)
    std::vector<int> first_part(Gall, -1);
    std::vector<char> multi(Gall, 0);
    for (int s = 0; s < S; ++s)
        for (int g : M.subs[s].vars) {
            if (first_part[g] < 0) first_part[g] = sub_part[s];
            else if (first_part[g] != sub_part[s]) multi[g] = 1;
        }
    std::vector<int> cutj(G, -1);
    std::vector<double> nt(G);
    std::vector<unsigned char> own(G);
    for (int g = 0; g < Gall; ++g)
        if (multi[g]) {
            if (loc[g] >= 0) cutj[loc[g]] = (int)sh->cut_global.size();
            sh->cut_global.push_back(g);
            sh->cut_local.push_back(loc[g]);
        }
    for (int l = 0; l < G; ++l) {
        const int g = sh->global_of_local[l];
        nt[l] = (double)ntot[g];
        own[l] = owner[g] == part ? 1 : 0;
    }
    sh->n_cut = (int)sh->cut_local.size();
    opf_handle *h = sh->h;
    auto up = [&](auto **dst, const auto &v) -> int {
        using E = typename std::decay<decltype(v[0])>::type;
        void *p = nullptr;
        const size_t n = std::max<size_t>(v.size(), 1);
        if (cudaMalloc(&p, n * sizeof(E)) != cudaSuccess) { cudaGetLastError(); return OPF_E_OOM; }
        h->allocs.push_back(p);
        if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(E), cudaMemcpyHostToDevice) != cudaSuccess)
            return OPF_E_CUDA;
        *dst = reinterpret_cast<std::remove_reference_t<decltype(**dst)> *>(p);
        return OPF_OK;
    };
    std::vector<double> zx(G, 0.0);
    if ((rc = up(&sh->d_cutj, cutj)) || (rc = up(&sh->d_ntot, nt)) || (rc = up(&sh->d_own, own)) ||
        (rc = up(&sh->d_cut_local, sh->cut_local)) || (rc = up(&sh->d_x, zx))) {
        opf_shard_destroy(sh);
        return fail(rc, "shard: device allocation");
    }
    *out = sh;
    return OPF_OK;
}

int opf_shard_precompute(opf_shard *sh) {
    if (!sh) return OPF_E_INVALID;
    const int rc = opf_precompute(sh->h);
    sh->started = false;
    if (rc != OPF_OK) return rc;
    // the tiling of the shard's subsystems exists from here on: room for the
    // per-tile test sums
    opf_handle *h = sh->h;
    sh->n_tiles = h->t64.n_tiles;
    if (sh->n_tiles > sh->part_cap) {
        if (sh->d_part) cudaFree(sh->d_part);
        sh->d_part = nullptr;
        sh->part_cap = 0;
        SH_CUDA(cudaMalloc(&sh->d_part, (size_t)sh->n_tiles * 6 * sizeof(double)));
        sh->part_cap = sh->n_tiles;
    }
    return OPF_OK;
}

int opf_shard_sizes(opf_shard *sh, int32_t *n_global, int32_t *n_cut, int32_t *n_slots) {
    if (!sh) return OPF_E_INVALID;
    if (n_global) *n_global = sh->G;
    if (n_cut) *n_cut = sh->n_cut;
    if (n_slots) *n_slots = sh->h->L;
    return OPF_OK;
}

int opf_shard_maps(opf_shard *sh, int32_t *global_of_local, int32_t *cut_global) {
    if (!sh) return OPF_E_INVALID;
    for (int l = 0; l < sh->G; ++l)
        if (global_of_local) global_of_local[l] = sh->global_of_local[l];
    for (int j = 0; j < sh->n_cut; ++j)
        if (cut_global) cut_global[j] = sh->cut_global[j];
    return OPF_OK;
}

int opf_shard_partial(opf_shard *sh, double rho, double *sig) {
    if (!sh || !(rho > 0) || (!sig && sh->n_cut)) return OPF_E_INVALID;
    opf_handle *h = sh->h;
    if (!h->precomputed) return OPF_E_STATE;
    SH_CUDA(cudaSetDevice(h->device));
    if (!sh->started || sh->rho != rho) {
        // u = rho x_s - lambda of the current state (the start point after a precompute)
        launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64 + (size_t)sh->parity * h->L,
                              nullptr, h->stream);
        sh->started = true;
        sh->rho = rho;
    }
    if (sh->n_cut)
        k_shard_partial<<<(sh->n_cut + 255) / 256, 256, 0, h->stream>>>(
            sh->n_cut, sh->d_cut_local, h->d_gseg, h->d_u64 + (size_t)sh->parity * h->L, sig);
    SH_CUDA(cudaGetLastError());
    return OPF_OK;
}

int opf_shard_step(opf_shard *sh, double rho, const double *sig_tot, double *sums) {
    if (!sh || !(rho > 0) || (!sig_tot && sh->n_cut)) return OPF_E_INVALID;
    opf_handle *h = sh->h;
    if (!h->precomputed || !sh->started || sh->rho != rho || h->t64.n_tiles > sh->part_cap) {
        set_last_error("shard: call opf_shard_precompute, then opf_shard_partial with the same rho before each step");
        return OPF_E_STATE;
    }
    SH_CUDA(cudaSetDevice(h->device));
    IterArgs<double> a;
    memset(&a, 0, sizeof(a));
    a.sub = h->d_sub; a.sub2 = h->d_sub2; a.items = h->d_items;
    a.meta = h->d_meta; a.segp = h->d_segp; a.gk = h->d_gk; a.pk = h->d_pk;
    a.c64 = h->d_c64;
    a.F = h->d_F64; a.bt = h->d_bbar64; a.mu = h->d_mu64; a.ds = h->d_ds64;
    a.ct = h->d_c64; a.lbt = h->d_lb64; a.ubt = h->d_ub64;
    a.tile_s0 = h->t64.d_s0;
    a.rho = rho; a.inv_rho = 1.0 / rho;
    const Tiling &t = h->t64;
    const size_t shm = ((size_t)t.xcap + t.vcap + t.tcap) * sizeof(double);
    const double *u_in = h->d_u64 + (size_t)sh->parity * h->L;
    double *u_out = h->d_u64 + (size_t)(1 - sh->parity) * h->L;
    if (sums)
        k_shard_iter<true><<<t.n_tiles, t.block, shm, h->stream>>>(a, u_in, u_out, sh->d_cutj, sh->d_ntot,
                                                                   sh->d_own, sig_tot, sh->d_x, sh->d_part,
                                                                   t.xcap, t.vcap);
    else
        k_shard_iter<false><<<t.n_tiles, t.block, shm, h->stream>>>(a, u_in, u_out, sh->d_cutj, sh->d_ntot,
                                                                    sh->d_own, sig_tot, sh->d_x, sh->d_part,
                                                                    t.xcap, t.vcap);
    if (sums) k_shard_sum<<<1, 32, 0, h->stream>>>(t.n_tiles, sh->d_part, sums);
    SH_CUDA(cudaGetLastError());
    sh->parity ^= 1;
    return OPF_OK;
}

int opf_shard_get_x(opf_shard *sh, double *x) {
    if (!sh || !x) return OPF_E_INVALID;
    SH_CUDA(cudaSetDevice(sh->h->device));
    SH_CUDA(cudaMemcpyAsync(x, sh->d_x, sh->G * sizeof(double), cudaMemcpyDeviceToHost, sh->h->stream));
    SH_CUDA(cudaStreamSynchronize(sh->h->stream));
    return OPF_OK;
}

int opf_shard_get_locals(opf_shard *sh, double *xs, double *lam, size_t n) {
    if (!sh) return OPF_E_INVALID;
    return opf_get_locals(sh->h, xs, lam, n);
}

void *opf_shard_stream(opf_shard *sh) { return sh ? (void *)sh->h->stream : nullptr; }

void opf_shard_destroy(opf_shard *sh) {
    if (!sh) return;
    if (sh->h) cudaSetDevice(sh->h->device);
    if (sh->h) cudaStreamSynchronize(sh->h->stream);
    if (sh->d_part) cudaFree(sh->d_part);
    opf_destroy(sh->h);      // frees the shard's other device arrays with the handle's
    delete sh;
}

int opf_test_rule(const double *sums, double rho, double eps_rel, double eps_abs_pres, double *out) {
    if (!sums || !(rho > 0)) return OPF_E_INVALID;
    const double pres = std::sqrt(sums[0]), dres = rho * std::sqrt(sums[1]);
    const double eprim = std::max(std::sqrt(sums[2]), std::sqrt(sums[3])), edual = std::sqrt(sums[4]);
    if (out) {
        out[0] = pres; out[1] = dres; out[2] = eprim; out[3] = edual; out[4] = sums[5];
    }
    if (!std::isfinite(pres) || !std::isfinite(dres)) return OPF_E_NUMERIC;
    return (pres <= eps_rel * eprim && dres <= eps_rel * edual && pres <= eps_abs_pres) ? 1 : 0;
}

}  // extern "C"
