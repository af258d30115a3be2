// C ABI of the ADMM library: handle life cycle, device layout, and the
// drivers that run Algorithm 1 on the device (see include/opf.h).
//
// Device layout
//   Subsystems are reordered by size class (lanes per subsystem W = 8, 16, 32;
//   R rows per lane for n_s > 32) and packed into warp tasks.  Local slots
//   follow that order.  The buffer u = rho x_s - lambda is stored in
//   "global-major" order: the copies of each global i are one contiguous
//   segment (in canonical slot order), so the global update of Eq. closed_1
//   is a fixed-order segment sum and needs no atomics.
//
// Solve loop
//   One CUDA graph per solve: a conditional WHILE node whose body runs a
//   chunk of iterations ending with the Sec. III-C test; the test kernel sets
//   the loop condition on the device, so a solve is one graph launch and one
//   final status read.
#include <algorithm>
#include <map>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "opf_internal.h"
#include "warp_place.h"

namespace opf {




int launch_precompute(const PreArgs &a, cudaStream_t st);
void launch_pack_factors(int S, const int4 *sub, const int4 *sub2, const long long *cap_off,
                         const double *src, double *dst64, float *dst32, cudaStream_t st);
template <typename T>
void launch_iterate(const IterArgs<T> &a, const T *u_in, T *u_out, double *partials,
                    const DevStatus *st, bool check, int n_tiles, int block, int xcap, int vcap,
                    int tcap, cudaStream_t s);
void launch_check(const double *partials, int nblk, DevStatus *st, double rho, int add,
                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);
void launch_copy_if_running(long long n, const double *src, double *dst, const DevStatus *st,
                            cudaStream_t s);
void launch_add_iters(DevStatus *st, long long n, cudaStream_t s);
template <typename T> int prepare_cluster_engine(unsigned bytes, int P);
template <typename T>
int launch_cluster_engine(const IterArgs<T> &g, const ClusterLayout &lay, const int *pr, T *u_glob,
                          int n_iters, int check_every, DevStatus *st, double rho,
                          cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);
template <typename T> int cluster_occupancy(const ClusterLayout &lay);
template <typename T> int prepare_persist_engine(unsigned bytes);
template <typename T> int persist_occupancy(int threads, unsigned bytes);
template <typename T>
int launch_persist_engine(const IterArgs<T> &g, const PersistLayout &lay, const PersistPtrs &pp, T *U,
                          int bar_extra, int n_iters, int check_every, DevStatus *st, double rho,
                          cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);
template <typename T> int prepare_warp_engine(unsigned bytes);
template <typename T>
int launch_warp_engine(const IterArgs<T> &g, const WarpLayout &lay, const int *pr, T *u_glob, int n_iters,
                       int check_every, DevStatus *st, double rho, cudaGraphConditionalHandle cond, int use_cond,
                       cudaStream_t s);
template <typename T> int warp_engine_occupancy(const WarpLayout &lay);
template <typename T>
void launch_make_u(int L, const int *pk, const T *ds, const T *mu, T rho, T *u, const DevStatus *st,
                   cudaStream_t s);
template <typename T>
int launch_global_x(int G, const int2 *gseg, const T *u, const T *ct, const T *lbt, const T *ubt,
                    const double *xr, const double *c64, T rho, double *x, double *obj_part,
                    const DevStatus *st, cudaStream_t s);
template <typename T>
void launch_init_state(int L, const int *gk, const double *x0, T *ds, T *mu, cudaStream_t s);
template <typename T>
void launch_unshift(int L, const int *gk, const double *xr, const double *lamr, const T *ds,
                    const T *mu, double *ds64, double *mu64, cudaStream_t s);
template <typename A, typename B>
void launch_cast(long long n, const A *src, B *dst, cudaStream_t s);
template <typename T>
void launch_recenter(int L, int G, int S, const int *gk, const double *xr_old, const double *xr_new,
                     T *ds, T *mu, double *lamr, const int2 *gseg, const int *uslot,
                     const double *c64, const double *lb, const double *ub, T *ct, T *lbt, T *ubt,
                     const int4 *sub, const int4 *sub2, const double *F64, const double *bbar,
                     double rho, T *bt, const DevStatus *st, cudaStream_t s);
void launch_enter_shift(int L, const int *gk, const double *xr, const double *ds64,
                        const double *mu64, float *ds32, float *mu32, double *lamr, cudaStream_t s);

}  // namespace opf

using namespace opf;

static thread_local std::string g_last_error;

void opf::set_last_error(const std::string &msg) { g_last_error = msg; }

double opf::steady_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            g_last_error = std::string(#call) + ": " + cudaGetErrorString(e_);           \
            return e_ == cudaErrorMemoryAllocation ? OPF_E_OOM : OPF_E_CUDA;             \
        }                                                                                \
    } while (0)

#include "handle.h"


template <typename T>
static int dalloc(opf_handle *h, T **p, size_t n) {
    if (n == 0) n = 1;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
        g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return OPF_E_OOM;
    }
    h->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return OPF_OK;
}

template <typename T>
static int upload(opf_handle *h, T **p, const std::vector<T> &v) {
    int rc = dalloc(h, p, v.size());
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
    h->h2d_bytes += (long long)(v.size() * sizeof(T));
    return OPF_OK;
}

#define TRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

static unsigned align16(unsigned x) { return (x + 15u) & ~15u; }
static int round4(int x) { return (x + 3) & ~3; }

// Greedy tiling: consecutive subsystems until a tile holds >= target slots.
static int make_tiling(opf_handle *h, Tiling *t, int target, int block) {
    std::vector<int> s0;
    t->xcap = t->vcap = t->tcap = 0;
    int s = 0;
    while (s < h->S) {
        s0.push_back(s);
        int slots = 0, v = 0, f = 0;
        while (s < h->S && (slots == 0 || slots + h->h_sn[s] <= target)) {
            slots += h->h_sn[s];
            v += round4(h->h_sn[s]);
            f += h->h_sf[s];
            ++s;
        }
        t->xcap = std::max(t->xcap, slots);
        t->vcap = std::max(t->vcap, v);
        t->tcap = std::max(t->tcap, f);
    }
    s0.push_back(h->S);
    t->n_tiles = (int)s0.size() - 1;
    t->block = block;
    t->vcap = round4(t->vcap);
    t->xcap = round4(t->xcap);
    CUDA_TRY(cudaMemcpyAsync(t->d_s0, s0.data(), s0.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    return OPF_OK;
}

static int build_layout(opf_handle *h) {
    HostModel &M = h->model;
    h->S = (int)M.subs.size();
    h->G = M.n;
    // device order: larger subsystems first (tiles then hold similar sizes)
    std::vector<int> order(h->S);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return M.subs[a].n > M.subs[b].n; });
    std::vector<int> csoff(h->S + 1, 0);
    for (int s = 0; s < h->S; ++s) csoff[s + 1] = csoff[s] + M.subs[s].n;
    h->L = csoff[h->S];
    if (h->L >= (1 << 24) || h->S >= (1 << 23)) {
        g_last_error = "more than 2^24 local slots or 2^23 subsystems";
        return OPF_E_CAPACITY;
    }
    std::vector<int> soff(h->S + 1), sn(h->S), sm(h->S), boff(h->S), meta(h->L);
    std::vector<long long> aoff(h->S), poff(h->S), fcap(h->S);
    std::vector<double> A, b;
    h->canon_slot_to_dev.assign(h->L, 0);
    std::vector<int> gk(h->L);
    long long ao = 0, po = 0, fo = 0, fc = 0;
    int so = 0, bo = 0;
    h->max_ns = 0;
    h->n_rows = 0;
    h->sh_m = 0;
    for (int d = 0; d < h->S; ++d) {
        const HostSub &s = M.subs[order[d]];
        soff[d] = so; sn[d] = s.n; sm[d] = s.m; boff[d] = bo;
        aoff[d] = ao; poff[d] = po; fcap[d] = fo;
        for (int r = 0; r < s.n; ++r) {
            h->canon_slot_to_dev[csoff[order[d]] + r] = so + r;
            gk[so + r] = s.vars[r];
            meta[so + r] = (d << 8) | r;
        }
        A.insert(A.end(), s.A.begin(), s.A.end());
        b.insert(b.end(), s.b.begin(), s.b.end());
        so += s.n; bo += s.m;
        ao += (long long)s.m * s.n;
        po += (long long)s.n * s.n + 33LL * (s.m + s.n) + 64;
        const int fmax = std::max(0, std::min(s.m, s.n / 2));
        fo += (long long)s.n * fmax;
        fc += (long long)round4(s.n) * fmax;
        h->max_ns = std::max(h->max_ns, s.n);
        h->sh_m = std::max(h->sh_m, s.m);
        h->n_rows += s.m;
    }
    soff[h->S] = so;
    h->h_boff = boff;
    h->dev_to_canon_sub = order;
    {
        std::vector<int> crow0(h->S + 1, 0);
        for (int cs = 0; cs < h->S; ++cs) crow0[cs + 1] = crow0[cs] + M.subs[cs].m;
        h->canon_row_to_dev.assign(crow0[h->S], 0);
        for (int d = 0; d < h->S; ++d)
            for (int i = 0; i < sm[d]; ++i) h->canon_row_to_dev[crow0[order[d]] + i] = boff[d] + i;
    }
    h->nA = ao; h->nB = bo; h->nP = po; h->nFcap = fo; h->nF = std::max<long long>(fc, 4);
    h->sh_m = std::min(h->sh_m, 64);
    h->sh_n = std::min(h->max_ns, 64);
    // u segments: copies of each global contiguous, canonical slot order inside
    std::vector<int> cnt(h->G, 0);
    for (int k = 0; k < h->L; ++k) cnt[gk[k]]++;
    for (int i = 0; i < h->G; ++i)
        if (cnt[i] > 255) {
            g_last_error = "a global variable with more than 255 local copies";
            return OPF_E_CAPACITY;
        }
    std::vector<int> gstart(h->G + 1, 0);
    for (int i = 0; i < h->G; ++i) gstart[i + 1] = gstart[i] + cnt[i];
    std::vector<int> fill(gstart.begin(), gstart.end() - 1);
    std::vector<int> pk(h->L), uslot(h->L), segp(h->L);
    for (int cs = 0; cs < h->L; ++cs) {            // canonical order
        int k = h->canon_slot_to_dev[cs];
        int g = gk[k];
        pk[k] = fill[g]++;
        uslot[pk[k]] = k;
    }
    std::vector<int2> gseg(h->G);
    for (int i = 0; i < h->G; ++i) gseg[i] = make_int2(gstart[i], cnt[i]);
    for (int k = 0; k < h->L; ++k) segp[k] = (gstart[gk[k]] << 8) | cnt[gk[k]];
    h->h_pk = pk;
    h->h_gk = gk;
    h->h_gstart = gstart;
    h->h_uslot = uslot;
    // start point of Sec. V-A
    std::vector<double> x0(h->G, 0.0);
    for (int i = 0; i < h->G; ++i) {
        double lo = M.lb[i], hi = M.ub[i];
        if (M.volt[i]) x0[i] = 1.0;
        else if (std::isfinite(lo) && std::isfinite(hi)) x0[i] = 0.5 * (lo + hi);
        else if (std::isfinite(lo)) x0[i] = lo;
        else if (std::isfinite(hi)) x0[i] = hi;
    }
    h->h_sn = sn;
    h->h_sm = sm;
    h->h_soff = soff;
    // ---- uploads
    TRY(upload(h, &h->d_soff, soff));
    TRY(upload(h, &h->d_sn, sn));
    TRY(upload(h, &h->d_sm, sm));
    TRY(upload(h, &h->d_boff, boff));
    TRY(upload(h, &h->d_aoff, aoff));
    TRY(upload(h, &h->d_poff, poff));
    TRY(upload(h, &h->d_fcap, fcap));
    TRY(upload(h, &h->d_gk, gk));
    TRY(upload(h, &h->d_pk, pk));
    TRY(upload(h, &h->d_uslot, uslot));
    TRY(upload(h, &h->d_meta, meta));
    TRY(upload(h, &h->d_segp, segp));
    TRY(upload(h, &h->d_gseg, gseg));
    TRY(upload(h, &h->d_A, A));
    TRY(upload(h, &h->d_b, b));
    TRY(upload(h, &h->d_c64, M.c));
    TRY(upload(h, &h->d_lb64, M.lb));
    TRY(upload(h, &h->d_ub64, M.ub));
    TRY(upload(h, &h->d_x0, x0));
    const size_t L = h->L, G = h->G;
    long long items_cap = 0;
    for (int d = 0; d < h->S; ++d) items_cap += std::max(0, std::min(sm[d], sn[d] / 2));
    TRY(dalloc(h, &h->d_sf, h->S));
    TRY(dalloc(h, &h->d_smode, h->S));
    TRY(dalloc(h, &h->d_pstatus, h->S));
    TRY(dalloc(h, &h->d_sub, h->S + 1));
    TRY(dalloc(h, &h->d_sub2, h->S + 1));
    TRY(dalloc(h, &h->d_items, std::max<long long>(items_cap, 1)));
    TRY(dalloc(h, &h->t64.d_s0, h->S + 1));
    TRY(dalloc(h, &h->t32.d_s0, h->S + 1));
    TRY(dalloc(h, &h->w32.d_pr, 8 * 17));
    TRY(dalloc(h, &h->w32.d_wrseg, h->L));
    TRY(dalloc(h, &h->w32.d_wdsp, h->L));
    TRY(dalloc(h, &h->w32.d_wdd, (size_t)h->L * 16));
    TRY(dalloc(h, &h->w32.d_wrep, h->L));
    TRY(dalloc(h, &h->w32.d_klb, h->S + 1));
    TRY(dalloc(h, &h->w32.d_fbig, h->S + 1));
    TRY(dalloc(h, &h->w32.d_F2, h->nF));
    for (PersistPlan *pp : {&h->p32, &h->p64}) {
        TRY(dalloc(h, &pp->d_pr, 5 * (kPersistMaxP + 1)));
        TRY(dalloc(h, &pp->d_srec, h->S + 1));
        TRY(dalloc(h, &pp->d_items, std::max<long long>(items_cap, 1)));
        TRY(dalloc(h, &pp->d_meta, h->L));
        TRY(dalloc(h, &pp->d_part, 6 * kPersistMaxP));
        TRY(dalloc(h, &pp->d_sync, 1));
    }
    for (ClusterPlan *cp : {&h->c32, &h->c64}) {
        TRY(dalloc(h, &cp->d_pr, 8 * 17));
        TRY(dalloc(h, &cp->d_srec, h->S + 1));
        TRY(dalloc(h, &cp->d_items, std::max<long long>(items_cap, 1)));
        TRY(dalloc(h, &cp->d_meta, h->L));
        TRY(dalloc(h, &cp->d_udst, h->L));
        TRY(dalloc(h, &cp->d_gsegp, h->G));
        TRY(dalloc(h, &cp->d_cdst, h->L));
    }
    TRY(dalloc(h, &h->d_W, h->nA));
    TRY(dalloc(h, &h->d_Bw, h->nB));
    TRY(dalloc(h, &h->d_P, h->nP));
    TRY(dalloc(h, &h->d_Fcap, h->nFcap));
    TRY(dalloc(h, &h->d_F64, h->nF));
    TRY(dalloc(h, &h->d_F32, h->nF));
    TRY(dalloc(h, &h->d_bbar64, L));
    TRY(dalloc(h, &h->d_xr, G));
    TRY(dalloc(h, &h->d_xr2, G));
    TRY(dalloc(h, &h->d_zeroG, G));
    TRY(dalloc(h, &h->d_x, G));
    TRY(dalloc(h, &h->d_objpart, 4096));
    TRY(dalloc(h, &h->d_ct32, G));
    TRY(dalloc(h, &h->d_lbt32, G));
    TRY(dalloc(h, &h->d_ubt32, G));
    TRY(dalloc(h, &h->d_recip64, 256));
    TRY(dalloc(h, &h->d_recip32, 256));
    TRY(dalloc(h, &h->d_ds64, L));
    TRY(dalloc(h, &h->d_mu64, L));
    TRY(dalloc(h, &h->d_u64, 2 * L));
    TRY(dalloc(h, &h->d_lamr, L));
    TRY(dalloc(h, &h->d_zeroL, L));
    TRY(dalloc(h, &h->d_ds32, L));
    TRY(dalloc(h, &h->d_mu32, L));
    TRY(dalloc(h, &h->d_u32, 2 * L));
    TRY(dalloc(h, &h->d_bt32, L));
    TRY(dalloc(h, &h->d_partials, (size_t)6 * (h->S + 1)));
    TRY(dalloc(h, &h->d_st, 1));
    CUDA_TRY(cudaMemsetAsync(h->d_zeroG, 0, G * sizeof(double), h->stream));
    CUDA_TRY(cudaMemsetAsync(h->d_zeroL, 0, L * sizeof(double), h->stream));
    CUDA_TRY(cudaMemsetAsync(h->d_st, 0, sizeof(DevStatus), h->stream));
    CUDA_TRY(cudaMallocHost(&h->h_st, sizeof(DevStatus)));
    memset(h->h_st, 0, sizeof(DevStatus));
    for (auto &e : h->ev) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

static int common_create(opf_handle *h, const opf_options *o) {
    h->device = o ? o->device : 0;
    CUDA_TRY(cudaSetDevice(h->device));
    if (o && o->stream) {
        h->stream = (cudaStream_t)o->stream;
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    return build_layout(h);
}

extern "C" int opf_create(const opf_feeder *f, const opf_options *o, opf_handle **out) {
    if (!out) return OPF_E_INVALID;
    *out = nullptr;
    opf_handle *h = new opf_handle();
    int rc = build_feeder_model(f, &h->model, &g_last_error);
    if (rc == OPF_OK) rc = common_create(h, o);
    if (rc != OPF_OK) { opf_destroy(h); return rc; }
    *out = h;
    return OPF_OK;
}

extern "C" int opf_create_generic(int32_t n, const double *c, const double *lb, const double *ub,
                                  const uint8_t *is_voltage, int32_t S, const int32_t *m_s,
                                  const int32_t *n_s, const double *A, const double *b,
                                  const int32_t *idx, const opf_options *o, opf_handle **out) {
    if (!out) return OPF_E_INVALID;
    *out = nullptr;
    opf_handle *h = new opf_handle();
    int rc = build_generic_model(n, c, lb, ub, is_voltage, S, m_s, n_s, A, b, idx, &h->model, &g_last_error);
    if (rc == OPF_OK) rc = common_create(h, o);
    if (rc != OPF_OK) { opf_destroy(h); return rc; }
    *out = h;
    return OPF_OK;
}

static int reset_state(opf_handle *h) {
    launch_init_state<double>(h->L, h->d_gk, h->d_x0, h->d_ds64, h->d_mu64, h->stream);
    CUDA_TRY(cudaGetLastError());
    h->have_prev_u = false;
    h->total_iters = 0;
    memset(h->h_st, 0, sizeof(DevStatus));
    CUDA_TRY(cudaMemsetAsync(h->d_st, 0, sizeof(DevStatus), h->stream));
    return OPF_OK;
}

// The precompute kernel on fresh work copies of A and b; with_pinv adds the
// A_s^+ outputs.
static int launch_precompute_kernel(opf_handle *h, bool with_pinv) {
    CUDA_TRY(cudaMemcpyAsync(h->d_W, h->d_A, std::max<long long>(h->nA, 1) * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_Bw, h->d_b, std::max<long long>(h->nB, 1) * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    PreArgs a;
    memset(&a, 0, sizeof(a));
    a.S = h->S; a.sh_m = h->sh_m; a.sh_n = h->sh_n;
    a.sm = h->d_sm; a.sn = h->d_sn; a.soff = h->d_soff;
    a.aoff = h->d_aoff; a.poff = h->d_poff; a.foff = h->d_fcap; a.boff = h->d_boff;
    a.W = h->d_W; a.Bw = h->d_Bw; a.P = h->d_P; a.F = h->d_Fcap;
    a.sf = h->d_sf; a.smode = h->d_smode; a.bbar = h->d_bbar64; a.status = h->d_pstatus;
    if (with_pinv) {
        a.Tw = h->d_Tw; a.toff = h->d_toff; a.pinv = h->d_pinv; a.pioff = h->d_pioff; a.nrej = h->d_nrej;
    }
    if (launch_precompute(a, h->stream)) { g_last_error = "cannot size the precompute kernel"; return OPF_E_CUDA; }
    CUDA_TRY(cudaGetLastError());
    return OPF_OK;
}

int opf::ensure_pinv(opf_handle *h) {
    if (h->have_pinv) return OPF_OK;
    if (!h->precomputed) return OPF_E_STATE;
    CUDA_TRY(cudaSetDevice(h->device));
    if (!h->d_pinv) {
        h->h_pioff.assign(h->S + 1, 0);
        h->h_toff.assign(h->S + 1, 0);
        for (int d = 0; d < h->S; ++d) {
            h->h_pioff[d + 1] = h->h_pioff[d] + (long long)h->h_sn[d] * h->h_sm[d];
            h->h_toff[d + 1] = h->h_toff[d] + 2LL * h->h_sm[d] * h->h_sm[d];
        }
        TRY(dalloc(h, &h->d_pinv, (size_t)std::max<long long>(h->h_pioff[h->S], 1)));
        TRY(dalloc(h, &h->d_Tw, (size_t)std::max<long long>(h->h_toff[h->S], 1)));
        TRY(upload(h, &h->d_pioff, h->h_pioff));
        TRY(upload(h, &h->d_toff, h->h_toff));
        TRY(dalloc(h, &h->d_nrej, (size_t)h->S));
    }
    TRY(launch_precompute_kernel(h, true));
    h->h_nrej.resize(h->S);
    CUDA_TRY(cudaMemcpyAsync(h->h_nrej.data(), h->d_nrej, h->S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->have_pinv = true;
    return OPF_OK;
}

const char *opf::last_error_cstr() { return g_last_error.c_str(); }

extern "C" int opf_precompute(opf_handle *h) {
    if (!h) return OPF_E_INVALID;
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaEventRecord(h->ev[0], h->stream));
    h->have_pinv = false;
    TRY(launch_precompute_kernel(h, false));
    std::vector<int> status(h->S);
    h->h_sf.resize(h->S);
    CUDA_TRY(cudaMemcpyAsync(status.data(), h->d_pstatus, h->S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->h_sf.data(), h->d_sf, h->S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int s = 0; s < h->S; ++s)
        if (status[s]) {
            g_last_error = "inconsistent local system A_s x_s = b_s";
            h->precomputed = false;
            return OPF_E_INFEASIBLE_LOCAL;
        }
    // iteration layout: per subsystem (first slot, n, f, mode) and (factor
    // offset, npad, padded-v prefix, f prefix); factor columns padded to npad
    h->h_mode.resize(h->S);
    CUDA_TRY(cudaMemcpyAsync(h->h_mode.data(), h->d_smode, h->S * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    std::vector<int4> sub(h->S + 1), sub2(h->S + 1);
    h->h_tpre.assign(h->S + 1, 0); h->h_vpre.assign(h->S + 1, 0); h->h_foff.assign(h->S + 1, 0);
    h->h_npad.assign(h->S, 0);
    std::vector<int> items;
    long long fo = 0, vpre = 0, tpre = 0;
    h->sum_nf = 0;
    for (int s = 0; s < h->S; ++s) {
        const int n = h->h_sn[s], f = h->h_sf[s], npad = round4(n);
        sub[s] = make_int4(h->h_soff[s], n, f, h->h_mode[s]);
        sub2[s] = make_int4((int)fo, npad, (int)vpre, (int)tpre);
        h->h_foff[s] = (int)fo; h->h_vpre[s] = (int)vpre; h->h_tpre[s] = (int)tpre; h->h_npad[s] = npad;
        for (int c = 0; c < f; ++c) items.push_back((s << 8) | c);
        fo += (long long)f * npad;
        vpre += npad;
        tpre += f;
        h->sum_nf += (long long)n * f;
    }
    sub[h->S] = make_int4(h->L, 0, 0, 0);
    h->h_foff[h->S] = (int)fo; h->h_vpre[h->S] = (int)vpre; h->h_tpre[h->S] = (int)tpre;
    sub2[h->S] = make_int4((int)fo, 0, (int)vpre, (int)tpre);
    h->nitems = (long long)items.size();
    CUDA_TRY(cudaMemcpyAsync(h->d_sub, sub.data(), sub.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_sub2, sub2.data(), sub2.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    if (!items.empty())
        CUDA_TRY(cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    launch_pack_factors(h->S, h->d_sub, h->d_sub2, h->d_fcap, h->d_Fcap, h->d_F64, h->d_F32, h->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(h->ev[1], h->stream));
    CUDA_TRY(cudaEventSynchronize(h->ev[1]));
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->timing[0] = ms;
    h->nF = std::max<long long>(fo, 4);
    TRY(make_tiling(h, &h->t64, 64, 64));
    TRY(make_tiling(h, &h->t32, 256, 128));
    h->c32.P = h->c64.P = 0;
    h->c32.ok = h->c64.ok = false;
    h->p32.P = h->p64.P = 0;
    h->p32.ok = h->p64.ok = h->p32.tried = h->p64.tried = false;
    h->w32.built = h->w32.ok = false;
    h->w64.built = h->w64.ok = false;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->g64.reset();
    h->gmix.reset();
    h->precomputed = true;
    return reset_state(h);
}

extern "C" int opf_reset(opf_handle *h) {
    if (!h) return OPF_E_INVALID;
    if (!h->precomputed) return OPF_E_STATE;
    CUDA_TRY(cudaSetDevice(h->device));
    int rc = reset_state(h);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

template <typename T>
static IterArgs<T> common_args(opf_handle *h) {
    IterArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.sub = h->d_sub; a.sub2 = h->d_sub2; a.items = h->d_items;
    a.meta = h->d_meta; a.segp = h->d_segp; a.gk = h->d_gk; a.pk = h->d_pk;
    a.c64 = h->d_c64;
    return a;
}

template <typename T>
static IterArgs<T> iter_args(opf_handle *h, double rho);

template <>
IterArgs<double> iter_args<double>(opf_handle *h, double rho) {
    IterArgs<double> a = common_args<double>(h);
    a.F = h->d_F64; a.bt = h->d_bbar64; a.mu = h->d_mu64; a.ds = h->d_ds64;
    a.ct = h->d_c64; a.lbt = h->d_lb64; a.ubt = h->d_ub64;
    a.xr = h->d_zeroG; a.lamr = h->d_zeroL; a.recip = h->d_recip64;
    a.tile_s0 = h->t64.d_s0;
    a.rho = rho; a.inv_rho = 1.0 / rho;
    return a;
}

template <>
IterArgs<float> iter_args<float>(opf_handle *h, double rho) {
    IterArgs<float> a = common_args<float>(h);
    a.F = h->d_F32; a.bt = h->d_bt32; a.mu = h->d_mu32; a.ds = h->d_ds32;
    a.ct = h->d_ct32; a.lbt = h->d_lbt32; a.ubt = h->d_ubt32;
    a.xr = h->d_xr; a.lamr = h->d_lamr; a.recip = h->d_recip32;
    a.tile_s0 = h->t32.d_s0;
    a.rho = (float)rho; a.inv_rho = (float)(1.0 / rho);
    return a;
}

static unsigned align16u(size_t x) { return (unsigned)((x + 15) & ~(size_t)15); }

// Partition the instance over P CTAs of one cluster (contiguous subsystem
// ranges balanced by work, contiguous global ranges balanced by copies), build
// the part-relative records and the shared-memory layout.
template <typename T>
static int build_cluster_plan(opf_handle *h, ClusterPlan *cp, int P) {
    cp->ok = false;
    cp->P = P;
    const int S = h->S, G = h->G, L = h->L;
    std::vector<double> cost(S);
    double total = 0;
    for (int s = 0; s < S; ++s) {
        cost[s] = 6.0 * h->h_sn[s] + (double)h->h_sf[s] * h->h_npad[s] + (double)h->h_sn[s] * h->h_sf[s];
        total += cost[s];
    }
    std::vector<int> sp(P + 1, S);
    sp[0] = 0;
    {
        double acc = 0;
        int p = 1;
        for (int s = 0; s < S && p < P; ++s) {
            acc += cost[s];
            while (p < P && acc >= total * p / P) sp[p++] = s + 1;
        }
        for (int p2 = 1; p2 <= P; ++p2) sp[p2] = std::max(sp[p2], sp[p2 - 1]);
        sp[P] = S;
    }
    std::vector<int> gp(P + 1, G);
    gp[0] = 0;
    {
        double tot = 0;
        for (int i = 0; i < G; ++i) tot += 1.0 + (h->h_gstart[i + 1] - h->h_gstart[i]);
        double acc = 0;
        int p = 1;
        for (int i = 0; i < G && p < P; ++i) {
            acc += 1.0 + (h->h_gstart[i + 1] - h->h_gstart[i]);
            while (p < P && acc >= tot * p / P) gp[p++] = i + 1;
        }
        for (int p2 = 1; p2 <= P; ++p2) gp[p2] = std::max(gp[p2], gp[p2 - 1]);
        gp[P] = G;
    }
    std::vector<int> part_of_sub(S), owner_of_g(G);
    for (int p = 0; p < P; ++p) {
        for (int s = sp[p]; s < sp[p + 1]; ++s) part_of_sub[s] = p;
        for (int i = gp[p]; i < gp[p + 1]; ++i) owner_of_g[i] = p;
    }
    std::vector<int> pr(8 * (P + 1));
    auto PR = [&](int field, int p) -> int & { return pr[field * (P + 1) + p]; };
    for (int p = 0; p <= P; ++p) {
        const int s = sp[p];
        PR(0, p) = h->h_soff[s];
        PR(1, p) = s;
        PR(2, p) = h->h_tpre[s];
        PR(3, p) = h->h_foff[s];
        PR(4, p) = h->h_vpre[s];
        PR(5, p) = h->h_tpre[s];
        PR(6, p) = gp[p];
        PR(7, p) = h->h_gstart[gp[p]];
    }
    std::vector<int4> srec(S + 1, make_int4(0, 0, 0, 0));
    std::vector<int> items, meta(L), udst(L), gsegp(G), cdst(L);
    for (int s = 0; s < S; ++s) {
        const int p = part_of_sub[s];
        srec[s] = make_int4(h->h_foff[s] - PR(3, p), h->h_vpre[s] - PR(4, p), h->h_tpre[s] - PR(5, p),
                            (h->h_sf[s] << 10) | (h->h_npad[s] << 1) | (h->h_mode[s] & 1));
        for (int c = 0; c < h->h_sf[s]; ++c) items.push_back(((s - sp[p]) << 8) | c);
        for (int r = 0; r < h->h_sn[s]; ++r) {
            const int k = h->h_soff[s] + r;
            meta[k] = ((s - sp[p]) << 8) | r;
            const int gi = h->h_gk[k];
            const int o = owner_of_g[gi];
            udst[k] = (o << 24) | (h->h_pk[k] - PR(7, o));
            cdst[h->h_pk[k]] = (p << 24) | (h->h_vpre[s] + r - PR(4, p));
        }
    }
    for (int i = 0; i < G; ++i) {
        const int o = owner_of_g[i];
        gsegp[i] = ((h->h_gstart[i] - PR(7, o)) << 8) | (h->h_gstart[i + 1] - h->h_gstart[i]);
    }
    // layout: maxima over the parts
    long long mf = 0, ms = 0, mj = 0, mk = 0, mv = 0, mg = 0, mu = 0;
    for (int p = 0; p < P; ++p) {
        mf = std::max<long long>(mf, PR(3, p + 1) - PR(3, p));
        ms = std::max<long long>(ms, PR(1, p + 1) - PR(1, p));
        mj = std::max<long long>(mj, PR(2, p + 1) - PR(2, p));
        mk = std::max<long long>(mk, PR(0, p + 1) - PR(0, p));
        mv = std::max<long long>(mv, PR(4, p + 1) - PR(4, p));
        mg = std::max<long long>(mg, PR(6, p + 1) - PR(6, p));
        mu = std::max<long long>(mu, PR(7, p + 1) - PR(7, p));
    }
    ClusterLayout &c = cp->lay;
    c = ClusterLayout{};
    c.P = P;
    c.L = L;
    size_t off = 0;
    auto take = [&](unsigned *o, size_t bytes) { *o = (unsigned)off; off = align16u(off + bytes); };
    take(&c.off_F, (size_t)mf * sizeof(T));
    take(&c.off_srec, (size_t)ms * sizeof(int4));
    take(&c.off_items, (size_t)mj * sizeof(int));
    take(&c.off_meta, (size_t)mk * sizeof(int));
    take(&c.off_udst, (size_t)mk * sizeof(int));
    take(&c.off_bt, (size_t)mk * sizeof(T));
    take(&c.off_ds, (size_t)mk * sizeof(T));
    take(&c.off_mu, (size_t)mk * sizeof(T));
    take(&c.off_vbx, (size_t)mv * sizeof(T));
    take(&c.off_vbw, (size_t)mv * sizeof(T));
    take(&c.off_tb, (size_t)mj * sizeof(T));
    take(&c.off_gsegp, (size_t)mg * sizeof(int));
    take(&c.off_ct, (size_t)mg * sizeof(T));
    take(&c.off_lbt, (size_t)mg * sizeof(T));
    take(&c.off_ubt, (size_t)mg * sizeof(T));
    take(&c.off_uloc, (size_t)mu * sizeof(T));
    take(&c.off_cdst, (size_t)mu * sizeof(int));
    take(&c.off_recip, 256 * sizeof(T));
    take(&c.off_red, 16 * 6 * sizeof(double) + 16);
    take(&c.off_xrg, (size_t)mg * sizeof(double));
    take(&c.off_cg, (size_t)mg * sizeof(double));
    take(&c.off_xrs, (size_t)mk * sizeof(double));
    take(&c.off_lrs, (size_t)mk * sizeof(double));
    c.bytes = (unsigned)off;
    long long work = std::max(mk, std::max(mg, mj));
    int threads = (int)std::min<long long>(1024, std::max<long long>(64, (work + 31) / 32 * 32));
    c.threads = threads;
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if ((long long)c.bytes + 4096 > optin) return OPF_OK;              // does not fit: plan not ok
    if (prepare_cluster_engine<T>(c.bytes, P)) { cudaGetLastError(); return OPF_OK; }
    if (cluster_occupancy<T>(c) < 1) { cudaGetLastError(); return OPF_OK; }
    CUDA_TRY(cudaMemcpyAsync(cp->d_pr, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(cp->d_srec, srec.data(), srec.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    if (!items.empty())
        CUDA_TRY(cudaMemcpyAsync(cp->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(cp->d_meta, meta.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(cp->d_udst, udst.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(cp->d_gsegp, gsegp.data(), G * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(cp->d_cdst, cdst.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    cp->ok = true;
    return OPF_OK;
}

// Cluster size: the requested one, else the smallest power of two giving at
// most `target` slots per CTA that fits; the plan is rebuilt when P changes.
template <typename T>
static int get_cluster_plan(opf_handle *h, ClusterPlan *cp, int requested, int target) {
    int want = requested;
    if (want <= 0) {
        want = 1;
        while (want < 16 && (long long)h->L > (long long)want * target) want *= 2;
    }
    want = std::min(16, std::max(1, want));
    if (cp->P == want && cp->ok) return OPF_OK;
    for (int P = want; P <= 16; P *= 2) {
        TRY(build_cluster_plan<T>(h, cp, P));
        if (cp->ok || requested > 0) break;
    }
    return OPF_OK;
}

// Partition the instance over P co-resident CTAs of the persistent grid
// engine: contiguous subsystem ranges balanced by work (the same cost as the
// cluster plan), part-relative records, and the shared-memory layout.  Leaves
// pp->ok false when a part does not fit one CTA or P CTAs cannot be resident.
template <typename T>
static int build_persist_plan(opf_handle *h, PersistPlan *pp, int P, int n_sm) {
    pp->ok = false;
    pp->P = P;
    if (P < 1 || P > kPersistMaxP) return OPF_OK;
    const int S = h->S, L = h->L;
    std::vector<double> cost(S);
    double total = 0;
    for (int s = 0; s < S; ++s) {
        cost[s] = 6.0 * h->h_sn[s] + (double)h->h_sf[s] * h->h_npad[s] + (double)h->h_sn[s] * h->h_sf[s];
        total += cost[s];
    }
    std::vector<int> sp(P + 1, S);
    sp[0] = 0;
    {
        double acc = 0;
        int p = 1;
        for (int s = 0; s < S && p < P; ++s) {
            acc += cost[s];
            while (p < P && acc >= total * p / P) sp[p++] = s + 1;
        }
        for (int p2 = 1; p2 <= P; ++p2) sp[p2] = std::max(sp[p2], sp[p2 - 1]);
        sp[P] = S;
    }
    const int P1 = P + 1;
    std::vector<int> pr(5 * P1);
    auto PR = [&](int field, int p) -> int & { return pr[field * P1 + p]; };
    for (int p = 0; p <= P; ++p) {
        const int s = sp[p];
        PR(0, p) = h->h_soff[s];
        PR(1, p) = s;
        PR(2, p) = h->h_tpre[s];
        PR(3, p) = h->h_foff[s];
        PR(4, p) = h->h_vpre[s];
    }
    // factors staged per part with column stride npad (+ 4 when npad % 8 == 0)
    std::vector<int4> srec(S + 1, make_int4(0, 0, 0, 0));
    std::vector<int> items, meta(L);
    std::vector<long long> fpart(P, 0);
    for (int p = 0; p < P; ++p) {
        for (int s = sp[p]; s < sp[p + 1]; ++s) {
            const int npad = h->h_npad[s], cs = npad + ((npad & 7) == 0 ? 4 : 0);
            srec[s] = make_int4((int)fpart[p], h->h_vpre[s] - PR(4, p), h->h_tpre[s] - PR(2, p),
                                (h->h_sf[s] << 10) | (npad << 1) | (h->h_mode[s] & 1));
            fpart[p] += (long long)h->h_sf[s] * cs;
            for (int c = 0; c < h->h_sf[s]; ++c) items.push_back(((s - sp[p]) << 8) | c);
            for (int r = 0; r < h->h_sn[s]; ++r) meta[h->h_soff[s] + r] = ((s - sp[p]) << 8) | r;
        }
    }
    long long mf = 0, ms = 0, mj = 0, mk = 0, mv = 0;
    for (int p = 0; p < P; ++p) {
        mk = std::max<long long>(mk, PR(0, p + 1) - PR(0, p));
        ms = std::max<long long>(ms, PR(1, p + 1) - PR(1, p));
        mj = std::max<long long>(mj, PR(2, p + 1) - PR(2, p));
        mf = std::max<long long>(mf, fpart[p]);
        mv = std::max<long long>(mv, PR(4, p + 1) - PR(4, p));
    }
    PersistLayout &c = pp->lay;
    c = PersistLayout{};
    c.P = P;
    c.L = L;
    size_t off = 0;
    auto take = [&](unsigned *o, size_t bytes) { *o = (unsigned)off; off = align16u(off + bytes); };
    take(&c.off_F, (size_t)mf * sizeof(T));
    take(&c.off_srec, (size_t)ms * sizeof(int4));
    take(&c.off_items, (size_t)mj * sizeof(int));
    take(&c.off_meta, (size_t)mk * sizeof(int));
    take(&c.off_segp, (size_t)mk * sizeof(int));
    take(&c.off_pk, (size_t)mk * sizeof(int));
    take(&c.off_bt, (size_t)mk * sizeof(T));
    take(&c.off_ds, (size_t)mk * sizeof(T));
    take(&c.off_mu, (size_t)mk * sizeof(T));
    take(&c.off_ct, (size_t)mk * sizeof(T));
    take(&c.off_lbt, (size_t)mk * sizeof(T));
    take(&c.off_ubt, (size_t)mk * sizeof(T));
    take(&c.off_vbx, (size_t)mv * sizeof(T));
    take(&c.off_vbw, (size_t)mv * sizeof(T));
    take(&c.off_tb, (size_t)mj * sizeof(T));
    take(&c.off_recip, 256 * sizeof(T));
    take(&c.off_xrs, (size_t)mk * sizeof(double));
    take(&c.off_lrs, (size_t)mk * sizeof(double));
    take(&c.off_cobj, (size_t)mk * sizeof(double));
    // flags (16 B), a DevStatus copy, the [32][6] block-sum scratch
    take(&c.off_misc, 16 + ((sizeof(DevStatus) + 15) & ~(size_t)15) + 32 * 6 * sizeof(double));
    c.bytes = (unsigned)off;
    c.threads = (int)std::min<long long>(kPersistMaxThreads, std::max<long long>(64, (std::max(mk, mj) + 31) / 32 * 32));
    // plans of small CTAs (one or a few subsystems each: the 123-bus feeder)
    // run phase B with each factor column on 4 lanes, given threads for it;
    // large ones keep one lane per column (the split measured slower there)
    c.split = 0;
    if (c.threads <= 128) {
        c.split = 1;
        c.threads = (int)std::min<long long>(kPersistMaxThreads, std::max<long long>(c.threads, (4 * mj + 31) / 32 * 32));
    }
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if ((long long)c.bytes > optin) return OPF_OK;
    if (prepare_persist_engine<T>(c.bytes)) { cudaGetLastError(); return OPF_OK; }
    const int occ = persist_occupancy<T>(c.threads, c.bytes);
    if ((long long)occ * n_sm < P) { cudaGetLastError(); return OPF_OK; }
    CUDA_TRY(cudaMemcpyAsync(pp->d_pr, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(pp->d_srec, srec.data(), srec.size() * sizeof(int4), cudaMemcpyHostToDevice, h->stream));
    if (!items.empty())
        CUDA_TRY(cudaMemcpyAsync(pp->d_items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 h->stream));
    CUDA_TRY(cudaMemcpyAsync(pp->d_meta, meta.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    pp->ok = true;
    return OPF_OK;
}

// CTA count: the requested one, else two per SM of the stream's SMs (one per
// SM when two do not fit), at most one CTA per 32 slots.
template <typename T>
static int get_persist_plan(opf_handle *h, PersistPlan *pp, int requested) {
    if (pp->tried && pp->req == requested) return OPF_OK;
    const int n_sm = stream_sm_count(h->stream, h->device);
    pp->tried = true;
    pp->req = requested;
    if (requested > 0) return build_persist_plan<T>(h, pp, requested, n_sm);
    const int cap = std::max(1, (h->L + 31) / 32);
    for (int per : {2, 1}) {
        TRY(build_persist_plan<T>(h, pp, std::min(per * n_sm, cap), n_sm));
        if (pp->ok) return OPF_OK;
    }
    return OPF_OK;
}

template <typename T>
static IterArgs<T> with_persist(IterArgs<T> a, const PersistPlan &pp) {
    a.srec = pp.d_srec; a.citems = pp.d_items; a.cmeta = pp.d_meta;
    return a;
}

constexpr int kWarpEngineWarps = 12;
// Warps per CTA when the cluster has room: one per SM sub-partition, so that
// the largest subsystems' warps do not share an FP64 pipe (FP64 iterations)
// or an issue slot (FP32: 5 % faster than 12 warps on the 13- and 34-bus feeders)
constexpr int kWarpEngineWarps64 = 4;

// Warp-engine plan for precision T.  Work items are warps: one per subsystem,
// or in FP64 two for the largest subsystems of more than 16 slots, as many as
// keep 4 warps per CTA (each takes half of its rows; the two sit in warp
// slots 2k, 2k + 1 of one CTA, on different SM sub-partitions, and add their
// halves of t = F^T v through shared memory).
// W items go to max(ceil(W / 12), min(16, ceil(W / 4))) CTAs unless req_P asks
// for a count: pairs first, round-robin over the CTAs, then single warps,
// round-robin in subsystem order.  FP32: factors of subsystems with n > 32 in
// shared memory (the rest in registers); FP64: every factor in shared memory.
template <typename T>
static int build_warp_plan(opf_handle *h, WarpPlan &wp, int req_P) {
    constexpr bool REG = sizeof(T) == 4;
    wp.built = true;
    wp.ok = false;
    wp.req = req_P;
    const int S = h->S, G = h->G, L = h->L;
    if (h->max_ns > 64) return OPF_OK;
    for (int s = 0; s < S; ++s)
        if (h->h_sf[s] > 32) return OPF_OK;
    // split the largest subsystems over two warps while the warps stay within
    // 4 per CTA of the cluster (16 CTAs, or req_P): in FP64 those of more than
    // 16 slots; in FP32 those of more than 32 (the ones whose factor is in
    // shared memory), up to 12 warps per CTA
    std::vector<int> nparts(S, 1);
    {
        const int min_n = REG ? 32 : 16;
        std::vector<int> big_first;
        for (int s = 0; s < S; ++s)
            if (h->h_sn[s] > min_n) big_first.push_back(s);
        std::stable_sort(big_first.begin(), big_first.end(), [&](int x, int y) {
            return h->h_sn[x] * (h->h_sf[x] + 4) > h->h_sn[y] * (h->h_sf[y] + 4);
        });
        const int per_cta = REG ? kWarpEngineWarps : kWarpEngineWarps64;
        const int budget = (req_P > 0 ? req_P : 16) * per_cta - S;
        for (int i = 0; i < (int)big_first.size() && i < budget; ++i) nparts[big_first[i]] = 2;
    }
    int W = 0;
    for (int s = 0; s < S; ++s) W += nparts[s];
    int P = (W + kWarpEngineWarps - 1) / kWarpEngineWarps;
    if (P < 1 || P > 16) return OPF_OK;
    P = std::max(P, std::min(16, (W + kWarpEngineWarps64 - 1) / kWarpEngineWarps64));
    if (req_P > 0) {
        if (req_P > 16) return OPF_OK;
        P = req_P;
    }
    // place the items: cta_of[s], first warp slot slot_of[s]
    std::vector<int> cta_of, slot_of;
    const int warps = place_warp_items_min(nparts, P, kWarpEngineWarps, &cta_of, &slot_of);
    if (warps == 0) return OPF_OK;
    if (!REG && !wp.d_pr) {
        TRY(dalloc(h, &wp.d_pr, 8 * 17));
        TRY(dalloc(h, &wp.d_wrseg, h->L));
        TRY(dalloc(h, &wp.d_wdsp, h->L));
        TRY(dalloc(h, &wp.d_wdd, (size_t)h->L * 16));
        TRY(dalloc(h, &wp.d_wrep, h->L));
        TRY(dalloc(h, &wp.d_klb, h->S + 1));
        TRY(dalloc(h, &wp.d_fbig, h->S + 1));
        TRY(dalloc(h, &wp.d_F2d, h->nF));
    }
    if (!wp.d_wmap) TRY(dalloc(h, &wp.d_wmap, 16 * kWarpEngineWarps));
    std::vector<int> wmap((size_t)P * warps, -1);
    for (int s = 0; s < S; ++s)
        for (int q = 0; q < nparts[s]; ++q)
            wmap[(size_t)cta_of[s] * warps + slot_of[s] + q] = (s << 8) | (q << 4) | nparts[s];
    auto in_smem = [&](int s) { return !REG || h->h_sn[s] > 32; };
    wp.P = P;
    // local slots of each CTA, in subsystem order
    std::vector<int> nk(P, 0), klb(S + 1, 0), fb(P, 0), fbig(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        const int p = cta_of[s];
        klb[s] = nk[p];
        nk[p] += h->h_sn[s];
        if (in_smem(s)) fb[p] += h->h_sf[s] * h->h_npad[s];
    }
    std::vector<int> kb(P + 1, 0), fb0(P + 1, 0);
    for (int p = 0; p < P; ++p) { kb[p + 1] = kb[p] + nk[p]; fb0[p + 1] = fb0[p] + fb[p]; }
    {
        std::vector<int> fill(fb0.begin(), fb0.end() - 1);
        for (int s = 0; s < S; ++s)
            if (in_smem(s)) {
                const int p = cta_of[s];
                fbig[s] = fill[p];
                const size_t cnt = (size_t)h->h_sf[s] * h->h_npad[s];
                if (cnt) {
                    if (REG)
                        CUDA_TRY(cudaMemcpyAsync(wp.d_F2 + fill[p], h->d_F32 + h->h_foff[s], cnt * sizeof(float),
                                                 cudaMemcpyDeviceToDevice, h->stream));
                    else
                        CUDA_TRY(cudaMemcpyAsync(wp.d_F2d + fill[p], h->d_F64 + h->h_foff[s], cnt * sizeof(double),
                                                 cudaMemcpyDeviceToDevice, h->stream));
                }
                fill[p] += (int)cnt;
            }
    }
    // per CTA: a replica segment for every global with a copy there
    std::vector<std::vector<int>> rbase(P);          // rbase[p][g] (or -1), built sparse via map
    std::vector<std::vector<int3>> rep(P);
    std::vector<int> nru(P, 0);
    std::vector<std::map<int, int>> seg_of(P);
    for (int s = 0; s < S; ++s) {
        const int p = cta_of[s];
        for (int r = 0; r < h->h_sn[s]; ++r) {
            const int gi = h->h_gk[h->h_soff[s] + r];
            if (seg_of[p].count(gi)) continue;
            const int cnt = h->h_gstart[gi + 1] - h->h_gstart[gi];
            seg_of[p][gi] = nru[p];
            rep[p].push_back(make_int3(nru[p], h->h_gstart[gi], cnt));
            nru[p] += cnt;
        }
    }
    // which CTAs hold copies of each global
    std::vector<std::vector<int>> holders(G);
    for (int p = 0; p < P; ++p)
        for (auto &kv : seg_of[p]) holders[kv.first].push_back(p);
    // per local slot: replica segment and destination list
    std::vector<int> wrseg(L), wdsp(L), wdd;
    std::vector<int> db(P + 1, 0);
    std::vector<std::vector<int>> dd(P);
    for (int s = 0; s < S; ++s) {
        const int p = cta_of[s];
        for (int r = 0; r < h->h_sn[s]; ++r) {
            const int k = h->h_soff[s] + r;
            const int gi = h->h_gk[k];
            const int q = h->h_pk[k] - h->h_gstart[gi];
            const int cnt = h->h_gstart[gi + 1] - h->h_gstart[gi];
            const int kl = kb[p] + klb[s] + r;
            wrseg[kl] = (seg_of[p][gi] << 8) | cnt;
            const int nd = (int)holders[gi].size();
            wdsp[kl] = ((int)dd[p].size() << 8) | nd;
            for (int p2 : holders[gi]) dd[p].push_back((p2 << 24) | (seg_of[p2][gi] + q));
        }
    }
    for (int p = 0; p < P; ++p) db[p + 1] = db[p] + (int)dd[p].size();
    for (int p = 0; p < P; ++p) wdd.insert(wdd.end(), dd[p].begin(), dd[p].end());
    std::vector<int3> wrep;
    std::vector<int> rb(P + 1, 0), ru(P + 1, 0);
    for (int p = 0; p < P; ++p) {
        rb[p + 1] = rb[p] + (int)rep[p].size();
        ru[p + 1] = ru[p] + nru[p];
        wrep.insert(wrep.end(), rep[p].begin(), rep[p].end());
    }
    std::vector<int> pr(8 * (P + 1), 0);
    auto PR = [&](int field, int p) -> int & { return pr[field * (P + 1) + p]; };
    for (int p = 0; p <= P; ++p) {
        PR(0, p) = kb[p];
        PR(2, p) = db[p];
        PR(3, p) = fb0[p];
        PR(4, p) = rb[p];
        PR(7, p) = ru[p];
    }
    int mru = 0, mdd = 0, mf = 0;
    for (int p = 0; p < P; ++p) {
        mru = std::max(mru, nru[p]);
        mdd = std::max(mdd, (int)dd[p].size());
        mf = std::max(mf, fb[p]);
    }
    WarpLayout &c = wp.lay;
    c = WarpLayout{};
    c.P = P; c.L = L; c.S = S; c.warps = warps;
    c.useg_len = (mru + 3) & ~3;
    c.fbig_len = (mf + 3) & ~3;
    size_t off = 0;
    auto take = [&](unsigned *o, size_t bytes) { *o = (unsigned)off; off = align16u(off + bytes); };
    take(&c.off_useg, (size_t)2 * c.useg_len * sizeof(T));
    take(&c.off_dd, (size_t)mdd * sizeof(int));
    take(&c.off_fbig, (size_t)2 * c.fbig_len * sizeof(T));   // column-major factors, then row-major copies
    take(&c.off_vbig, (size_t)warps * 64 * sizeof(T));
    take(&c.off_tpart, (size_t)(warps / 2 + 1) * 64 * sizeof(T));   // per warp pair: two halves of t
    take(&c.off_red, 16 * 6 * sizeof(double) + 16);
    c.bytes = (unsigned)off;
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if ((long long)c.bytes + 4096 > optin) return OPF_OK;
    if (prepare_warp_engine<T>(c.bytes)) { cudaGetLastError(); return OPF_OK; }
    if (warp_engine_occupancy<T>(c) < 1) { cudaGetLastError(); return OPF_OK; }
    if ((size_t)wdd.size() > (size_t)h->L * 16 || wrep.size() > (size_t)h->L) return OPF_OK;
    CUDA_TRY(cudaMemcpyAsync(wp.d_pr, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(wp.d_wmap, wmap.data(), wmap.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(wp.d_klb, klb.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(wp.d_fbig, fbig.data(), (S + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(wp.d_wrseg, wrseg.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(wp.d_wdsp, wdsp.data(), L * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (!wdd.empty())
        CUDA_TRY(cudaMemcpyAsync(wp.d_wdd, wdd.data(), wdd.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    if (!wrep.empty())
        CUDA_TRY(cudaMemcpyAsync(wp.d_wrep, wrep.data(), wrep.size() * sizeof(int3), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    wp.ok = true;
    return OPF_OK;
}

static IterArgs<float> with_warp_plan(opf_handle *h, IterArgs<float> a, const WarpPlan &wp) {
    a.wmap = wp.d_wmap;
    a.klb = wp.d_klb; a.fbig = wp.d_fbig; a.F2 = wp.d_F2;
    a.wrseg = wp.d_wrseg; a.wdsp = wp.d_wdsp; a.wdd = wp.d_wdd; a.wrep = wp.d_wrep;
    a.u_prev_out = h->d_u32 + h->L;
    return a;
}

static IterArgs<double> with_warp_plan(opf_handle *h, IterArgs<double> a, const WarpPlan &wp) {
    a.wmap = wp.d_wmap;
    a.klb = wp.d_klb; a.fbig = wp.d_fbig; a.F2 = wp.d_F2d;
    a.wrseg = wp.d_wrseg; a.wdsp = wp.d_wdsp; a.wdd = wp.d_wdd; a.wrep = wp.d_wrep;
    a.u_prev_out = h->d_u64 + h->L;
    return a;
}

template <typename T>
static IterArgs<T> with_plan(IterArgs<T> a, const ClusterPlan &cp) {
    a.srec = cp.d_srec; a.citems = cp.d_items; a.cmeta = cp.d_meta;
    a.udst = cp.d_udst; a.gsegp = cp.d_gsegp; a.cdst = cp.d_cdst;
    return a;
}

// recip[N] = 1 / (rho N) for the global update, in both precisions
static int set_recip(opf_handle *h, double rho) {
    if (h->recip_rho == rho) return OPF_OK;
    std::vector<double> r64(256, 0.0);
    std::vector<float> r32(256, 0.0f);
    for (int n = 1; n < 256; ++n) {
        r64[n] = 1.0 / (rho * n);
        r32[n] = (float)r64[n];
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_recip64, r64.data(), 256 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_recip32, r32.data(), 256 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->recip_rho = rho;
    return OPF_OK;
}

template <typename T> static const Tiling &tiling(opf_handle *h);
template <> const Tiling &tiling<double>(opf_handle *h) { return h->t64; }
template <> const Tiling &tiling<float>(opf_handle *h) { return h->t32; }

// Enqueue one chunk of k grid iterations (the last one tested) and the test.
template <typename T>
static void enqueue_grid_chunk(opf_handle *h, const IterArgs<T> &a, T *u, int k, double rho,
                               cudaGraphConditionalHandle cond, int use_cond) {
    const Tiling &t = tiling<T>(h);
    for (int i = 0; i < k; ++i) {
        const T *uin = u + (size_t)(i & 1) * h->L;
        T *uout = u + (size_t)((i + 1) & 1) * h->L;
        launch_iterate<T>(a, uin, uout, h->d_partials, h->d_st, i == k - 1, t.n_tiles, t.block, t.xcap,
                          t.vcap, t.tcap, h->stream);
    }
    launch_check(h->d_partials, t.n_tiles, h->d_st, rho, k, cond, use_cond, h->stream);
}

// Build a graph "while (!done) body" where body is enqueued by fn(cond, 1).
// With host_loop the graph is the body alone (fn(0, 0)), relaunched by the
// host until the device status says done (profilers see its kernel nodes).
template <typename Fn>
static int build_while_graph(opf_handle *h, GraphCache *gc, Fn fn, bool host_loop) {
    gc->reset();
    if (host_loop) {
        gc->host_loop = true;
        return OPF_OK;
    }
    gc->host_loop = false;
    CUDA_TRY(cudaGraphCreate(&gc->graph, 0));
    cudaGraphConditionalHandle cond;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, gc->graph, 1, cudaGraphCondAssignDefault));
    // the parameter union has no default constructor in C++: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams *cp = reinterpret_cast<cudaGraphNodeParams *>(raw);
    cp->type = cudaGraphNodeTypeConditional;
    cp->conditional.handle = cond;
    cp->conditional.type = cudaGraphCondTypeWhile;
    cp->conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, gc->graph, nullptr, nullptr, 0, cp));
    cudaGraph_t body = cp->conditional.phGraph_out[0];
    CUDA_TRY(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    fn(cond, 1);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(h->stream, &captured);
    if (ec != cudaSuccess) {
        g_last_error = std::string("stream capture: ") + cudaGetErrorString(ec);
        gc->reset();
        return OPF_E_CUDA;
    }
    CUDA_TRY(cudaGraphInstantiate(&gc->exec, gc->graph, 0));
    return OPF_OK;
}

static int set_status(opf_handle *h, const opf_solve_opts &o, bool keep_iter) {
    DevStatus st{};
    st.iter = keep_iter ? h->h_st->iter : 0;
    st.max_iter = o.max_iter;
    st.eps_rel = o.eps_rel;
    st.eps_abs_pres = o.eps_abs_pres;
    *h->h_st = st;
    CUDA_TRY(cudaMemcpyAsync(h->d_st, h->h_st, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

static int read_status(opf_handle *h) {
    CUDA_TRY(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

// One launch of the WHILE graph, or (host loop) direct launches of the body
// until the status says done.
template <typename Fn>
static int run_graph(opf_handle *h, GraphCache *gc, Fn fn) {
    if (!gc->host_loop) {
        CUDA_TRY(cudaGraphLaunch(gc->exec, h->stream));
        return read_status(h);
    }
    for (;;) {
        fn(cudaGraphConditionalHandle{}, 0);
        CUDA_TRY(cudaGetLastError());
        TRY(read_status(h));
        if (h->h_st->done) return OPF_OK;
        if (h->cancel.load() || (h->deadline > 0.0 && opf::steady_seconds() > h->deadline)) {
            g_last_error = "solve stopped by its deadline or a cancel request";
            h->total_iters = h->h_st->iter;      // iterations run so far (opf_get_residuals)
            return OPF_E_TIMEOUT;
        }
    }
}

// FP64 iterations on the whole grid until the test or max_iter.
static int run_grid64(opf_handle *h, const opf_solve_opts &o) {
    const double rho = o.rho;
    TRY(set_recip(h, rho));
    launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    CUDA_TRY(cudaGetLastError());
    const bool hl = (o.flags & OPF_SOLVE_HOST_LOOP) != 0;
    IterArgs<double> a = iter_args<double>(h, rho);
    auto body = [&](cudaGraphConditionalHandle c, int use) {
        enqueue_grid_chunk<double>(h, a, h->d_u64, o.check_every, rho, c, use);
    };
    if (h->g64.kind != 0 || h->g64.rho != rho || h->g64.k != o.check_every || h->g64.host_loop != hl) {
        TRY(build_while_graph(h, &h->g64, body, hl));
        h->g64.kind = 0; h->g64.rho = rho; h->g64.k = o.check_every;
    }
    TRY(run_graph(h, &h->g64, body));
    h->have_prev_u = h->h_st->iter > 0;
    return OPF_OK;
}

// FP64 iterations by the cluster engine (same arithmetic, instance in the
// shared memory of one thread-block cluster), one launch up to max_iter.
static int run_cluster64(opf_handle *h, const opf_solve_opts &o) {
    const double rho = o.rho;
    TRY(set_recip(h, rho));
    launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    IterArgs<double> a = with_plan(iter_args<double>(h, rho), h->c64);
    if (launch_cluster_engine<double>(a, h->c64.lay, h->c64.d_pr, h->d_u64, o.max_iter, o.check_every, h->d_st,
                                      rho, cudaGraphConditionalHandle{}, 0, h->stream)) {
        g_last_error = "cluster engine launch failed";
        return OPF_E_CUDA;
    }
    CUDA_TRY(cudaGetLastError());
    TRY(read_status(h));
    h->have_prev_u = h->h_st->iter > 0;
    return OPF_OK;
}

// Iterations per launch of the persistent engine when it runs to the test
// (FP64 plain solves and the polish): the host reads the status in between.
constexpr int kPersistLaunchIters = 20000;

// Test hook: one arrival more than the grid has, so the first barrier's
// bounded wait runs out.
static int bar_extra(const opf_solve_opts &o) { return (o.flags & OPF_SOLVE_TEST_BARRIER_TIMEOUT) ? 1 : 0; }

static int fault_error(opf_handle *h) {
    if (!h->h_st->fault) return OPF_OK;
    g_last_error = "persistent grid engine: a grid barrier wait ran out";
    return OPF_E_TIMEOUT;
}

// FP64 iterations by the persistent grid engine until the test or max_iter.
static int run_persist64(opf_handle *h, const opf_solve_opts &o) {
    const double rho = o.rho;
    TRY(set_recip(h, rho));
    launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    CUDA_TRY(cudaGetLastError());
    const PersistPlan &pp = h->p64;
    IterArgs<double> a = with_persist(iter_args<double>(h, rho), pp);
    const int k = o.check_every;
    const int per = std::max(k, (kPersistLaunchIters / k) * k);
    for (;;) {
        if (launch_persist_engine<double>(a, pp.lay, pp.ptrs(), h->d_u64, bar_extra(o), per, k, h->d_st, rho,
                                          cudaGraphConditionalHandle{}, 0, h->stream)) {
            g_last_error = std::string("persistent grid engine launch failed: ") +
                           cudaGetErrorString(cudaGetLastError());
            return OPF_E_CUDA;
        }
        TRY(read_status(h));
        TRY(fault_error(h));
        if (h->h_st->done) break;
    }
    h->have_prev_u = h->h_st->iter > 0;
    return OPF_OK;
}

// FP64 iterations by the warp engine (the instance in one cluster, factors in
// shared memory), one launch up to max_iter.
static int run_warp64(opf_handle *h, const opf_solve_opts &o) {
    const double rho = o.rho;
    TRY(set_recip(h, rho));
    launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    IterArgs<double> a = with_warp_plan(h, iter_args<double>(h, rho), h->w64);
    if (launch_warp_engine<double>(a, h->w64.lay, h->w64.d_pr, h->d_u64, o.max_iter, o.check_every, h->d_st, rho,
                                   cudaGraphConditionalHandle{}, 0, h->stream)) {
        g_last_error = std::string("warp engine launch failed: ") + cudaGetErrorString(cudaGetLastError());
        return OPF_E_CUDA;
    }
    CUDA_TRY(cudaGetLastError());
    TRY(read_status(h));
    h->have_prev_u = h->h_st->iter > 0;
    return OPF_OK;
}

// FP64 iterations on the engine chosen for the solve: 4 persistent grid,
// 3 warp engine, else whole-grid kernels.
static int run_fp64(opf_handle *h, const opf_solve_opts &o, int e64) {
    if (e64 == 4 && h->p64.ok) return run_persist64(h, o);
    if (e64 == 3 && h->w64.ok) return run_warp64(h, o);
    return run_grid64(h, o);
}

// FP32 iterations in the shifted frame, re-centred in FP64 every R iterations.
// eng: 1 whole-grid kernels, 2 cluster engine, 3 warp engine, 4 persistent grid
static int run_mixed(opf_handle *h, const opf_solve_opts &o, int eng, bool recenter) {
    const double rho = o.rho;
    TRY(set_recip(h, rho));
    const int L = h->L, G = h->G, S = h->S;
    const int k = o.check_every;
    int R = o.recenter_every > 0 ? o.recenter_every : 1000;
    R = std::max(k, (R / k) * k);
    if (!recenter) R = std::max(k, (std::min(o.max_iter, 1 << 30) / k + 1) * k);
    // reference = next global update of the current FP64 state; lambda_ref = lambda
    launch_make_u<double>(L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    launch_global_x<double>(G, h->d_gseg, h->d_u64, h->d_c64, h->d_lb64, h->d_ub64, h->d_zeroG, h->d_c64,
                            rho, h->d_xr, h->d_objpart, nullptr, h->stream);
    launch_enter_shift(L, h->d_gk, h->d_xr, h->d_ds64, h->d_mu64, h->d_ds32, h->d_mu32, h->d_lamr, h->stream);
    launch_recenter<float>(L, G, S, h->d_gk, h->d_xr, h->d_xr, h->d_ds32, h->d_mu32, h->d_lamr,
                           h->d_gseg, h->d_uslot, h->d_c64, h->d_lb64, h->d_ub64, h->d_ct32, h->d_lbt32,
                           h->d_ubt32, h->d_sub, h->d_sub2, h->d_F64, h->d_bbar64, rho, h->d_bt32,
                           nullptr, h->stream);
    launch_make_u<float>(L, h->d_pk, h->d_ds32, h->d_mu32, (float)rho, h->d_u32, nullptr, h->stream);
    CUDA_TRY(cudaGetLastError());

    const int kind = eng + (recenter ? 0 : 8);
    bool hl = (o.flags & OPF_SOLVE_HOST_LOOP) != 0 || (eng == 4 && h->persist_graph_failed);
    IterArgs<float> a = eng == 3   ? with_warp_plan(h, iter_args<float>(h, rho), h->w32)
                        : eng == 4 ? with_persist(iter_args<float>(h, rho), h->p32)
                                   : with_plan(iter_args<float>(h, rho), h->c32);
    int launch_rc = 0;
    auto body = [&](cudaGraphConditionalHandle c, int use) {
            if (eng == 4) {
                const PersistPlan &pp = h->p32;
                launch_rc |= launch_persist_engine<float>(a, pp.lay, pp.ptrs(), h->d_u32, bar_extra(o), R, k,
                                                          h->d_st, rho, c, use, h->stream);
            } else if (eng == 3) {
                launch_warp_engine<float>(a, h->w32.lay, h->w32.d_pr, h->d_u32, R, k, h->d_st, rho, c, use, h->stream);
            } else if (eng == 2) {
                launch_cluster_engine<float>(a, h->c32.lay, h->c32.d_pr, h->d_u32, R, k, h->d_st, rho, c, use,
                                             h->stream);
            } else {
                const int chunks = recenter ? R / k : 1;
                for (int i = 0; i < chunks; ++i) enqueue_grid_chunk<float>(h, a, h->d_u32, k, rho, c, use);
            }
            if (!recenter) return;
            // re-centre on the next global update (u of the last iteration is in buffer 0)
            launch_global_x<float>(G, h->d_gseg, h->d_u32, h->d_ct32, h->d_lbt32, h->d_ubt32, h->d_xr,
                                   h->d_c64, (float)rho, h->d_xr2, h->d_objpart, h->d_st, h->stream);
            launch_recenter<float>(L, G, S, h->d_gk, h->d_xr, h->d_xr2, h->d_ds32, h->d_mu32, h->d_lamr,
                                   h->d_gseg, h->d_uslot, h->d_c64, h->d_lb64, h->d_ub64, h->d_ct32,
                                   h->d_lbt32, h->d_ubt32, h->d_sub, h->d_sub2, h->d_F64, h->d_bbar64, rho,
                                   h->d_bt32, h->d_st, h->stream);
            launch_copy_if_running(G, h->d_xr2, h->d_xr, h->d_st, h->stream);
            launch_make_u<float>(L, h->d_pk, h->d_ds32, h->d_mu32, (float)rho, h->d_u32, h->d_st, h->stream);
    };
    const int planP = eng == 4 ? 10000 + h->p32.P : eng == 3 ? 100 + h->w32.P : eng == 2 ? h->c32.P : 0;
    if (h->gmix.kind != kind || h->gmix.rho != rho || h->gmix.k != k || h->gmix.R != R ||
        h->gmix.host_loop != hl || h->gmix.P != planP) {
        int rc = build_while_graph(h, &h->gmix, body, hl);
        if (rc != OPF_OK && eng == 4 && !hl) {
            // a cooperative launch that cannot be captured: drive it from the host
            cudaGetLastError();
            h->persist_graph_failed = true;
            hl = true;
            launch_rc = 0;
            rc = build_while_graph(h, &h->gmix, body, true);
        }
        TRY(rc);
        h->gmix.kind = kind; h->gmix.rho = rho; h->gmix.k = k; h->gmix.R = R;
        h->gmix.P = planP;
    }
    TRY(run_graph(h, &h->gmix, body));
    if (launch_rc) {
        g_last_error = "persistent grid engine launch failed";
        return OPF_E_CUDA;
    }
    TRY(fault_error(h));
    // back to the unshifted FP64 state
    launch_unshift<float>(L, h->d_gk, h->d_xr, h->d_lamr, h->d_ds32, h->d_mu32, h->d_ds64, h->d_mu64, h->stream);
    CUDA_TRY(cudaGetLastError());
    TRY(read_status(h));
    h->have_prev_u = false;
    return OPF_OK;
}

static opf_solve_opts default_opts() {
    opf_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.rho = 100.0;
    o.eps_rel = 1e-8;
    o.eps_abs_pres = 1e-4;
    o.max_iter = 1000000;
    o.check_every = 50;
    o.precision = OPF_PREC_FP64;
    return o;
}

extern "C" int opf_solve_ex(opf_handle *h, const opf_solve_opts *opts) {
    if (!h) return OPF_E_INVALID;
    if (!h->precomputed) return OPF_E_STATE;
    opf_solve_opts o = opts ? *opts : default_opts();
    const bool bad_cluster = o.engine == 4   ? (o.cluster < 0 || o.cluster > kPersistMaxP)
                             : o.engine == 3 ? (o.cluster < 0 || o.cluster > 16)
                                             : (o.cluster < 0 || o.cluster > 16 || (o.cluster & (o.cluster - 1)));
    if (!(o.rho > 0) || o.max_iter < 1 || o.check_every < 2 || (o.check_every & 1) ||
        o.precision < 0 || o.precision > 2 || o.engine < 0 || o.engine > 4 || bad_cluster ||
        std::isnan(o.eps_rel) || std::isnan(o.eps_abs_pres)) {
        g_last_error = "solve options: need rho > 0, max_iter >= 1, even check_every >= 2";
        return OPF_E_INVALID;
    }
    o.max_iter = cap_at_tests(o.max_iter, o.check_every);
    CUDA_TRY(cudaSetDevice(h->device));
    h->last_rho = o.rho;
    TRY(set_status(h, o, false));
    CUDA_TRY(cudaEventRecord(h->ev[1], h->stream));
    // FP64 iterations (plain solves and the polish): on the warp engine when
    // asked for, or automatically when the instance fits one cluster of it
    // with at most 4 warps per CTA (with more, the warps of an SM queue on its
    // FP64 pipe); else on the persistent grid engine when asked for, or
    // automatically when its plan fits (123 buses: 5.5 us per iteration
    // against 7.3 us for whole-grid kernels); else whole-grid kernels
    bool w64 = false, p64 = false;
    if (o.precision != OPF_PREC_FP32 && (o.engine == 0 || o.engine == 3)) {
        const int req = o.engine == 3 ? o.cluster : 0;
        if (!h->w64.built || h->w64.req != req) TRY(build_warp_plan<double>(h, h->w64, req));
        w64 = h->w64.ok && (o.engine == 3 || h->w64.lay.warps <= kWarpEngineWarps64);
    }
    if (!w64 && (o.engine == 4 || (o.engine == 0 && o.precision != OPF_PREC_FP32))) {
        TRY(get_persist_plan<double>(h, &h->p64, o.engine == 4 ? o.cluster : 0));
        if (!h->p64.ok && o.engine == 4 && o.cluster > 0) TRY(get_persist_plan<double>(h, &h->p64, 0));
        p64 = h->p64.ok;
    }
    const int e64 = w64 ? 3 : p64 ? 4 : 1;
    if (o.precision == OPF_PREC_FP64) {
        bool cl = false;
        if (o.engine == 2) {
            TRY(get_cluster_plan<double>(h, &h->c64, o.cluster, 96));
            cl = h->c64.ok;
        }
        if (o.engine == 3 && !w64) { g_last_error = "instance does not fit the warp engine in FP64"; return OPF_E_CAPACITY; }
        if (o.engine == 2 && !cl) { g_last_error = "instance does not fit one cluster in FP64"; return OPF_E_CAPACITY; }
        if (o.engine == 4 && !p64) {
            g_last_error = "instance does not fit the persistent grid engine in FP64";
            return OPF_E_CAPACITY;
        }
        if (cl) TRY(run_cluster64(h, o));
        else TRY(run_fp64(h, o, e64));
        h->main_iters = h->h_st->iter;
        h->recenters = 0;
        CUDA_TRY(cudaEventRecord(h->ev[2], h->stream));
        CUDA_TRY(cudaEventRecord(h->ev[3], h->stream));
    } else {
        int eng = 1;
        if (o.engine == 0 || o.engine == 3) {
            const int req = o.engine == 3 ? o.cluster : 0;
            if (!h->w32.built || h->w32.req != req) TRY(build_warp_plan<float>(h, h->w32, req));
            if (h->w32.ok) eng = 3;
        }
        if (eng == 1 && (o.engine == 0 || o.engine == 2)) {
            TRY(get_cluster_plan<float>(h, &h->c32, o.cluster, 192));
            if (h->c32.ok) eng = 2;
        }
        if (eng == 1 && (o.engine == 0 || o.engine == 4)) {
            TRY(get_persist_plan<float>(h, &h->p32, o.engine == 4 ? o.cluster : 0));
            if (h->p32.ok) eng = 4;
        }
        if ((o.engine == 2 || o.engine == 3 || o.engine == 4) && eng != o.engine) {
            g_last_error = "instance does not fit the requested resident engine";
            return OPF_E_CAPACITY;
        }
        TRY(run_mixed(h, o, eng, o.precision == OPF_PREC_MIXED));
        h->main_iters = h->h_st->iter;
        {
            int R = o.recenter_every > 0 ? o.recenter_every : 1000;
            R = std::max(o.check_every, (R / o.check_every) * o.check_every);
            // one re-centring per completed body of R iterations before the stop
            h->recenters = o.precision == OPF_PREC_MIXED ? (h->main_iters - 1) / R : 0;
        }
        CUDA_TRY(cudaEventRecord(h->ev[2], h->stream));
        if (o.precision == OPF_PREC_FP32) {
            // global x of the last FP32 state, evaluated in FP64
            launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, o.rho, h->d_u64 + h->L, nullptr, h->stream);
            CUDA_TRY(cudaGetLastError());
            h->have_prev_u = true;
        }
        if (o.precision == OPF_PREC_MIXED && !h->h_st->numeric) {
            // FP64 polish: continue in FP64 until the test holds there too
            long long it = h->h_st->iter;
            h->h_st->done = 0;
            DevStatus st = *h->h_st;
            st.done = 0; st.converged = 0; st.iter = it;
            st.max_iter = std::max<long long>(o.max_iter, it + o.check_every);
            *h->h_st = st;
            CUDA_TRY(cudaMemcpyAsync(h->d_st, h->h_st, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
            TRY(run_fp64(h, o, e64));
        }
        CUDA_TRY(cudaEventRecord(h->ev[3], h->stream));
    }
    CUDA_TRY(cudaEventSynchronize(h->ev[3]));
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, h->ev[1], h->ev[2]);
    cudaEventElapsedTime(&b, h->ev[2], h->ev[3]);
    h->timing[1] = a;
    h->timing[2] = b;
    h->timing[3] = (double)h->main_iters;
    h->timing[4] = (double)(h->h_st->iter - h->main_iters);
    h->timing[5] = (double)h->recenters;
    h->total_iters = h->h_st->iter;
    if (h->h_st->numeric) { g_last_error = "NaN or Inf in the residuals"; return OPF_E_NUMERIC; }
    return h->h_st->converged ? OPF_OK : OPF_NOT_CONVERGED;
}

extern "C" int opf_solve(opf_handle *h, double rho, double eps, int32_t max_iter) {
    opf_solve_opts o = default_opts();
    o.rho = rho;
    o.eps_rel = eps;
    o.max_iter = max_iter;
    return opf_solve_ex(h, &o);
}

extern "C" int opf_step(opf_handle *h, double rho, int32_t n_iters) {
    if (!h) return OPF_E_INVALID;
    if (!h->precomputed) return OPF_E_STATE;
    if (!(rho > 0) || n_iters < 0) return OPF_E_INVALID;
    CUDA_TRY(cudaSetDevice(h->device));
    if (n_iters == 0) return OPF_OK;
    h->last_rho = rho;
    opf_solve_opts o = default_opts();
    o.max_iter = 0x7fffffff;
    TRY(set_status(h, o, false));
    TRY(set_recip(h, rho));
    launch_make_u<double>(h->L, h->d_pk, h->d_ds64, h->d_mu64, rho, h->d_u64, nullptr, h->stream);
    IterArgs<double> a = iter_args<double>(h, rho);
    const Tiling &t = h->t64;
    for (int i = 0; i < n_iters; ++i) {
        const double *uin = h->d_u64 + (size_t)(i & 1) * h->L;
        double *uout = h->d_u64 + (size_t)((i + 1) & 1) * h->L;
        launch_iterate<double>(a, uin, uout, h->d_partials, h->d_st, i == n_iters - 1, t.n_tiles, t.block,
                               t.xcap, t.vcap, t.tcap, h->stream);
    }
    launch_check(h->d_partials, t.n_tiles, h->d_st, rho, n_iters, cudaGraphConditionalHandle{}, 0, h->stream);
    CUDA_TRY(cudaGetLastError());
    TRY(read_status(h));
    // make the previous-u buffer be the one at offset L
    if (n_iters & 1) {
        CUDA_TRY(cudaMemcpyAsync(h->d_u64 + h->L, h->d_u64, h->L * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->have_prev_u = true;
    h->total_iters = h->h_st->iter;
    return OPF_OK;
}

extern "C" int opf_get_solution(opf_handle *h, double *x, size_t n, double *objective) {
    if (!h) return OPF_E_INVALID;
    if (!h->have_prev_u) return OPF_E_STATE;
    if (x && n < (size_t)h->G) return OPF_E_INVALID;
    CUDA_TRY(cudaSetDevice(h->device));
    int nb = launch_global_x<double>(h->G, h->d_gseg, h->d_u64 + h->L, h->d_c64, h->d_lb64, h->d_ub64,
                                     h->d_zeroG, h->d_c64, h->last_rho, h->d_x, h->d_objpart, nullptr,
                                     h->stream);
    CUDA_TRY(cudaGetLastError());
    std::vector<double> part(nb);
    CUDA_TRY(cudaMemcpyAsync(part.data(), h->d_objpart, nb * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (x) CUDA_TRY(cudaMemcpyAsync(x, h->d_x, h->G * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    double o = 0.0;
    for (double p : part) o += p;
    if (objective) *objective = o;
    return OPF_OK;
}

extern "C" int opf_get_residuals(opf_handle *h, double *pres, double *dres, double *eps_prim,
                                 double *eps_dual, int64_t *iters) {
    if (!h) return OPF_E_INVALID;
    if (pres) *pres = h->h_st->pres;
    if (dres) *dres = h->h_st->dres;
    if (eps_prim) *eps_prim = h->h_st->eprim;
    if (eps_dual) *eps_dual = h->h_st->edual;
    if (iters) *iters = h->total_iters;
    return OPF_OK;
}

extern "C" int opf_get_locals(opf_handle *h, double *xs, double *lam, size_t L) {
    if (!h) return OPF_E_INVALID;
    if (!h->precomputed) return OPF_E_STATE;
    if (L < (size_t)h->L) return OPF_E_INVALID;
    CUDA_TRY(cudaSetDevice(h->device));
    std::vector<double> a(h->L), b(h->L);
    CUDA_TRY(cudaMemcpyAsync(a.data(), h->d_ds64, h->L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(b.data(), h->d_mu64, h->L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < h->L; ++c) {
        if (xs) xs[c] = a[h->canon_slot_to_dev[c]];
        if (lam) lam[c] = b[h->canon_slot_to_dev[c]];
    }
    return OPF_OK;
}

extern "C" int opf_set_locals(opf_handle *h, const double *xs, const double *lam, size_t L) {
    if (!h || !xs || !lam) return OPF_E_INVALID;
    if (!h->precomputed) return OPF_E_STATE;
    if (L < (size_t)h->L) return OPF_E_INVALID;
    CUDA_TRY(cudaSetDevice(h->device));
    std::vector<double> a(h->L), b(h->L);
    for (int c = 0; c < h->L; ++c) {
        a[h->canon_slot_to_dev[c]] = xs[c];
        b[h->canon_slot_to_dev[c]] = lam[c];
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_ds64, a.data(), h->L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_mu64, b.data(), h->L * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->have_prev_u = false;
    return OPF_OK;
}

extern "C" int opf_get_sizes(opf_handle *h, opf_sizes *out) {
    if (!h || !out) return OPF_E_INVALID;
    out->n_global = h->G;
    out->n_sub = h->S;
    out->n_slots = h->L;
    out->n_rows = h->n_rows;
    out->sum_nf = h->sum_nf;
    out->max_ns = h->max_ns;
    out->h2d_bytes = h->h2d_bytes;
    return OPF_OK;
}

extern "C" int opf_set_loads(opf_handle *h, const double *load_p, const double *load_q) {
    if (!h || !load_p || !load_q) return OPF_E_INVALID;
    HostModel &M = h->model;
    if (M.n_load == 0) { g_last_error = "loads: the handle was not built from a feeder"; return OPF_E_INVALID; }
    // rows fed by a load value: their rhs and, with a ZIP exponent, their w
    // coefficient (VDLM-1..5); every other row is unchanged
    std::vector<double> b((size_t)h->nB);
    size_t cr = 0;
    bool a_changed = false;
    for (HostSub &sub : M.subs)
        for (int i = 0; i < sub.m; ++i, ++cr) {
            if (i < (int)sub.rsrc.size() && sub.rsrc[i] >= 0) {
                const int src = sub.rsrc[i];
                const double val = ((src & 1) ? load_q : load_p)[src >> 1];
                sub.b[i] = sub.rcoef[i] * val;
                if (sub.acol[i] >= 0) {
                    sub.A[(size_t)i * sub.n + sub.acol[i]] = sub.acoef[i] * val;
                    a_changed = true;
                }
            }
            b[h->canon_row_to_dev[cr]] = sub.b[i];
        }
    CUDA_TRY(cudaSetDevice(h->device));
    CUDA_TRY(cudaMemcpyAsync(h->d_b, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    std::vector<double> A;
    if (a_changed) {
        // A in device subsystem order (the precompute factors it again)
        A.reserve((size_t)h->nA);
        std::vector<int> order(h->S);
        for (int d = 0; d < h->S; ++d) order[d] = h->dev_to_canon_sub[d];
        for (int d = 0; d < h->S; ++d) {
            const HostSub &sub = M.subs[order[d]];
            A.insert(A.end(), sub.A.begin(), sub.A.end());
        }
        CUDA_TRY(cudaMemcpyAsync(h->d_A, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->precomputed = false;
    h->have_pinv = false;
    return OPF_OK;
}

extern "C" int opf_get_timing(opf_handle *h, double *ms, int n) {
    if (!h || !ms) return OPF_E_INVALID;
    for (int i = 0; i < n && i < 6; ++i) ms[i] = h->timing[i];
    return OPF_OK;
}

extern "C" void opf_destroy(opf_handle *h) {
    if (!h) return;
    if (h->device >= 0) cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->g64.reset();
    h->gmix.reset();
    for (void *p : h->allocs) cudaFree(p);
    if (h->h_st) cudaFreeHost(h->h_st);
    for (auto &e : h->ev) if (e) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

extern "C" const char *opf_strerror(int code) {
    switch (code) {
        case OPF_OK: return "ok";
        case OPF_NOT_CONVERGED: return "iteration limit reached before the stopping test held";
        case OPF_E_INVALID: return "invalid argument or malformed input";
        case OPF_E_INFEASIBLE_LOCAL: return "inconsistent local system A_s x_s = b_s";
        case OPF_E_STATE: return "call out of order";
        case OPF_E_OOM: return "out of memory";
        case OPF_E_NUMERIC: return "NaN or Inf in the residuals";
        case OPF_E_TIMEOUT: return "bounded device wait gave up";
        case OPF_E_CUDA: return "CUDA runtime error";
        case OPF_E_CAPACITY: return "size beyond a documented limit";
        default: return "unknown status";
    }
}

extern "C" const char *opf_last_error(void) { return g_last_error.c_str(); }
