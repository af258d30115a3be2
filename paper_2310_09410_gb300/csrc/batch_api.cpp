// Batched solves (C ABI opf_batch_*): many instances of one model that share
// A_s, c and the bounds and differ in their right-hand sides b (load
// scenarios of one feeder under constant-power loads, Sec. II-A).
//
// Plan (per arithmetic type): a CTA owns K instances (engine columns); the
// subsystems are packed into warp tasks of J = 32 / K member positions (a
// subsystem with more than 4 NQ slots spans p = 2, 4, .. positions), tasks
// are spread over the W warps of the CTA by longest-first list scheduling,
// and the factors are repacked per task so that one 16-byte shared-memory
// load serves the 4 consecutive slots of a lane.  The FP32 plan is picked by
// timing the candidate shapes on the batch itself (autotune).
//
// Solve: CUDA graph "while (an instance runs) { re-centre; engine for R
// iterations with the test every k; back to FP64 }" in FP32, then the same
// loop in FP64 (the polish) until every instance passes the test in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "batch_tables.h"

namespace opf {
template <typename T> int batch_engine_prepare(int K, int nq, bool fg, bool tm, unsigned bytes);
template <typename T>
int batch_engine_launch(const BatchArgs<T> &a, int nq, bool fg, int ctas, int threads, unsigned bytes, int n_iters,
                        int check_every, cudaStream_t s);
template <typename T> int batch_engine_max_ctas_per_sm(int K, int nq, bool fg, bool tm, int threads, unsigned bytes);
void launch_bwarm(int i0, int cnt, int L, const double *xs0, const double *lam0, double *xs, double *lam,
                  cudaStream_t s);
void launch_binit(int i0, int cnt, int L, const int *gk, const double *x0, double *xs, double *lam,
                  DevStatus *st, long long max_iter, double eps_rel, double eps_abs, cudaStream_t s);
void launch_bfill(int cnt, int nrows, const double *b0, double *rhs, cudaStream_t s);
void launch_brhs_perm(int i0, int cnt, int nrows, const int *c2d, const double *src, double *rhs, cudaStream_t s);
void launch_brhs_loads(int i0, int cnt, int nrows, int nload, const int *rsrc, const double *rcoef,
                       const double *b0, const double *lp, const double *lq, double *rhs, cudaStream_t s);
void launch_bbar(int i0, int cnt, int L, const int *meta, const int *sm, const int *boff, const long long *pioff,
                 const double *pinv, int nrows, const double *rhs, double *bbar, cudaStream_t s);
void launch_bconsistent(int i0, int cnt, int S, const int *sm, const int *boff, const long long *toff,
                        const int *nrej, const double *Tw, int nrows, const double *rhs, int *bad, cudaStream_t s);
template <typename T>
void launch_bref(int n_inst, int S, int G, int L, int K, int kshift, int NCH, int NB, const int *ipos,
                 const int2 *gseg, const int *uslot, const int *bidx, const double *c64, const double *lb,
                 const double *ub, double rho, const double *xsv, const double *lam, DevStatus *st,
                 double *xref, double *dref, T *ct, T *xrf, T *lbt, T *ubt, T *cbt, const int4 *sub,
                 const int4 *sub2, const double *F64, const int *gk, const int *sch, const double *bbar, T *bt,
                 T *ds, T *mu, T *lref, cudaStream_t s);
template <typename T>
void launch_bunshift(int n_inst, int G, int L, int K, int kshift, int NCH, const int *ipos, const int *gk,
                     const int *sch, const double *xref, const double *dref, const T *ds, const T *mu, const T *xo,
                     const DevStatus *st, double *xsv, double *lam, double *x, cudaStream_t s);
void launch_bany(int n_inst, const int *ipos, DevStatus *st, int *flag, cudaGraphConditionalHandle cond,
                 int use_cond, cudaStream_t s);
void launch_bobjective(int n_inst, int G, const double *c64, const double *x, double *obj, cudaStream_t s);
void launch_brestart(int n_inst, DevStatus *st, long long add_max, cudaStream_t s);
template <typename T>
void launch_bpack(int n_tasks, int J, const BatchTask *tasks, const int *memb, const int4 *sub, const int4 *sub2,
                  const double *F64, T *dst, cudaStream_t s);
}  // namespace opf

namespace opf {
namespace bx {


int ilog2(int x) {
    int l = 0;
    while ((1 << l) < x) ++l;
    return l;
}

// Builds the tables of a plan with K instance columns, W warps and NQ chunks
// per lane; returns OPF_E_CAPACITY when the shape cannot hold the model.
int build_plan(opf_batch *b, BPlan *p, bool dbl, int K, int W, int nq, bool fg) {
    opf_handle *h = b->h;
    cudaStream_t st = h->stream;
    p->release();
    p->dbl = dbl;
    p->fg = fg;
    p->K = K; p->ks = ilog2(K); p->J = 32 / K; p->W = W; p->nq = nq; p->threads = 32 * W;
    const int J = p->J, S = h->S, L = h->L, G = h->G;
    const size_t sz = dbl ? sizeof(double) : sizeof(float);
    // warp tasks, tensor-memory quadrants, chunk and slot tables (batch_tables.h)
    TaskPlan tp;
    const int trc = build_task_plan(S, L, h->h_npad, h->h_sf, h->h_mode, h->h_soff, h->h_sn, h->h_gk, K, nq,
                                    !dbl && b->allow_tmem && W % 4 == 0, &tp);
    if (trc == 1) { set_last_error("batch plan: a subsystem needs more lanes than a task has"); return OPF_E_CAPACITY; }
    if (trc) { set_last_error("batch plan: slot without a chunk"); return OPF_E_INVALID; }
    std::vector<BatchTask> &tasks = tp.tasks;
    std::vector<int> &memb = tp.memb, &sch = tp.sch;
    std::vector<int4> chg(tp.chg.size() / 4);
    for (size_t c = 0; c < chg.size(); ++c)
        chg[c] = make_int4(tp.chg[4 * c], tp.chg[4 * c + 1], tp.chg[4 * c + 2], tp.chg[4 * c + 3]);
    p->tm = tp.tm;
    p->tm_cols = tp.tm_cols;
    for (int q = 0; q < 5; ++q) p->qstart[q] = tp.qstart[q];
    p->NCH = tp.NCH;
    p->nF = tp.nF;
    p->n_tasks = (int)tasks.size();
    p->NB = b->NB;
    // slot-array row of every copy (global-major copy order)
    std::vector<int> crow(L);
    for (int i = 0; i < G; ++i) {
        const int s0 = h->h_gstart[i], cnt = h->h_gstart[i + 1] - s0;
        for (int q = 0; q < cnt; ++q) {
            const int pos = sch[h->h_uslot[s0 + q]];
            const int ch = pos >> 2, e = pos & 3;
            crow[s0 + q] = (ch * 4 + (e ^ (ch & 3))) * K;
        }
    }
    // global-update tables (batch_tables.h): gperm, the computed globals'
    // entries, later-copy rows and every global's first row
    GlobalTables gt;
    if (!build_global_tables(G, h->h_gstart, crow, b->h_bidx, &gt)) {
        set_last_error("batch plan: global table");
        return OPF_E_CAPACITY;
    }
    p->Gs = gt.Gs;
    std::vector<int4> gtab(std::max(p->Gs, 1), make_int4(0, 0, 0, -1));
    for (int j = 0; j < p->Gs; ++j)
        gtab[j] = make_int4(gt.gtab[4 * j], gt.gtab[4 * j + 1], gt.gtab[4 * j + 2], gt.gtab[4 * j + 3]);
    const std::vector<int> &gperm = gt.gperm, &uxt = gt.uxt, &gx = gt.gx;
    p->n_uxt = (int)uxt.size();
    // shared memory
    p->off_u = fg ? 0u : a16((size_t)p->nF * sz);
    p->off_gt = p->off_u + a16((size_t)p->NCH * K * 4 * sz);
    p->off_rc = p->off_gt + a16((size_t)p->Gs * sizeof(int4));
    p->off_task = p->off_rc + a16((size_t)kBatchRecip * sz);
    p->off_useg = p->off_task + a16((size_t)p->n_tasks * sizeof(BatchTask));
    p->off_bnd = p->off_useg + a16((size_t)p->n_uxt * sizeof(int));
    p->off_red = p->off_bnd + a16((size_t)b->NB * 3 * K * sz);
    p->off_flag = p->off_red + a16((size_t)W * K * 6 * sizeof(double));
    p->bytes = p->off_flag + a16((size_t)(2 * K + 4) * sizeof(int));
    if (p->bytes > kMaxSmem) { set_last_error("batch plan: shared memory"); return OPF_E_CAPACITY; }
    const int rc = dbl ? batch_engine_prepare<double>(K, nq, fg, p->tm, p->bytes)
                       : batch_engine_prepare<float>(K, nq, fg, p->tm, p->bytes);
    if (rc) { set_last_error("batch plan: engine attributes"); return OPF_E_CUDA; }
    const int occ = dbl ? batch_engine_max_ctas_per_sm<double>(K, nq, fg, p->tm, p->threads, p->bytes)
                        : batch_engine_max_ctas_per_sm<float>(K, nq, fg, p->tm, p->threads, p->bytes);
    if (occ < 1) { set_last_error("batch plan: the engine does not fit an SM"); return OPF_E_CAPACITY; }
    // columns
    p->C = (b->n + K - 1) / K;
    std::vector<int> inst((size_t)p->C * K, -1), ipos(b->n);
    for (int i = 0; i < b->n; ++i) { inst[i] = i; ipos[i] = i; }
    // device tables
    std::vector<void *> &A = p->allocs;
    BTRY(bupload(A, &p->d_tasks, tasks, st));
    BTRY(bupload(A, &p->d_memb, memb, st));
    BTRY(bupload(A, &p->d_sch, sch, st));
    BTRY(bupload(A, &p->d_uxt, uxt, st));
    BTRY(bupload(A, &p->d_gx, gx, st));
    BTRY(bupload(A, &p->d_chg, chg, st));
    BTRY(bupload(A, &p->d_gtab, gtab, st));
    BTRY(bupload(A, &p->d_gperm, gperm, st));
    BTRY(bupload(A, &p->d_inst, inst, st));
    BTRY(bupload(A, &p->d_ipos, ipos, st));
    const size_t nslot = (size_t)p->C * p->NCH * K * 4, nglob = (size_t)p->C * G * K;
    const size_t nbnd = (size_t)p->C * std::max(p->NB, 1) * K;
    auto arr = [&](void **q, size_t n) -> int {
        if (dbl) { double *t; BTRY(balloc(A, &t, n)); *q = t; }
        else { float *t; BTRY(balloc(A, &t, n)); *q = t; }
        BCUDA(cudaMemsetAsync(*q, 0, n * sz, st));
        return OPF_OK;
    };
    BTRY(arr(&p->d_F, (size_t)p->nF));
    BTRY(arr(&p->d_recip, (size_t)kBatchRecip));
    BTRY(arr(&p->d_cost, (size_t)G));
    BTRY(arr(&p->mu, nslot)); BTRY(arr(&p->ds, nslot)); BTRY(arr(&p->bt, nslot)); BTRY(arr(&p->lref, nslot));
    BTRY(arr(&p->xo, nglob)); BTRY(arr(&p->ct, nglob)); BTRY(arr(&p->xrf, nglob));
    BTRY(arr(&p->lbt, nbnd)); BTRY(arr(&p->ubt, nbnd)); BTRY(arr(&p->cbt, nbnd));
    if (dbl) launch_bpack<double>(p->n_tasks, J, p->d_tasks, p->d_memb, h->d_sub, h->d_sub2, h->d_F64,
                                  (double *)p->d_F, st);
    else launch_bpack<float>(p->n_tasks, J, p->d_tasks, p->d_memb, h->d_sub, h->d_sub2, h->d_F64,
                             (float *)p->d_F, st);
    BCUDA(cudaGetLastError());
    {
        std::vector<double> c64 = h->model.c;
        if (dbl) BCUDA(cudaMemcpyAsync(p->d_cost, c64.data(), G * sizeof(double), cudaMemcpyHostToDevice, st));
        else {
            std::vector<float> c32(c64.begin(), c64.end());
            BCUDA(cudaMemcpyAsync(p->d_cost, c32.data(), G * sizeof(float), cudaMemcpyHostToDevice, st));
            BCUDA(cudaStreamSynchronize(st));
        }
    }
    BCUDA(cudaStreamSynchronize(st));
    p->rho = -1.0;
    p->ok = true;
    return OPF_OK;
}

constexpr int kBatchRecenter = 4000;
constexpr int kPolishCheck = 2;     // test interval of a mixed solve's FP64 polish

int plan_set_rho(opf_batch *b, BPlan *p, double rho) {
    if (p->rho == rho) return OPF_OK;
    opf_handle *h = b->h;
    const int G = h->G;
    // 1 / (rho N) by copy count N (a global has fewer than kBatchRecip copies)
    (void)G;
    std::vector<double> r(kBatchRecip, 0.0);
    for (int n = 1; n < kBatchRecip; ++n) r[n] = 1.0 / (rho * n);
    if (p->dbl) BCUDA(cudaMemcpyAsync(p->d_recip, r.data(), kBatchRecip * sizeof(double), cudaMemcpyHostToDevice,
                                      h->stream));
    else {
        std::vector<float> f(r.begin(), r.end());
        BCUDA(cudaMemcpyAsync(p->d_recip, f.data(), kBatchRecip * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
    BCUDA(cudaStreamSynchronize(h->stream));
    p->rho = rho;
    p->graph.reset();
    return OPF_OK;
}

template <typename T>
BatchArgs<T> engine_args(opf_batch *b, const BPlan &p, double rho) {
    BatchArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.K = p.K; a.kshift = p.ks; a.J = p.J; a.NCH = p.NCH; a.G = b->G; a.NB = p.NB; a.n_tasks = p.n_tasks;
    a.nF = p.nF;
    a.L = b->L;
    a.off_u = p.off_u; a.off_gt = p.off_gt; a.off_rc = p.off_rc; a.off_task = p.off_task; a.off_useg = p.off_useg;
    a.off_bnd = p.off_bnd;
    a.off_red = p.off_red; a.off_flag = p.off_flag;
    a.tasks = p.d_tasks; a.chg = p.d_chg; a.gtab = p.d_gtab; a.gperm = p.d_gperm; a.Gs = p.Gs;
    a.uxt = p.d_uxt; a.gx = p.d_gx; a.n_uxt = p.n_uxt;
    a.Fpk = (const T *)p.d_F; a.cost = (const T *)p.d_cost;
    a.mu = (T *)p.mu; a.ds = (T *)p.ds; a.xo = (T *)p.xo;
    a.bt = (const T *)p.bt; a.lref = (const T *)p.lref; a.xrf = (const T *)p.xrf;
    a.lbt = (const T *)p.lbt; a.ubt = (const T *)p.ubt; a.cbt = (const T *)p.cbt;
    a.inst = p.d_inst; a.st = b->d_st;
    a.rho = (T)rho; a.inv_rho = (T)(1.0 / rho); a.rho_d = rho;
    a.tm = p.tm ? 1 : 0;
    a.tm_cols = p.tm_cols;
    for (int q = 0; q < 5; ++q) a.qstart[q] = p.qstart[q];
    return a;
}

// One pass of the loop body: re-centre, n_iters engine iterations, unshift,
// "still running" flag (and graph condition).
template <typename T>
void enqueue_body(opf_batch *b, BPlan &p, double rho, int n_iters, int check_every,
                  cudaGraphConditionalHandle cond, int use_cond, cudaEvent_t e0 = nullptr,
                  cudaEvent_t e1 = nullptr, int ctas = -1, cudaStream_t stream = nullptr) {
    opf_handle *h = b->h;
    cudaStream_t s = stream ? stream : h->stream;
    launch_bref<T>(b->n, h->S, b->G, b->L, p.K, p.ks, p.NCH, p.NB, p.d_ipos, h->d_gseg, h->d_uslot, b->d_bidx,
                   h->d_c64, h->d_lb64, h->d_ub64, rho, b->d_xs, b->d_lam, b->d_st, b->d_xref, b->d_dref, (T *)p.ct,
                   (T *)p.xrf, (T *)p.lbt, (T *)p.ubt, (T *)p.cbt, h->d_sub, h->d_sub2, h->d_F64, h->d_gk, p.d_sch,
                   b->d_bbar, (T *)p.bt, (T *)p.ds, (T *)p.mu, (T *)p.lref, s);
    if (e0) cudaEventRecord(e0, s);
    const int grid = ctas >= 0 ? std::min(ctas, p.C) : p.C;
    if (p.lane) {
        // tiles of kLaneInst instances, one cluster each
        if (grid > 0)
            lane_engine_launch(lane_args(b, p, rho), grid, p.threads, p.bytes, n_iters, check_every, s);
    } else if (grid > 0) {
        BatchArgs<T> a = engine_args<T>(b, p, rho);
        batch_engine_launch<T>(a, p.nq, p.fg, grid, p.threads, p.bytes, n_iters, check_every, s);
    }
    if (e1) cudaEventRecord(e1, s);
    launch_bunshift<T>(b->n, b->G, b->L, p.K, p.ks, p.NCH, p.d_ipos, h->d_gk, p.d_sch, b->d_xref, b->d_dref,
                       (const T *)p.ds, (const T *)p.mu, (const T *)p.xo, b->d_st, b->d_xs, b->d_lam, b->d_x, s);
    launch_bany(b->n, p.d_ipos, b->d_st, p.dbl ? b->d_flag + 1 : b->d_flag, cond, use_cond, s);
}

void enqueue_body_any(opf_batch *b, BPlan &p, double rho, int n_iters, int k, cudaGraphConditionalHandle c,
                      int use, cudaEvent_t e0, cudaEvent_t e1, int ctas, cudaStream_t stream) {
    if (p.dbl) enqueue_body<double>(b, p, rho, n_iters, k, c, use, e0, e1, ctas, stream);
    else enqueue_body<float>(b, p, rho, n_iters, k, c, use, e0, e1, ctas, stream);
}

int read_status(opf_batch *b) {
    b->h_st.resize(b->n);
    BCUDA(cudaMemcpyAsync(b->h_st.data(), b->d_st, b->n * sizeof(DevStatus), cudaMemcpyDeviceToHost, b->h->stream));
    BCUDA(cudaStreamSynchronize(b->h->stream));
    return OPF_OK;
}

// Runs "while (an instance runs) body" (a WHILE graph, or host relaunches).
int run_loop(opf_batch *b, BPlan &p, double rho, int R, int k, bool host_loop) {
    opf_handle *h = b->h;
    BTRY(plan_set_rho(b, &p, rho));
    if (host_loop) {
        // direct launches; the engine launches are timed alone with events
        for (;;) {
            enqueue_body_any(b, p, rho, R, k, cudaGraphConditionalHandle{}, 0, b->eng_ev[0], b->eng_ev[1]);
            BCUDA(cudaGetLastError());
            int flag = 0;
            BCUDA(cudaMemcpyAsync(&flag, p.dbl ? b->d_flag + 1 : b->d_flag, sizeof(int), cudaMemcpyDeviceToHost,
                                  h->stream));
            BCUDA(cudaStreamSynchronize(h->stream));
            float ms = 0;
            cudaEventElapsedTime(&ms, b->eng_ev[0], b->eng_ev[1]);
            b->engine_ms[p.dbl ? 1 : 0] += ms;
            b->bodies[p.dbl ? 1 : 0] += 1;
            if (!flag) return OPF_OK;
        }
    }
    GraphCache &gc = p.graph;
    if (!gc.exec || gc.rho != rho || gc.k != k || gc.R != R) {
        gc.reset();
        BCUDA(cudaGraphCreate(&gc.graph, 0));
        cudaGraphConditionalHandle cond;
        BCUDA(cudaGraphConditionalHandleCreate(&cond, gc.graph, 1, cudaGraphCondAssignDefault));
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams *cp = reinterpret_cast<cudaGraphNodeParams *>(raw);
        cp->type = cudaGraphNodeTypeConditional;
        cp->conditional.handle = cond;
        cp->conditional.type = cudaGraphCondTypeWhile;
        cp->conditional.size = 1;
        cudaGraphNode_t node;
        BCUDA(cudaGraphAddNode(&node, gc.graph, nullptr, nullptr, 0, cp));
        cudaGraph_t body = cp->conditional.phGraph_out[0];
        BCUDA(cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        enqueue_body_any(b, p, rho, R, k, cond, 1);
        cudaGraph_t captured = nullptr;
        cudaError_t ec = cudaStreamEndCapture(h->stream, &captured);
        if (ec != cudaSuccess) {
            set_last_error(std::string("stream capture: ") + cudaGetErrorString(ec));
            gc.reset();
            return OPF_E_CUDA;
        }
        BCUDA(cudaGraphInstantiate(&gc.exec, gc.graph, 0));
        gc.rho = rho; gc.k = k; gc.R = R;
    }
    // the WHILE node tests its condition before the first pass: start it set
    // only when some instance runs (the first body pass recomputes it)
    BCUDA(cudaGraphLaunch(gc.exec, h->stream));
    BCUDA(cudaStreamSynchronize(h->stream));
    // passes of the loop: every pass runs R iterations of the instances still
    // running, so the longest-running instance decides their number
    BTRY(read_status(b));
    long long most = 0;
    for (const DevStatus &st : b->h_st) most = std::max(most, st.iter - b->iter_base[p.dbl ? 1 : 0]);
    b->bodies[p.dbl ? 1 : 0] += std::max(1LL, (most + R - 1) / R);
    return OPF_OK;
}

// Plans: FP32 shapes tried on the batch (fastest wins) unless fixed by
// opf_batch_set_shape; FP64 uses the largest K <= 4 that fits.
int ensure_plan(opf_batch *b, bool dbl, double rho, int k) {
    BPlan &p = dbl ? b->p64 : b->p32;
    if (p.ok) return OPF_OK;
    opf_handle *h = b->h;
    if (dbl) {
        // factors in shared memory when they fit, else read through L1/L2 (the
        // FP64 iteration is bound by the FP64 FMA rate either way)
        const int fk = b->force_k64, fw = b->force_w64 > 0 ? b->force_w64 : 16;
        const int ks[] = {4, 2, 1};
        for (int fg = 0; fg < 2; ++fg)
            for (int K : ks) {
                if (fk && K != fk) continue;
                if (build_plan(b, &p, true, K, fw, 2, fg != 0) == OPF_OK) return OPF_OK;
            }
        p.release();
        set_last_error("batch: no FP64 engine shape fits");
        return OPF_E_CAPACITY;
    }
    // candidates (K, W); K = kLaneInst (the lane engine, W / 4 warps per lane
    // quadrant) only when asked for: it measured several times slower than
    // these shapes on the feeders it holds
    std::vector<std::pair<int, int>> cand;
    if (b->force_k32) cand.push_back({b->force_k32, b->force_w32 > 0 ? b->force_w32 : 16});
    else {
        const int Ks[] = {8, 4, 2};
        const int Ws[] = {16, 12, 8};
        for (int K : Ks) for (int W : Ws) cand.push_back({K, W});
    }
    auto build = [&](int K, int W) -> int {
        if (K == kLaneInst) return build_lane_plan(b, &p, W / 4, 16);
        return build_plan(b, &p, false, K, W, 4, false);
    };
    b->tune_log.clear();
    if (cand.size() == 1) {
        BTRY(build(cand[0].first, cand[0].second));
        return OPF_OK;
    }
    // timing runs on a copy of the status; the FP64 state is not touched by
    // the engine (it works on the plan's own arrays)
    BCUDA(cudaMemcpyAsync(b->d_st_save, b->d_st, b->n * sizeof(DevStatus), cudaMemcpyDeviceToDevice, h->stream));
    double best = 1e300;
    int bk = 0, bw = 0;
    const int iters = 2 * std::max(k, 2);
    for (auto &c : cand) {
        if (build(c.first, c.second) != OPF_OK) continue;
        BTRY(plan_set_rho(b, &p, rho));
        launch_bref<float>(b->n, h->S, b->G, b->L, p.K, p.ks, p.NCH, p.NB, p.d_ipos, h->d_gseg, h->d_uslot,
                           b->d_bidx, h->d_c64, h->d_lb64, h->d_ub64, rho, b->d_xs, b->d_lam, b->d_st, b->d_xref,
                           b->d_dref, (float *)p.ct, (float *)p.xrf, (float *)p.lbt, (float *)p.ubt, (float *)p.cbt,
                           h->d_sub, h->d_sub2,
                           h->d_F64, h->d_gk, p.d_sch, b->d_bbar, (float *)p.bt, (float *)p.ds, (float *)p.mu,
                           (float *)p.lref, h->stream);
        auto run = [&](int n_it) {
            if (p.lane) lane_engine_launch(lane_args(b, p, rho), p.C, p.threads, p.bytes, n_it, 0, h->stream);
            else batch_engine_launch<float>(engine_args<float>(b, p, rho), p.nq, false, p.C, p.threads, p.bytes,
                                            n_it, 0, h->stream);
        };
        run(4);   // warm-up
        BCUDA(cudaEventRecord(b->ev[0], h->stream));
        run(iters);
        BCUDA(cudaEventRecord(b->ev[1], h->stream));
        BCUDA(cudaEventSynchronize(b->ev[1]));
        BCUDA(cudaGetLastError());
        float ms = 0;
        cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
        b->tune_log.push_back(c.first);
        b->tune_log.push_back(c.second);
        b->tune_log.push_back(ms);
        if (ms < best) { best = ms; bk = c.first; bw = c.second; }
        BCUDA(cudaMemcpyAsync(b->d_st, b->d_st_save, b->n * sizeof(DevStatus), cudaMemcpyDeviceToDevice, h->stream));
    }
    // the status copies carry the pad (shifted) marks of the timing runs: clear them
    BCUDA(cudaMemcpyAsync(b->d_st, b->d_st_save, b->n * sizeof(DevStatus), cudaMemcpyDeviceToDevice, h->stream));
    if (!bk) { p.release(); set_last_error("batch: no FP32 engine shape fits"); return OPF_E_CAPACITY; }
    BTRY(build(bk, bw));
    return OPF_OK;
}

int check_range(opf_batch *b, int first, int count) {
    if (!b || first < 0 || count < 0 || first > b->n || count > b->n - first) {
        set_last_error("batch: instance range out of bounds");
        return OPF_E_INVALID;
    }
    return OPF_OK;
}

int stage(opf_batch *b, size_t n) {
    if (n <= b->stage_len) return OPF_OK;
    if (b->d_stage) cudaFree(b->d_stage);
    b->d_stage = nullptr;
    b->stage_len = 0;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(double));
    if (e != cudaSuccess) { set_last_error("cudaMalloc (batch staging)"); return OPF_E_OOM; }
    b->d_stage = (double *)q;
    b->stage_len = n;
    return OPF_OK;
}

// bbar, consistency and a fresh start for instances [first, first + count)
// whose rhs is in place.
int after_rhs(opf_batch *b, int first, int count) {
    opf_handle *h = b->h;
    cudaStream_t s = h->stream;
    BCUDA(cudaMemsetAsync(b->d_bad + first, 0, count * sizeof(int), s));
    launch_bconsistent(first, count, h->S, h->d_sm, h->d_boff, h->d_toff, h->d_nrej, h->d_Tw, b->nrows, b->d_rhs,
                       b->d_bad, s);
    launch_bbar(first, count, h->L, h->d_meta, h->d_sm, h->d_boff, h->d_pioff, h->d_pinv, b->nrows, b->d_rhs,
                b->d_bbar, s);
    launch_binit(first, count, h->L, h->d_gk, h->d_x0, b->d_xs, b->d_lam, b->d_st, b->init_max_iter,
                 b->init_eps_rel, b->init_eps_abs, s);
    if (b->d_start) launch_bwarm(first, count, h->L, b->d_start, b->d_start + h->L, b->d_xs, b->d_lam, s);
    BCUDA(cudaGetLastError());
    b->have_x = false;
    // full-row-rank local systems are consistent for every rhs: nothing to read
    bool any_rej = false;
    for (int r : h->h_nrej) any_rej = any_rej || r > 0;
    if (!any_rej) return OPF_OK;
    std::vector<int> bad(count);
    if (count) BCUDA(cudaMemcpyAsync(bad.data(), b->d_bad + first, count * sizeof(int), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
        if (bad[i]) {
            set_last_error("batch: inconsistent local system A_s x_s = b_s for instance " + std::to_string(first + i));
            return OPF_E_INFEASIBLE_LOCAL;
        }
    b->have_x = false;
    return OPF_OK;
}

int write_status(opf_batch *b, int first, int count) {
    BCUDA(cudaMemcpyAsync(b->d_st + first, b->h_st.data() + first, count * sizeof(DevStatus), cudaMemcpyHostToDevice,
                          b->h->stream));
    return OPF_OK;
}

}  // namespace bx
}  // namespace opf

int opf::bx::set_loads_impl(opf_batch *b, int first, int count, const double *load_p, const double *load_q,
                            bool on_device) {
    BTRY(check_range(b, first, count));
    if (count == 0) return OPF_OK;
    opf_handle *h = b->h;
    const int nl = h->model.n_load;
    if (nl == 0 || !load_p || !load_q) { set_last_error("batch: loads need a feeder model and both arrays"); return OPF_E_INVALID; }
    if (h->model.A_depends_on_loads) {
        set_last_error("batch: a ZIP load exponent makes A_s depend on the load values (one handle per instance)");
        return OPF_E_INVALID;
    }
    BCUDA(cudaSetDevice(h->device));
    const size_t n = (size_t)count * nl * 3;
    const double *lp = load_p, *lq = load_q;
    if (!on_device) {
        BTRY(stage(b, 2 * n));
        BCUDA(cudaMemcpyAsync(b->d_stage, load_p, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        BCUDA(cudaMemcpyAsync(b->d_stage + n, load_q, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        lp = b->d_stage;
        lq = b->d_stage + n;
    }
    launch_brhs_loads(first, count, b->nrows, nl, b->d_rsrc, b->d_rcoef, b->d_b0, lp, lq, b->d_rhs, h->stream);
    BCUDA(cudaGetLastError());
    return after_rhs(b, first, count);
}

using namespace opf::bx;

extern "C" {

int opf_batch_create(opf_handle *h, int32_t n_inst, opf_batch **out) {
    if (!h || !out || n_inst < 1) { set_last_error("batch: need a handle, n_inst >= 1"); return OPF_E_INVALID; }
    *out = nullptr;
    if (!h->precomputed) return OPF_E_STATE;
    BCUDA(cudaSetDevice(h->device));
    BTRY(ensure_pinv(h));
    opf_batch *b = new opf_batch();
    b->h = h;
    b->n = n_inst;
    b->G = h->G; b->L = h->L; b->S = h->S; b->nrows = (int)h->n_rows;
    auto fail = [&](int rc) { opf_batch_destroy(b); return rc; };
    const size_t n = n_inst, L = h->L, G = h->G, R = h->n_rows;
    std::vector<void *> &A = b->allocs;
    int rc = OPF_OK;
    if ((rc = balloc(A, &b->d_rhs, n * R)) || (rc = balloc(A, &b->d_bbar, n * L)) || (rc = balloc(A, &b->d_xs, n * L)) ||
        (rc = balloc(A, &b->d_lam, n * L)) || (rc = balloc(A, &b->d_xref, n * G)) ||
        (rc = balloc(A, &b->d_dref, n * G)) || (rc = balloc(A, &b->d_x, n * G)) ||
        (rc = balloc(A, &b->d_obj, n)) || (rc = balloc(A, &b->d_st, n)) || (rc = balloc(A, &b->d_st_save, n)) ||
        (rc = balloc(A, &b->d_flag, 2)) || (rc = balloc(A, &b->d_bad, n)))
        return fail(rc);
    // rhs sources (device row order) and bounded globals
    std::vector<int> rsrc(R, -1);
    std::vector<double> rcoef(R, 0.0), b0(R, 0.0);
    {
        // canonical rows in canonical subsystem order map to device rows
        size_t cr = 0;
        for (const HostSub &s : h->model.subs)
            for (int i = 0; i < s.m; ++i, ++cr) {
                const int dr = h->canon_row_to_dev[cr];
                b0[dr] = s.b[i];
                if (i < (int)s.rsrc.size()) { rsrc[dr] = s.rsrc[i]; rcoef[dr] = s.rcoef[i]; }
            }
    }
    b->h_bidx.assign(G, -1);
    b->NB = 0;
    for (size_t i = 0; i < G; ++i)
        if (std::isfinite(h->model.lb[i]) || std::isfinite(h->model.ub[i])) b->h_bidx[i] = b->NB++;
    if ((rc = bupload(A, &b->d_rsrc, rsrc, h->stream)) || (rc = bupload(A, &b->d_rcoef, rcoef, h->stream)) ||
        (rc = bupload(A, &b->d_b0, b0, h->stream)) || (rc = bupload(A, &b->d_c2d, h->canon_row_to_dev, h->stream)) ||
        (rc = bupload(A, &b->d_bidx, b->h_bidx, h->stream)))
        return fail(rc);
    for (int i = 0; i < 4; ++i)
        if (cudaEventCreate(&b->ev[i]) != cudaSuccess) { set_last_error("cudaEventCreate"); return fail(OPF_E_CUDA); }
    for (int i = 0; i < 2; ++i)
        if (cudaEventCreate(&b->eng_ev[i]) != cudaSuccess) { set_last_error("cudaEventCreate"); return fail(OPF_E_CUDA); }
    // every instance starts as a copy of the handle's own right-hand side
    launch_bfill(n_inst, b->nrows, b->d_b0, b->d_rhs, h->stream);
    if ((rc = after_rhs(b, 0, n_inst))) return fail(rc);
    *out = b;
    return OPF_OK;
}

int opf_batch_set_rhs(opf_batch *b, int32_t first, int32_t count, const double *rhs) {
    BTRY(check_range(b, first, count));
    if (count == 0) return OPF_OK;
    if (!rhs) { set_last_error("batch: null rhs"); return OPF_E_INVALID; }
    opf_handle *h = b->h;
    BCUDA(cudaSetDevice(h->device));
    const size_t n = (size_t)count * b->nrows;
    BTRY(stage(b, n));
    BCUDA(cudaMemcpyAsync(b->d_stage, rhs, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    launch_brhs_perm(first, count, b->nrows, b->d_c2d, b->d_stage, b->d_rhs, h->stream);
    BCUDA(cudaGetLastError());
    return after_rhs(b, first, count);
}

int opf_batch_set_loads(opf_batch *b, int32_t first, int32_t count, const double *load_p, const double *load_q) {
    return set_loads_impl(b, first, count, load_p, load_q, false);
}

int opf_batch_set_loads_device(opf_batch *b, int32_t first, int32_t count, const double *load_p,
                               const double *load_q) {
    return set_loads_impl(b, first, count, load_p, load_q, true);
}

int opf_batch_set_shape(opf_batch *b, int32_t precision, int32_t k_inst, int32_t warps) {
    const int wmax = 16;
    const bool lane = precision == OPF_PREC_FP32 && k_inst == kLaneInst;
    if (!b || (precision != OPF_PREC_FP32 && precision != OPF_PREC_FP64) || k_inst < 0 ||
        (!lane && (k_inst > 32 || (k_inst & (k_inst - 1)) || warps < 0 || warps > wmax)) ||
        (lane && (warps < 0 || warps > wmax || warps % 4 != 0))) {
        set_last_error("batch shape: precision FP32 or FP64, K a power of two <= 32 (0: auto), warps <= 16; "
                       "FP32 K = 128: the lane engine, warps 4, 8, 12 or 16");
        return OPF_E_INVALID;
    }
    if (precision == OPF_PREC_FP32) { b->force_k32 = k_inst; b->force_w32 = warps; b->p32.release(); }
    else { b->force_k64 = k_inst; b->force_w64 = warps; b->p64.release(); }
    return OPF_OK;
}

int opf_batch_set_tmem(opf_batch *b, int32_t enable) {
    if (!b) return OPF_E_INVALID;
    b->allow_tmem = enable != 0;
    b->p32.release();
    return OPF_OK;
}

int opf_batch_get_shape(opf_batch *b, int32_t precision, int32_t *out, int32_t n_out) {
    if (!b || !out || n_out < 1) return OPF_E_INVALID;
    const BPlan &p = precision == OPF_PREC_FP64 ? b->p64 : b->p32;
    const int32_t v[11] = {p.ok ? 1 : 0, p.K, p.W, p.nq, p.n_tasks, p.NCH, (int32_t)p.bytes, p.C, p.tm ? 1 : 0,
                           p.tm_cols, p.lane ? p.lane_C : 0};
    for (int i = 0; i < n_out && i < 11; ++i) out[i] = v[i];
    return OPF_OK;
}

int opf_batch_solve(opf_batch *b, const opf_solve_opts *opts) {
    if (!b) return OPF_E_INVALID;
    opf_handle *h = b->h;
    opf_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.rho = 100.0; o.eps_rel = 1e-8; o.eps_abs_pres = 1e-4; o.max_iter = 1000000; o.check_every = 50;
    o.precision = OPF_PREC_MIXED;
    if (opts) o = *opts;
    if (!(o.rho > 0) || o.max_iter < 1 || o.check_every < 2 || (o.check_every & 1) || o.precision < 0 ||
        o.precision > 2 || std::isnan(o.eps_rel) || std::isnan(o.eps_abs_pres)) {
        set_last_error("batch solve options: need rho > 0, max_iter >= 1, even check_every >= 2");
        return OPF_E_INVALID;
    }
    o.max_iter = cap_at_tests(o.max_iter, o.check_every);
    BCUDA(cudaSetDevice(h->device));
    const int k = o.check_every;
    // default interval: 4000 (a batch pays a re-centring pass over every
    // instance; on the 1024 x 123-bus batch 1000 -> 2000 measured 2.6 % less
    // time, then 2000 / 3000 / 4000 / 6000 gave 181.4 / 178.8 / 177.5 / 176.3
    // ms per solve, the same stopping iterations)
    int R = o.recenter_every > 0 ? o.recenter_every : kBatchRecenter;
    R = std::max(k, (R / k) * k);
    const bool hl = (o.flags & OPF_SOLVE_HOST_LOOP) != 0;
    // statuses: fresh test parameters, iteration counts from zero
    BTRY(read_status(b));
    for (DevStatus &s : b->h_st) {
        DevStatus z;
        memset(&z, 0, sizeof(z));
        z.max_iter = o.max_iter;
        z.eps_rel = o.eps_rel;
        z.eps_abs_pres = o.eps_abs_pres;
        s = z;
    }
    BCUDA(cudaMemcpyAsync(b->d_st, b->h_st.data(), b->n * sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
    BCUDA(cudaEventRecord(b->ev[0], h->stream));
    double tune_ms = 0;
    b->bodies[0] = b->bodies[1] = 0;
    b->engine_ms[0] = b->engine_ms[1] = 0;
    b->iter_base[0] = 0;
    if (o.precision != OPF_PREC_FP64) {
        cudaEvent_t t0 = b->ev[2], t1 = b->ev[3];
        const bool tuned_before = b->p32.ok;
        BCUDA(cudaEventRecord(t0, h->stream));
        BTRY(ensure_plan(b, false, o.rho, k));
        BCUDA(cudaEventRecord(t1, h->stream));
        BCUDA(cudaEventSynchronize(t1));
        if (!tuned_before) { float ms = 0; cudaEventElapsedTime(&ms, t0, t1); tune_ms = ms; }
        BCUDA(cudaEventRecord(b->ev[0], h->stream));
        BTRY(run_loop(b, b->p32, o.rho, o.precision == OPF_PREC_MIXED ? R : std::max(k, (std::min(o.max_iter, 1 << 30) / k + 1) * k), k, hl));
    }
    BCUDA(cudaEventRecord(b->ev[1], h->stream));
    if (o.precision != OPF_PREC_FP32) {
        BTRY(ensure_plan(b, true, o.rho, k));
        BTRY(read_status(b));
        long long least = 0;
        for (size_t i = 0; i < b->h_st.size(); ++i) least = i ? std::min(least, b->h_st[i].iter) : b->h_st[i].iter;
        b->iter_base[1] = least;
        // the polish of a mixed solve starts from iterates that already met the
        // test in FP32: it tests every kPolishCheck iterations (at most 2 k of
        // them), so an instance whose FP64 iterates meet the test at once stops
        // after kPolishCheck FP64 iterations instead of k
        const int kp = o.precision == OPF_PREC_MIXED ? std::min(k, kPolishCheck) : k;
        if (o.precision == OPF_PREC_MIXED) launch_brestart(b->n, b->d_st, 2LL * k, h->stream);
        BTRY(run_loop(b, b->p64, o.rho, std::max(kp, (R / kp) * kp), kp, hl));
    }
    launch_bobjective(b->n, b->G, h->d_c64, b->d_x, b->d_obj, h->stream);
    BCUDA(cudaEventRecord(b->ev[2], h->stream));
    BCUDA(cudaEventSynchronize(b->ev[2]));
    BCUDA(cudaGetLastError());
    float a = 0, c = 0;
    cudaEventElapsedTime(&a, b->ev[0], b->ev[1]);
    cudaEventElapsedTime(&c, b->ev[1], b->ev[2]);
    b->timing[0] = a;
    b->timing[1] = c;
    b->timing[2] = tune_ms;
    b->have_x = true;
    BTRY(read_status(b));
    int n_conv = 0, n_num = 0;
    double it_sum = 0;
    for (const DevStatus &s : b->h_st) {
        n_conv += s.converged;
        n_num += s.numeric;
        it_sum += (double)s.iter;
    }
    b->timing[3] = it_sum / b->n;
    b->timing[4] = n_conv;
    b->timing[5] = (double)b->bodies[0];
    b->timing[6] = (double)b->bodies[1];
    b->timing[7] = b->engine_ms[0];
    if (n_num) { set_last_error("batch: NaN or Inf in some instance's residuals"); return OPF_E_NUMERIC; }
    return n_conv == b->n ? OPF_OK : OPF_NOT_CONVERGED;
}

int opf_batch_step(opf_batch *b, double rho, int32_t n_iters) {
    if (!b || !(rho > 0) || n_iters < 0) return OPF_E_INVALID;
    if (n_iters == 0) return OPF_OK;
    opf_handle *h = b->h;
    BCUDA(cudaSetDevice(h->device));
    BTRY(ensure_plan(b, true, rho, 2));
    BTRY(plan_set_rho(b, &b->p64, rho));
    // every instance runs: clear the done marks, keep the counts
    launch_brestart(b->n, b->d_st, (long long)n_iters + 1, h->stream);
    enqueue_body<double>(b, b->p64, rho, n_iters, 0, cudaGraphConditionalHandle{}, 0);
    BCUDA(cudaGetLastError());
    BCUDA(cudaStreamSynchronize(h->stream));
    b->have_x = true;
    return OPF_OK;
}

int opf_batch_get_solution(opf_batch *b, int32_t first, int32_t count, double *x, double *obj) {
    BTRY(check_range(b, first, count));
    if (!b->have_x) { set_last_error("batch: no iteration yet"); return OPF_E_STATE; }
    opf_handle *h = b->h;
    BCUDA(cudaSetDevice(h->device));
    launch_bobjective(b->n, b->G, h->d_c64, b->d_x, b->d_obj, h->stream);
    if (x && count)
        BCUDA(cudaMemcpyAsync(x, b->d_x + (size_t)first * b->G, (size_t)count * b->G * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
    if (obj && count)
        BCUDA(cudaMemcpyAsync(obj, b->d_obj + first, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    BCUDA(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

int opf_batch_get_status(opf_batch *b, int32_t first, int32_t count, double *res, int32_t *iters,
                         int32_t *converged) {
    BTRY(check_range(b, first, count));
    BCUDA(cudaSetDevice(b->h->device));
    BTRY(read_status(b));
    for (int i = 0; i < count; ++i) {
        const DevStatus &s = b->h_st[first + i];
        if (res) { res[4 * i] = s.pres; res[4 * i + 1] = s.dres; res[4 * i + 2] = s.eprim; res[4 * i + 3] = s.edual; }
        if (iters) iters[i] = (int32_t)s.iter;
        if (converged) converged[i] = s.converged;
    }
    return OPF_OK;
}

int opf_batch_set_start(opf_batch *b, const double *xs, const double *lam) {
    if (!b || (!xs) != (!lam)) return OPF_E_INVALID;
    opf_handle *h = b->h;
    BCUDA(cudaSetDevice(h->device));
    const int L = b->L;
    if (!xs) {
        if (b->d_start) cudaFree(b->d_start);
        b->d_start = nullptr;
        return OPF_OK;
    }
    std::vector<double> dev(2 * (size_t)L);
    for (int cs = 0; cs < L; ++cs) {
        const int k = h->canon_slot_to_dev[cs];
        if (!std::isfinite(xs[cs]) || !std::isfinite(lam[cs])) {
            set_last_error("batch start: non-finite entry");
            return OPF_E_INVALID;
        }
        dev[k] = xs[cs];
        dev[(size_t)L + k] = lam[cs];
    }
    if (!b->d_start) {
        void *q = nullptr;
        if (cudaMalloc(&q, 2 * (size_t)L * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_last_error("cudaMalloc (batch start)");
            return OPF_E_OOM;
        }
        b->d_start = (double *)q;
    }
    BCUDA(cudaMemcpyAsync(b->d_start, dev.data(), dev.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    BCUDA(cudaStreamSynchronize(h->stream));
    return OPF_OK;
}

int opf_batch_get_locals(opf_batch *b, int32_t inst, double *xs, double *lam) {
    if (!b || inst < 0 || inst >= b->n || !xs || !lam) return OPF_E_INVALID;
    opf_handle *h = b->h;
    BCUDA(cudaSetDevice(h->device));
    const int L = b->L;
    std::vector<double> a(L), c(L);
    BCUDA(cudaMemcpyAsync(a.data(), b->d_xs + (size_t)inst * L, L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    BCUDA(cudaMemcpyAsync(c.data(), b->d_lam + (size_t)inst * L, L * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    BCUDA(cudaStreamSynchronize(h->stream));
    for (int cs = 0; cs < L; ++cs) {
        const int k = h->canon_slot_to_dev[cs];
        xs[cs] = a[k];
        lam[cs] = c[k];
    }
    return OPF_OK;
}

int opf_batch_get_timing(opf_batch *b, double *out, int32_t n_out) {
    if (!b || !out || n_out < 0) return OPF_E_INVALID;
    for (int i = 0; i < n_out && i < 8; ++i) out[i] = b->timing[i];
    return OPF_OK;
}

int opf_batch_get_tune_log(opf_batch *b, double *out, int32_t n_out) {
    if (!b || n_out < 0) return OPF_E_INVALID;
    for (int i = 0; out && i < n_out && i < (int)b->tune_log.size(); ++i) out[i] = b->tune_log[i];
    return (int)b->tune_log.size();
}

void opf_batch_destroy(opf_batch *b) {
    if (!b) return;
    if (b->h) cudaSetDevice(b->h->device);
    if (b->h) cudaStreamSynchronize(b->h->stream);
    b->p32.release();
    b->p64.release();
    for (void *p : b->allocs) cudaFree(p);
    if (b->d_stage) cudaFree(b->d_stage);
    if (b->d_start) cudaFree(b->d_start);
    for (auto &e : b->ev) if (e) cudaEventDestroy(e);
    for (auto &e : b->eng_ev) if (e) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
