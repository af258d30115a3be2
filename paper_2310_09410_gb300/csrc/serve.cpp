// Request server (C ABI opf_server_*): OPF solves of several feeders and load
// scenarios arriving over time, served with continuous batching.
//
// A model is one feeder topology.  A model whose subsystems fit the batched
// engine gets a batch whose instances are request slots; every pass of
// opf_server_step
//   1. admits queued requests into free slots (slot count bounded by the
//      device-memory budget given at creation),
//   2. advances every running slot on the model's own stream: slots in the
//      FP32 phase by one re-centring interval of FP32 iterations, slots in the
//      FP64 polish by a shorter interval of FP64 iterations (an FP64
//      iteration costs several FP32 ones, and the next pass waits for both),
//   3. moves slots whose FP32 test held to the polish and retires slots whose
//      FP64 test held (or that hit max_iter), freeing them for the next pass.
// Models run on separate streams, so their work overlaps on the device.  An
// instance's arithmetic never involves another slot, and its passes start
// at multiples of the interval from its own admission, so a request gets the
// same result alone or in any mix.
// A model whose subsystems exceed the batched engine (the largest feeders)
// is served by single-instance handles given by the caller, one request per
// handle at a time, each solved by a worker thread.
// Admission (opf_server_set_admission): a model may bound its queue and the
// time a request waits for a slot.  A request is refused at submit when the
// queue is full or when the wait predicted from the model's measured service
// time exceeds the bound, and a queued request that has waited longer than
// the bound is shed; both are counted, and a shed request is reported by
// opf_server_poll_ex with status OPF_E_TIMEOUT, so no request stays pending
// without a status when a model cannot keep up with its arrivals.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "batch_internal.h"

namespace opf {
void launch_bobjective(int n_inst, int G, const double *c64, const double *x, double *obj, cudaStream_t s);
}

using namespace opf;
using namespace opf::bx;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Request {
    int64_t tag;
    std::vector<double> lp, lq;
    double t_submit;
};

struct Done {
    int64_t tag;
    int32_t model, converged, iters, status;
    double objective, t_submit, t_admit, t_done;
    std::vector<double> x;
};

struct Worker {                      // single-instance slot
    opf_handle *h = nullptr;
    std::thread th;
    std::atomic<bool> busy{false}, finished{false};
    double t_admit = 0.0;                 // start of the request it runs (set by the stepping thread)
    Done result;
};

struct Model {
    int id = 0;
    bool batched = false;
    opf_handle *h = nullptr;
    opf_batch *b = nullptr;
    int cap = 0, G = 0, nload = 0;
    size_t slot_bytes = 0;
    double eps_rel = 1e-8, eps_abs = 1e-4;   // stopping test of this model's requests
    std::vector<int> state;          // per slot: 0 free, 1 FP32 phase, 2 FP64 polish
    std::vector<int64_t> tag;
    std::vector<double> t_submit, t_admit;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Worker>> workers;
    std::vector<double> obj;
    bool inflight = false;           // a pass is enqueued and not yet collected
    cudaEvent_t ev = nullptr;        // recorded after the pass (on the model's stream)
    cudaStream_t s64 = nullptr;      // FP64 slots' pass, beside the FP32 slots'
    cudaEvent_t ev64 = nullptr, ev_start = nullptr;
    int n32 = 0, n64 = 0;            // slots in each phase during the pass
    int max_queue = 0;               // admission: queued requests at most (0: no bound)
    double max_wait_s = 0.0;         // admission: seconds a request may wait for a slot (0: no bound)
    double max_service_s = 0.0;      // seconds a request may run once admitted (0: no bound)
    std::vector<double> start_xs, start_lam;   // warm start of worker requests (empty: Sec. V-A point)
    double svc_s = 0.0;              // mean service time (admission to finish) of finished requests
    int64_t n_svc = 0;
    std::atomic<int64_t> n_sub{0}, n_done{0}, n_conv{0}, n_refused{0}, n_shed{0}, n_stopped{0};
    int running() const {
        int n = 0;
        for (int v : state) n += v != 0;
        return n;
    }
};

#define SCUDA(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return e_ == cudaErrorMemoryAllocation ? OPF_E_OOM : OPF_E_CUDA;             \
        }                                                                                \
    } while (0)
#define STRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

}  // namespace

struct opf_server {
    opf_server_opts o{};
    std::vector<std::unique_ptr<Model>> models;
    std::vector<Done> done;          // finished, not yet polled
    std::vector<std::pair<int64_t, std::vector<double>>> kept;   // solutions by tag (keep_solutions)
    std::mutex mu;                   // guards `done` and `kept` (worker threads append)
    int64_t mem_used = 0;
    int64_t n_submitted = 0, n_completed = 0, n_passes = 0;
};

namespace {

// A finished request: counted on its model (service time for the admission
// estimate) and queued for opf_server_poll.  Called with s->mu held.
void finish_locked(opf_server *s, Model &m, Done &&d) {
    if (d.status == OPF_E_TIMEOUT && d.t_done > d.t_admit) ++m.n_stopped;   // ran into its service bound
    if (d.status != OPF_E_TIMEOUT || d.t_done > d.t_admit) {
        ++m.n_done;
        if (d.converged) ++m.n_conv;
        const double svc = d.t_done - d.t_admit;
        m.svc_s = (m.svc_s * (double)m.n_svc + svc) / (double)(m.n_svc + 1);
        ++m.n_svc;
    }
    s->done.push_back(std::move(d));
}

// Queued requests of model m that waited longer than its bound leave the
// queue with status OPF_E_TIMEOUT (shed).
void shed_expired(opf_server *s, Model &m) {
    if (!(m.max_wait_s > 0.0)) return;
    const double t = now_s();
    while (!m.queue.empty() && t - m.queue.front().t_submit > m.max_wait_s) {
        Request r = std::move(m.queue.front());
        m.queue.pop_front();
        Done d;
        d.tag = r.tag;
        d.model = m.id;
        d.converged = 0;
        d.iters = 0;
        d.status = OPF_E_TIMEOUT;
        d.objective = NAN;
        d.t_submit = r.t_submit;
        d.t_admit = t;
        d.t_done = t;
        ++m.n_shed;
        std::lock_guard<std::mutex> g(s->mu);
        s->done.push_back(std::move(d));
    }
}

// Estimated device bytes of one batch slot: per-instance FP64 arrays and the
// share of both engines' per-column arrays.
size_t batch_slot_bytes(opf_handle *h) {
    const size_t L = h->L, G = h->G, R = h->n_rows;
    size_t fp64 = 8 * (R + 4 * L + 3 * G) + sizeof(DevStatus) * 2 + 16;
    size_t eng = (size_t)(1.6 * L) * (4 * 4 + 4 * 8) + G * (3 * 4 + 3 * 8);
    return fp64 + eng;
}

// Engine columns of both plans: the slots of each phase packed from column 0
// (every pass re-centres from the FP64 state, so a slot may change column
// between passes); n32 / n64 count them.
int upload_maps(Model &m) {
    opf_batch *b = m.b;
    for (int pi = 0; pi < 2; ++pi) {
        BPlan &p = pi ? b->p64 : b->p32;
        const int want = pi ? 2 : 1;
        std::vector<int> inst((size_t)p.C * p.K, -1), ipos(b->n, -1);
        int col = 0;
        for (int i = 0; i < b->n; ++i)
            if (m.state[i] == want) { inst[col] = i; ipos[i] = col; ++col; }
        (pi ? m.n64 : m.n32) = col;
        SCUDA(cudaMemcpyAsync(p.d_inst, inst.data(), inst.size() * sizeof(int), cudaMemcpyHostToDevice, b->h->stream));
        SCUDA(cudaMemcpyAsync(p.d_ipos, ipos.data(), ipos.size() * sizeof(int), cudaMemcpyHostToDevice, b->h->stream));
    }
    return OPF_OK;
}

void single_worker(opf_server *s, Model *m, Worker *w, Request req, double t_admit) {
    const opf_server_opts &o = s->o;
    Done d;
    d.tag = req.tag;
    d.model = m->id;
    d.t_submit = req.t_submit;
    d.t_admit = t_admit;
    d.converged = 0;
    d.iters = 0;
    d.objective = NAN;
    int rc = opf_set_loads(w->h, req.lp.data(), req.lq.data());
    if (!rc) rc = opf_precompute(w->h);
    if (!rc && !m->start_xs.empty())
        rc = opf_set_locals(w->h, m->start_xs.data(), m->start_lam.data(), m->start_xs.size());
    if (!rc) {
        opf_solve_opts so;
        memset(&so, 0, sizeof(so));
        so.rho = o.rho; so.eps_rel = m->eps_rel; so.eps_abs_pres = m->eps_abs; so.max_iter = o.max_iter;
        so.check_every = o.check_every; so.precision = OPF_PREC_MIXED; so.recenter_every = o.chunk_iters;
        // direct launches: the handle's stream may belong to an SM partition,
        // where the solve graph of opf_solve_ex cannot be instantiated (and
        // the host loop honours the service bound and a cancel)
        so.flags = OPF_SOLVE_HOST_LOOP;
        w->h->deadline = m->max_service_s > 0.0 ? steady_seconds() + m->max_service_s : 0.0;
        rc = opf_solve_ex(w->h, &so);
        w->h->deadline = 0.0;
        d.converged = rc == OPF_OK;
        if (rc == OPF_OK || rc == OPF_NOT_CONVERGED) {
            if (o.keep_solutions) d.x.resize(m->G);
            double obj = 0;
            opf_get_solution(w->h, o.keep_solutions ? d.x.data() : nullptr, o.keep_solutions ? m->G : 0, &obj);
            d.objective = obj;
            double pr, dr, ep, ed;
            int64_t it = 0;
            opf_get_residuals(w->h, &pr, &dr, &ep, &ed, &it);
            d.iters = (int32_t)it;
            rc = OPF_OK;
        } else if (rc == OPF_E_TIMEOUT) {     // stopped by the service bound: iterations run so far
            double pr, dr, ep, ed;
            int64_t it = 0;
            opf_get_residuals(w->h, &pr, &dr, &ep, &ed, &it);
            d.iters = (int32_t)it;
        }
    }
    d.status = rc;
    d.t_done = now_s();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (o.keep_solutions) s->kept.emplace_back(d.tag, std::move(d.x));
        finish_locked(s, *m, std::move(d));
        w->finished = true;       // with the result queued: a worker counts as running until then
    }
}

int step_single(opf_server *s, Model &m) {
    for (auto &wp : m.workers) {
        Worker &w = *wp;
        if (w.busy && w.finished) {
            w.th.join();
            w.busy = false;
            w.finished = false;
        }
        if (!w.busy && !m.queue.empty()) {
            Request r = std::move(m.queue.front());
            m.queue.pop_front();
            w.busy = true;
            w.finished = false;
            w.t_admit = now_s();
            w.th = std::thread(single_worker, s, &m, &w, std::move(r), w.t_admit);
        }
    }
    return OPF_OK;
}

// Admission and one pass of a batched model (enqueue only).
int step_batched_enqueue(opf_server *s, Model &m) {
    opf_batch *b = m.b;
    for (int i = 0; i < m.cap && !m.queue.empty(); ++i) {
        if (m.state[i]) continue;
        Request r = std::move(m.queue.front());
        m.queue.pop_front();
        STRY(set_loads_impl(b, i, 1, r.lp.data(), r.lq.data(), false));
        m.state[i] = 1;
        m.tag[i] = r.tag;
        m.t_submit[i] = r.t_submit;
        m.t_admit[i] = now_s();
    }
    if (!m.running()) return OPF_OK;
    STRY(upload_maps(m));
    const int R = s->o.chunk_iters, k = s->o.check_every;
    const int R64 = s->o.polish_chunk_iters;
    // FP32 slots on the model's stream, FP64 slots on a second stream: the
    // two passes touch disjoint instances and run side by side
    SCUDA(cudaEventRecord(m.ev_start, b->h->stream));
    SCUDA(cudaStreamWaitEvent(m.s64, m.ev_start, 0));
    if (m.n32) {
        STRY(plan_set_rho(b, &b->p32, s->o.rho));
        enqueue_body_any(b, b->p32, s->o.rho, R, k, cudaGraphConditionalHandle{}, 0, nullptr, nullptr,
                         (m.n32 + b->p32.K - 1) / b->p32.K);
    }
    if (m.n64) {
        // slots in the polish met the test in FP32 already: tested every 2
        // FP64 iterations, so most leave after the first test
        STRY(plan_set_rho(b, &b->p64, s->o.rho));
        enqueue_body_any(b, b->p64, s->o.rho, R64, std::min(k, 2), cudaGraphConditionalHandle{}, 0, nullptr,
                         nullptr, (m.n64 + b->p64.K - 1) / b->p64.K, m.s64);
    }
    SCUDA(cudaEventRecord(m.ev64, m.s64));
    SCUDA(cudaStreamWaitEvent(b->h->stream, m.ev64, 0));
    launch_bobjective(b->n, b->G, b->h->d_c64, b->d_x, b->d_obj, b->h->stream);
    SCUDA(cudaGetLastError());
    SCUDA(cudaEventRecord(m.ev, b->h->stream));
    m.inflight = true;
    return OPF_OK;
}

// Phase changes and retirement after the model's stream finished the pass.
int step_batched_collect(opf_server *s, Model &m) {
    opf_batch *b = m.b;
    m.inflight = false;
    STRY(read_status(b));
    m.obj.resize(b->n);
    SCUDA(cudaMemcpyAsync(m.obj.data(), b->d_obj, b->n * sizeof(double), cudaMemcpyDeviceToHost, b->h->stream));
    SCUDA(cudaStreamSynchronize(b->h->stream));
    bool wrote = false;
    const double t = now_s();
    for (int i = 0; i < m.cap; ++i) {
        DevStatus &st = b->h_st[i];
        if (!m.state[i] || !st.done) continue;
        if (m.state[i] == 1 && st.converged && !st.numeric) {
            // the FP32 test held: continue in FP64 from the same state
            st.done = 0;
            st.converged = 0;
            st.max_iter = std::max<long long>(st.max_iter, st.iter + 2LL * s->o.check_every);
            m.state[i] = 2;
            wrote = true;
            continue;
        }
        Done d;
        d.tag = m.tag[i];
        d.model = m.id;
        d.converged = st.converged;
        d.iters = (int32_t)st.iter;
        d.status = st.numeric ? OPF_E_NUMERIC : (st.converged ? OPF_OK : OPF_NOT_CONVERGED);
        d.objective = m.obj[i];
        d.t_submit = m.t_submit[i];
        d.t_admit = m.t_admit[i];
        d.t_done = t;
        std::vector<double> x;
        if (s->o.keep_solutions) {
            x.resize(m.G);
            SCUDA(cudaMemcpyAsync(x.data(), b->d_x + (size_t)i * m.G, m.G * sizeof(double), cudaMemcpyDeviceToHost,
                                  b->h->stream));
            SCUDA(cudaStreamSynchronize(b->h->stream));
        }
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->o.keep_solutions) s->kept.emplace_back(d.tag, std::move(x));
            finish_locked(s, m, std::move(d));
        }
        m.state[i] = 0;
    }
    // running slots past the model's service bound leave with OPF_E_TIMEOUT
    if (m.max_service_s > 0.0) {
        for (int i = 0; i < m.cap; ++i) {
            if (!m.state[i] || t - m.t_admit[i] <= m.max_service_s) continue;
            Done d;
            d.tag = m.tag[i];
            d.model = m.id;
            d.converged = 0;
            d.iters = (int32_t)b->h_st[i].iter;
            d.status = OPF_E_TIMEOUT;
            d.objective = NAN;
            d.t_submit = m.t_submit[i];
            d.t_admit = m.t_admit[i];
            d.t_done = t;
            std::lock_guard<std::mutex> g(s->mu);
            finish_locked(s, m, std::move(d));
            m.state[i] = 0;
        }
    }
    if (wrote) {
        STRY(write_status(b, 0, b->n));
        SCUDA(cudaStreamSynchronize(b->h->stream));
    }
    return OPF_OK;
}

}  // namespace

extern "C" {

int opf_server_create(const opf_server_opts *o, opf_server **out) {
    if (!o || !out || !(o->rho > 0) || o->max_iter < 1 || o->check_every < 2 || (o->check_every & 1) ||
        o->chunk_iters < o->check_every || o->chunk_iters % o->check_every || o->mem_budget < 0 ||
        o->polish_chunk_iters < 0 || o->polish_chunk_iters % o->check_every) {
        set_last_error("server options: rho > 0, max_iter >= 1, even check_every >= 2, chunk_iters and "
                       "polish_chunk_iters multiples of check_every, mem_budget >= 0");
        return OPF_E_INVALID;
    }
    opf_server *s = new opf_server();
    s->o = *o;
    s->o.max_iter = cap_at_tests(o->max_iter, o->check_every);
    if (s->o.polish_chunk_iters == 0) s->o.polish_chunk_iters = 2 * o->check_every;
    *out = s;
    return OPF_OK;
}

int opf_server_add_model(opf_server *s, opf_handle *const *handles, int32_t n_handles, int32_t capacity,
                         int32_t *model_id) {
    if (!s || !handles || n_handles < 1 || capacity < 1 || !model_id) return OPF_E_INVALID;
    opf_handle *h = handles[0];
    if (!h || !h->precomputed) return OPF_E_STATE;
    if (h->model.n_load == 0) { set_last_error("server: models are feeders (loads per request)"); return OPF_E_INVALID; }

    auto m = std::make_unique<Model>();
    m->id = (int)s->models.size();
    m->h = h;
    m->G = h->G;
    m->nload = h->model.n_load;
    m->eps_rel = s->o.eps_rel;
    m->eps_abs = s->o.eps_abs_pres;
    // batched when both engine plans fit the model
    const size_t per = batch_slot_bytes(h);
    int cap = capacity;
    if (s->o.mem_budget > 0) {
        const int64_t left = s->o.mem_budget - s->mem_used;
        cap = (int)std::min<int64_t>(cap, left > 0 ? left / (int64_t)per : 0);
    }
    bool batched = false;
    // a ZIP exponent makes A_s (hence M_s) depend on the request's loads: each
    // request then gets its own factorization on a single-instance handle
    if (h->model.A_depends_on_loads) cap = 0;
    if (cap >= 1) {
        // does the batched engine hold this model?  (probe with one slot)
        opf_batch *probe = nullptr;
        int rc = opf_batch_create(h, 1, &probe);
        if (rc == OPF_OK) rc = ensure_plan(probe, false, s->o.rho, s->o.check_every);
        if (rc == OPF_OK) rc = ensure_plan(probe, true, s->o.rho, s->o.check_every);
        opf_batch_destroy(probe);
        if (rc != OPF_OK && rc != OPF_E_CAPACITY) return rc;
        if (rc == OPF_E_CAPACITY) cap = 0;
    }
    if (cap >= 1) {
        opf_batch *b = nullptr;
        int rc = opf_batch_create(h, cap, &b);
        if (rc == OPF_OK) {
            b->init_max_iter = s->o.max_iter;
            b->init_eps_rel = s->o.eps_rel;
            b->init_eps_abs = s->o.eps_abs_pres;
            rc = ensure_plan(b, false, s->o.rho, s->o.check_every);
            if (rc == OPF_OK) rc = ensure_plan(b, true, s->o.rho, s->o.check_every);
        }
        if (rc == OPF_OK) {
            m->b = b;
            batched = true;
        } else {
            opf_batch_destroy(b);
            if (rc != OPF_E_CAPACITY) return rc;
        }
    }
    if (batched) {
        SCUDA(cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming));
        SCUDA(cudaEventCreateWithFlags(&m->ev64, cudaEventDisableTiming));
        SCUDA(cudaEventCreateWithFlags(&m->ev_start, cudaEventDisableTiming));
        STRY(stream_sibling(h->stream, &m->s64));
        m->batched = true;
        m->cap = cap;
        m->slot_bytes = per;
        s->mem_used += (int64_t)per * cap;
        m->state.assign(cap, 0);
        m->tag.assign(cap, 0);
        m->t_submit.assign(cap, 0.0);
        m->t_admit.assign(cap, 0.0);
    } else {
        // one request per caller handle at a time
        const int64_t per1 = (int64_t)h->h2d_bytes * 4 + (int64_t)(h->L + h->G) * 64;
        int n = n_handles;
        if (s->o.mem_budget > 0) {
            const int64_t left = s->o.mem_budget - s->mem_used;
            n = (int)std::min<int64_t>(n, left > 0 ? left / per1 : 0);
        }
        if (n < 1) { set_last_error("server: the memory budget admits no slot of this model"); return OPF_E_CAPACITY; }
        for (int i = 0; i < n; ++i) {
            if (!handles[i]) return OPF_E_INVALID;
            auto w = std::make_unique<Worker>();
            w->h = handles[i];
            m->workers.push_back(std::move(w));
        }
        m->cap = n;
        s->mem_used += per1 * n;
    }
    *model_id = m->id;
    s->models.push_back(std::move(m));
    return OPF_OK;
}

int opf_server_set_model_tolerance(opf_server *s, int32_t model, double eps_rel, double eps_abs_pres) {
    if (!s || model < 0 || model >= (int)s->models.size() || !(eps_rel >= 0) || !(eps_abs_pres >= 0))
        return OPF_E_INVALID;
    Model &m = *s->models[model];
    m.eps_rel = eps_rel;
    m.eps_abs = eps_abs_pres;
    if (m.b) {
        m.b->init_eps_rel = eps_rel;
        m.b->init_eps_abs = eps_abs_pres;
    }
    return OPF_OK;
}

int opf_server_set_model_shape(opf_server *s, int32_t model, int32_t k_inst, int32_t warps) {
    if (!s || model < 0 || model >= (int)s->models.size()) return OPF_E_INVALID;
    Model &m = *s->models[model];
    if (!m.batched) {
        set_last_error("server: the model is served by worker threads (no batched engine)");
        return OPF_E_INVALID;
    }
    if (m.inflight) {
        set_last_error("server: a pass of the model is in flight (set the shape between steps)");
        return OPF_E_STATE;
    }
    STRY(opf_batch_set_shape(m.b, OPF_PREC_FP32, k_inst, warps));
    // the plan for the next pass (each pass re-centres from the FP64 state)
    return ensure_plan(m.b, false, s->o.rho, s->o.check_every);
}

int opf_server_set_model_start(opf_server *s, int32_t model, const double *xs, const double *lam) {
    if (!s || model < 0 || model >= (int)s->models.size() || (!xs) != (!lam)) return OPF_E_INVALID;
    Model &m = *s->models[model];
    if (m.b) return opf_batch_set_start(m.b, xs, lam);
    const size_t L = (size_t)m.h->L;
    if (xs) {
        m.start_xs.assign(xs, xs + L);
        m.start_lam.assign(lam, lam + L);
    } else {
        m.start_xs.clear();
        m.start_lam.clear();
    }
    return OPF_OK;
}

int opf_server_set_admission(opf_server *s, int32_t model, int32_t max_queue, double max_wait_s,
                             double max_service_s) {
    if (!s || model < 0 || model >= (int)s->models.size() || max_queue < 0 || !(max_wait_s >= 0.0) ||
        !(max_service_s >= 0.0))
        return OPF_E_INVALID;
    Model &m = *s->models[model];
    m.max_queue = max_queue;
    m.max_wait_s = max_wait_s;
    m.max_service_s = max_service_s;
    return OPF_OK;
}

int opf_server_submit(opf_server *s, int32_t model, const double *load_p, const double *load_q, int64_t tag) {
    if (!s || model < 0 || model >= (int)s->models.size() || !load_p || !load_q) return OPF_E_INVALID;
    Model &m = *s->models[model];
    ++m.n_sub;
    ++s->n_submitted;
    if (m.max_queue > 0 && (int)m.queue.size() >= m.max_queue) {
        ++m.n_refused;
        set_last_error("server: model " + std::to_string(model) + " queue is full (" +
                       std::to_string(m.max_queue) + " requests)");
        return OPF_E_CAPACITY;
    }
    if (m.max_wait_s > 0.0) {
        // predicted wait for a slot: the requests ahead (queued and running)
        // served cap at a time, each taking the model's mean service time;
        // before any request of the model finished, the longest time a
        // running one has run so far (its service time is at least that)
        double svc;
        {
            std::lock_guard<std::mutex> g(s->mu);
            svc = m.n_svc ? m.svc_s : 0.0;
        }
        const bool no_history = svc == 0.0;
        const double t = now_s();
        int busy = 0;
        if (m.batched) {
            busy = m.running();
            if (no_history)
                for (int i = 0; i < m.cap; ++i)
                    if (m.state[i]) svc = std::max(svc, t - m.t_admit[i]);
        } else {
            for (auto &w : m.workers) {
                if (!w->busy || w->finished) continue;
                ++busy;
                if (no_history) svc = std::max(svc, t - w->t_admit);
            }
        }
        const int ahead = (int)m.queue.size() + busy;
        const double wait = ahead < m.cap ? 0.0 : (double)((ahead - m.cap) / m.cap + 1) * svc;
        if (wait > m.max_wait_s) {
            ++m.n_refused;
            set_last_error("server: model " + std::to_string(model) + " cannot start the request within " +
                           std::to_string(m.max_wait_s) + " s (predicted wait " + std::to_string(wait) + " s)");
            return OPF_E_CAPACITY;
        }
    }
    Request r;
    r.tag = tag;
    r.lp.assign(load_p, load_p + (size_t)m.nload * 3);
    r.lq.assign(load_q, load_q + (size_t)m.nload * 3);
    r.t_submit = now_s();
    m.queue.push_back(std::move(r));
    return OPF_OK;
}

int opf_server_step(opf_server *s) {
    if (!s) return OPF_E_INVALID;
    for (auto &m : s->models) {
        shed_expired(s, *m);
        if (!m->batched) {
            STRY(step_single(s, *m));
            continue;
        }
        // each model advances on its own: collect a finished pass, start the next
        if (m->inflight) {
            const cudaError_t q = cudaEventQuery(m->ev);
            if (q == cudaErrorNotReady) continue;
            SCUDA(q);
            STRY(step_batched_collect(s, *m));
            ++s->n_passes;
        }
        STRY(step_batched_enqueue(s, *m));
    }
    return OPF_OK;
}

int opf_server_poll_ex(opf_server *s, int64_t *tags, int32_t *status, int32_t *converged, double *objective,
                       int32_t *iters, double *latency_s, int32_t max_n) {
    if (!s || max_n < 0) return OPF_E_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    const int n = std::min<int>(max_n, (int)s->done.size());
    for (int i = 0; i < n; ++i) {
        const Done &d = s->done[i];
        if (tags) tags[i] = d.tag;
        if (status) status[i] = d.status;
        if (converged) converged[i] = d.converged;
        if (objective) objective[i] = d.objective;
        if (iters) iters[i] = d.iters;
        if (latency_s) latency_s[i] = d.t_done - d.t_submit;
    }
    s->done.erase(s->done.begin(), s->done.begin() + n);
    s->n_completed += n;
    return n;
}

int opf_server_poll(opf_server *s, int64_t *tags, int32_t *converged, double *objective, int32_t *iters,
                    double *latency_s, int32_t max_n) {
    return opf_server_poll_ex(s, tags, nullptr, converged, objective, iters, latency_s, max_n);
}

int opf_server_take_solution(opf_server *s, int64_t tag, double *x, int32_t n) {
    if (!s || !x) return OPF_E_INVALID;
    std::lock_guard<std::mutex> g(s->mu);
    for (size_t i = 0; i < s->kept.size(); ++i)
        if (s->kept[i].first == tag) {
            if (n < (int)s->kept[i].second.size()) return OPF_E_INVALID;
            std::copy(s->kept[i].second.begin(), s->kept[i].second.end(), x);
            s->kept.erase(s->kept.begin() + i);
            return OPF_OK;
        }
    set_last_error("server: no kept solution with this tag");
    return OPF_E_STATE;
}

int opf_server_stats(opf_server *s, int64_t *out, int32_t n) {
    if (!s || !out) return OPF_E_INVALID;
    int64_t queued = 0, running = 0, slots = 0;
    for (auto &m : s->models) {
        queued += (int64_t)m->queue.size();
        slots += m->cap;
        if (m->batched) running += m->running();
        else
            for (auto &w : m->workers) running += (w->busy && !w->finished) ? 1 : 0;
    }
    const int64_t v[7] = {s->n_submitted, s->n_completed, queued, running, slots, s->n_passes, s->mem_used};
    for (int i = 0; i < n && i < 7; ++i) out[i] = v[i];
    return OPF_OK;
}

int opf_server_model_stats(opf_server *s, int32_t model, int64_t *out, int32_t n) {
    if (!s || !out || model < 0 || model >= (int)s->models.size()) return OPF_E_INVALID;
    Model &m = *s->models[model];
    int64_t running = 0;
    if (m.batched) running = m.running();
    else
        for (auto &w : m.workers) running += (w->busy && !w->finished) ? 1 : 0;
    double svc;
    {
        std::lock_guard<std::mutex> g(s->mu);
        svc = m.n_svc ? m.svc_s : 0.0;
    }
    const int64_t v[10] = {m.n_sub.load(), m.n_done.load(), m.n_conv.load(), m.n_refused.load(), m.n_shed.load(),
                           (int64_t)m.queue.size(), running, (int64_t)m.cap, (int64_t)(svc * 1e6),
                           m.n_stopped.load()};
    for (int i = 0; i < n && i < 10; ++i) out[i] = v[i];
    return OPF_OK;
}

void opf_server_destroy(opf_server *s) {
    if (!s) return;
    for (auto &m : s->models)           // running worker solves stop at their next chunk
        for (auto &w : m->workers) w->h->cancel = 1;
    for (auto &m : s->models) {
        for (auto &w : m->workers) {
            if (w->th.joinable()) w->th.join();
            w->h->cancel = 0;
        }
        if (m->b) opf_batch_destroy(m->b);
        if (m->ev) cudaEventDestroy(m->ev);
        if (m->ev64) cudaEventDestroy(m->ev64);
        if (m->ev_start) cudaEventDestroy(m->ev_start);
        if (m->s64) cudaStreamDestroy(m->s64);
    }
    delete s;
}

}  // extern "C"
