// Internal records of the batched engine (shared by the batch C ABI and the
// request server).
#pragma once

#include <string>
#include <vector>

#include "handle.h"

// One engine plan: shape, tables and the engine-layout arrays.
struct BPlan {
    bool ok = false, dbl = false, fg = false;   // fg: factors read from global memory
    int K = 0, ks = 0, J = 0, W = 0, nq = 0, threads = 0;
    int NCH = 0, NB = 0, nF = 0, n_tasks = 0, C = 0, Gs = 0;
    bool tm = false;                  // lambda and bbar~ in tensor memory (FP32 plans)
    int tm_cols = 0, qstart[5] = {0, 0, 0, 0, 0};
    unsigned off_u = 0, off_gt = 0, off_rc = 0, off_task = 0, off_useg = 0, off_bnd = 0, off_red = 0, off_flag = 0;
    unsigned bytes = 0;
    double rho = -1.0;
    std::vector<void *> allocs;
    BatchTask *d_tasks = nullptr;
    int *d_memb = nullptr, *d_sch = nullptr, *d_uxt = nullptr, *d_gx = nullptr;
    int n_uxt = 0;
    int *d_inst = nullptr, *d_ipos = nullptr, *d_gperm = nullptr;
    int4 *d_chg = nullptr, *d_gtab = nullptr;
    void *d_F = nullptr, *d_recip = nullptr, *d_cost = nullptr;
    void *mu = nullptr, *ds = nullptr, *xo = nullptr, *bt = nullptr, *lref = nullptr;
    void *ct = nullptr, *xrf = nullptr, *lbt = nullptr, *ubt = nullptr, *cbt = nullptr;
    // lane-engine plans (K = kLaneInst, C = tiles of K instances)
    bool lane = false;
    int lane_C = 0, lane_nslm = 0, lane_maxux = 0;
    unsigned loff[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    LanePart *d_lparts = nullptr;
    int4 *d_lsub = nullptr, *d_lgi = nullptr;
    int *d_lcp = nullptr, *d_lux = nullptr, *d_lgk = nullptr;
    GraphCache graph;
    void release() {
        graph.reset();
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        ok = false;
        lane = false;
    }
};

struct opf_batch {
    opf_handle *h = nullptr;
    int n = 0;
    int G = 0, L = 0, S = 0, nrows = 0;
    std::vector<void *> allocs;
    double *d_rhs = nullptr, *d_bbar = nullptr, *d_xs = nullptr, *d_lam = nullptr, *d_xref = nullptr;
    double *d_dref = nullptr;            // per (instance, global): lambda - lambda_ref of its copies
    double *d_x = nullptr, *d_obj = nullptr, *d_b0 = nullptr, *d_rcoef = nullptr, *d_stage = nullptr;
    double *d_start = nullptr;           // warm start (x_s then lambda, device slot order), or none
    size_t stage_len = 0;
    int *d_rsrc = nullptr, *d_c2d = nullptr, *d_bidx = nullptr, *d_bad = nullptr;
    int *d_flag = nullptr;               // [0] FP32 plan, [1] FP64 plan: an instance still runs
    DevStatus *d_st = nullptr, *d_st_save = nullptr;
    std::vector<DevStatus> h_st;
    int NB = 0;
    std::vector<int> h_bidx;
    BPlan p32, p64;
    int force_k32 = 0, force_w32 = 0, force_k64 = 0, force_w64 = 0;
    bool allow_tmem = true;              // FP32 plans may keep lambda and bbar~ in tensor memory
    bool have_x = false;
    double timing[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // test parameters given to an instance when its rhs is set
    long long init_max_iter = 1000000;
    double init_eps_rel = 1e-8, init_eps_abs = 1e-4;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t eng_ev[2] = {nullptr, nullptr};
    double engine_ms[2] = {0, 0};        // host-loop runs: engine launches alone (FP32, FP64)
    long long bodies[2] = {0, 0};        // loop passes of the last solve (FP32, FP64)
    long long iter_base[2] = {0, 0};     // iteration count at the start of each phase
    std::vector<double> tune_log;   // (K, W, ms) triples of the last autotune
};

#define BCUDA(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return e_ == cudaErrorMemoryAllocation ? OPF_E_OOM : OPF_E_CUDA;             \
        }                                                                                \
    } while (0)
#define BTRY(x) do { int rc_ = (x); if (rc_) return rc_; } while (0)

constexpr unsigned kMaxSmem = 227u * 1024u;   // dynamic shared memory of one CTA

namespace opf {

// Lane engine (lane.cu): kernel attributes for clusters of C CTAs, clusters
// the device holds at once, a launch of `tiles` clusters, factor packing.
int lane_engine_prepare(int C, unsigned bytes);
int lane_engine_max_clusters(int C, int threads, unsigned bytes);
int lane_engine_ctas_per_sm(int threads, unsigned bytes);
int lane_engine_launch(const LaneArgs &a, int tiles, int threads, unsigned bytes, int n_iters, int check_every,
                       cudaStream_t s);
void launch_lpack(int nrec, const int4 *desc, const int4 *sub, const int4 *sub2, const double *F64, float *dst,
                  cudaStream_t s);

namespace bx {

// Device allocation recorded in `list` (freed with the plan or batch).
template <typename T>
inline int balloc(std::vector<void *> &list, T **p, size_t n) {
    if (n == 0) n = 1;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return OPF_E_OOM;
    }
    list.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return OPF_OK;
}

// Allocation filled from v on stream s.
template <typename T>
inline int bupload(std::vector<void *> &list, T **p, const std::vector<T> &v, cudaStream_t s) {
    BTRY(balloc(list, p, v.size()));
    if (!v.empty()) BCUDA(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return OPF_OK;
}

inline unsigned a16(size_t x) { return (unsigned)((x + 15) & ~(size_t)15); }

// Lane-engine plan (FP32): K = kLaneInst instances per tile, C tiles, clusters
// of lane_C <= maxC CTAs, WG warps per lane quadrant; OPF_E_CAPACITY when the
// model does not fit (a part above the tensor-memory or shared-memory budget).
int build_lane_plan(opf_batch *b, BPlan *p, int WG, int maxC);
LaneArgs lane_args(opf_batch *b, const BPlan &p, double rho);

// Engine plan for one arithmetic type (built on first use; FP32 autotuned).
int ensure_plan(opf_batch *b, bool dbl, double rho, int k);
int plan_set_rho(opf_batch *b, BPlan *p, double rho);
// One loop pass on the handle's stream: re-centre, n_iters engine iterations
// (test every k), back to FP64, "still running" flag.
// ctas >= 0 launches only the first ctas CTAs of the engine (columns packed
// from the front).
void enqueue_body_any(opf_batch *b, BPlan &p, double rho, int n_iters, int k, cudaGraphConditionalHandle c,
                      int use, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr, int ctas = -1,
                      cudaStream_t stream = nullptr);
int read_status(opf_batch *b);
// Loads of instances [first, first + count) (host or device arrays) into rhs,
// bbar, start point and fresh status; sync_check reads the consistency flags.
int set_loads_impl(opf_batch *b, int first, int count, const double *load_p, const double *load_q,
                   bool on_device);
// Device -> host status of one instance range, host -> device.
int write_status(opf_batch *b, int first, int count);

}  // namespace bx
}  // namespace opf
