// Host-side state of one ADMM handle (internal; shared by the single-instance
// drivers and the batched engine).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "opf_internal.h"

// The handle type is declared at global scope by opf.h; the helper records
// live beside it.
using namespace opf;

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    bool host_loop = false;
    double rho = 0;
    int k = 0, R = 0, kind = -1, P = 0;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        kind = -1;
    }
};

// Cluster plan for one precision: P CTAs, part ranges and part-relative records.
struct ClusterPlan {
    int P = 0;
    bool ok = false;
    ClusterLayout lay{};
    int *d_pr = nullptr;
    int4 *d_srec = nullptr;
    int *d_items = nullptr, *d_meta = nullptr, *d_udst = nullptr, *d_gsegp = nullptr, *d_cdst = nullptr;
};

// Persistent grid engine plan for one precision: P co-resident CTAs, part
// ranges, part-relative records, the partial sums and the barrier counter.
constexpr int kPersistMaxP = 2048;
struct PersistPlan {
    int P = 0;
    bool ok = false;
    bool tried = false;          // built (ok or not) for the current factors and request
    int req = 0;                 // requested CTA count of that build (0: automatic)
    PersistLayout lay{};
    int *d_pr = nullptr;         // 5 * (kPersistMaxP + 1)
    int4 *d_srec = nullptr;
    int *d_items = nullptr, *d_meta = nullptr;
    double *d_part = nullptr;    // 6 * kPersistMaxP
    unsigned long long *d_sync = nullptr;
    PersistPtrs ptrs() const { return PersistPtrs{d_pr, d_part, d_sync}; }
};

// Warp-engine plan for one precision: warp slots of the CTAs of one cluster.
struct WarpPlan {
    int P = 0;
    int req = 0;               // CTA count asked for when built (0 = automatic)
    bool built = false, ok = false;
    WarpLayout lay{};
    int *d_pr = nullptr, *d_klb = nullptr, *d_fbig = nullptr;
    int *d_wrseg = nullptr, *d_wdsp = nullptr, *d_wdd = nullptr;
    int *d_wmap = nullptr;     // per (CTA, warp slot): (subsystem << 8) | (part << 4) | parts, or -1
    int3 *d_wrep = nullptr;
    float *d_F2 = nullptr;     // FP32 plan: factors of the subsystems with n > 32
    double *d_F2d = nullptr;   // FP64 plan: every factor
};

// Grid tiling for one precision: tile t covers subsystems [s0[t], s0[t+1]).
struct Tiling {
    int n_tiles = 0, block = 128, xcap = 0, vcap = 0, tcap = 0;
    int *d_s0 = nullptr;
};

struct opf_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    HostModel model;
    int S = 0, L = 0, G = 0;
    long long nA = 0, nB = 0, nP = 0, nFcap = 0, nF = 0, sum_nf = 0, n_rows = 0, nitems = 0;
    int max_ns = 0, sh_m = 0, sh_n = 0;
    std::vector<int> canon_slot_to_dev;     // canonical slot -> device slot
    std::vector<int> h_sn, h_sm, h_soff, h_sf, h_mode;
    std::vector<void *> allocs;
    // per subsystem
    int *d_soff = nullptr, *d_sn = nullptr, *d_sm = nullptr, *d_sf = nullptr, *d_smode = nullptr;
    int *d_boff = nullptr, *d_pstatus = nullptr;
    long long *d_aoff = nullptr, *d_poff = nullptr, *d_fcap = nullptr;
    int4 *d_sub = nullptr, *d_sub2 = nullptr;
    int *d_items = nullptr;
    // per slot
    int *d_gk = nullptr, *d_pk = nullptr, *d_uslot = nullptr, *d_meta = nullptr, *d_segp = nullptr;
    int2 *d_gseg = nullptr;
    double *d_A = nullptr, *d_b = nullptr, *d_W = nullptr, *d_Bw = nullptr, *d_P = nullptr;
    double *d_Fcap = nullptr, *d_F64 = nullptr, *d_bbar64 = nullptr;
    float *d_F32 = nullptr;
    // per global
    double *d_c64 = nullptr, *d_lb64 = nullptr, *d_ub64 = nullptr, *d_x0 = nullptr;
    double *d_xr = nullptr, *d_xr2 = nullptr, *d_zeroG = nullptr, *d_x = nullptr, *d_objpart = nullptr;
    float *d_ct32 = nullptr, *d_lbt32 = nullptr, *d_ubt32 = nullptr;
    double *d_recip64 = nullptr;
    float *d_recip32 = nullptr;
    // state
    double *d_ds64 = nullptr, *d_mu64 = nullptr, *d_u64 = nullptr, *d_lamr = nullptr, *d_zeroL = nullptr;
    float *d_ds32 = nullptr, *d_mu32 = nullptr, *d_u32 = nullptr, *d_bt32 = nullptr;
    double *d_partials = nullptr;
    DevStatus *d_st = nullptr;
    DevStatus *h_st = nullptr;
    Tiling t64, t32;
    // bookkeeping
    bool precomputed = false;
    bool have_prev_u = false;    // d_u64 + L holds the u that produced the last global update
    double last_rho = 100.0, recip_rho = -1.0;
    // Stop for solves whose body the host relaunches (OPF_SOLVE_HOST_LOOP):
    // past `deadline` (steady-clock seconds, 0 = none) or once `cancel` is
    // set by another thread, the solve returns OPF_E_TIMEOUT at its next
    // chunk with the iterate of that chunk readable (the request server's
    // service-time bound and its shutdown).
    double deadline = 0.0;
    std::atomic<int> cancel{0};
    long long total_iters = 0;
    long long main_iters = 0, recenters = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double timing[6] = {0, 0, 0, 0, 0, 0};
    long long h2d_bytes = 0;
    GraphCache g64, gmix;
    ClusterPlan c32, c64;
    PersistPlan p32, p64;
    bool persist_graph_failed = false;   // the cooperative launch could not be captured in a graph
    WarpPlan w32, w64;
    std::vector<int> h_tpre, h_vpre, h_foff, h_npad, h_pk, h_gk, h_gstart, h_uslot;
    std::vector<int> h_boff;                 // device subsystem -> first row (device row order)
    std::vector<int> dev_to_canon_sub;       // device subsystem -> canonical subsystem
    std::vector<int> canon_row_to_dev;       // canonical row -> device row
    // A_s^+ and the rejected-row combinations, computed on first use (batches)
    bool have_pinv = false;
    double *d_pinv = nullptr, *d_Tw = nullptr;
    long long *d_pioff = nullptr, *d_toff = nullptr;
    int *d_nrej = nullptr;
    std::vector<long long> h_pioff, h_toff;
    std::vector<int> h_nrej;
    double *d_x0_dev = nullptr;              // start point per global (alias of d_x0)
};

namespace opf {
// Runs the precompute kernel again with the A_s^+ outputs (same factors and
// bbar as opf_precompute, which must have succeeded).  Returns an OPF_ code.
int ensure_pinv(opf_handle *h);
// Thread-local message behind opf_last_error.
const char *last_error_cstr();
}  // namespace opf
