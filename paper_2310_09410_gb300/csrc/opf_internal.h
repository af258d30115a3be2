// Internal declarations of the ADMM library (host model, device layout,
// kernel launchers).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opf.h"

namespace opf {

// ---------------------------------------------------------------- host model
// One subsystem of Eq. OurModel: m x n block A (row-major), b, and the global
// index of each local slot (ascending for feeder models).
struct HostSub {
    int m = 0, n = 0;
    std::vector<int> vars;
    std::vector<double> A, b;
};

struct HostModel {
    int n = 0;
    std::vector<double> c, lb, ub;
    std::vector<uint8_t> volt;
    std::vector<HostSub> subs;   // canonical subsystem order
};

// Sec. II-A rows + Sec. V-A decomposition.  Returns OPF_OK or an error code
// with a message in *err.
int build_feeder_model(const opf_feeder *f, HostModel *out, std::string *err);
int build_generic_model(int n, const double *c, const double *lb, const double *ub,
                        const uint8_t *volt, int S, const int *m_s, const int *n_s,
                        const double *A, const double *b, const int *idx,
                        HostModel *out, std::string *err);

// ------------------------------------------------------------ device layout
// A warp task covers 32 / W subsystems of one size class (W lanes each, R
// rows per lane, n <= W * R).
struct Task {
    int first;   // first subsystem (device order)
    int count;   // subsystems in this task
    int W;       // lanes per subsystem: 8, 16 or 32
    int R;       // rows per lane (1..8, W == 32 when R > 1)
};

constexpr int RMAX = 8;

// Arguments of one iteration, in precision T.  All pointers may address
// global or shared memory (generic addressing).
template <typename T>
struct IterArgs {
    // per subsystem (device order)
    const int *soff;      // first slot
    const int *sn;        // n_s
    const int *sf;        // f_s: columns of the stored factor
    const int *smode;     // 0: M = I - F F^T, 1: M = F F^T
    const long long *sfoff;   // factor offset (elements)
    const T *F;           // factors, column-major n x f per subsystem
    // per slot (device order)
    const int2 *seg;      // (start, count) of the slot's global in u
    const int *gk;        // global index
    const int *pk;        // position of the slot in u
    const T *bt;          // bbar shifted by the reference point
    T *mu;                // lambda - lambda_ref
    T *ds;                // x_s - x_ref[g]
    // per global
    const T *ct;          // c + sum lambda_ref
    const T *lbt, *ubt;   // bounds - x_ref
    // FP64 data read only on tested iterations
    const double *xr;     // x_ref per global
    const double *lamr;   // lambda_ref per slot
    const double *c64;    // original costs
    // tasks
    const int4 *tasks;    // (first, count, W, R)
    int n_tasks;
    T rho, inv_rho;
};

// Device status of a solve: iteration count, the Sec. III-C quantities of the
// last test and the loop flags.
struct DevStatus {
    long long iter;        // iterations completed
    double pres, dres, eprim, edual, obj;
    int converged, numeric, done, pad;
    long long max_iter;
    double eps_rel, eps_abs_pres;
};

// Per subsystem s (device order): A_s (m x n row-major) at W + aoff[s] and b_s
// at Bw + boff[s] are work copies, overwritten.  P + poff[s] is n x n scratch.
struct PreArgs {
    int S;
    const int *sm, *sn, *soff;
    const long long *aoff, *poff, *foff;
    const int *boff;
    double *W, *Bw, *P;
    double *F;          // out: factor, column-major n x f
    int *sf, *smode;    // out
    double *bbar;       // out: per slot
    int *status;        // out: 0 ok, 1 inconsistent local system
};

// Byte offsets of the one-CTA engine's shared-memory image.
struct CtaLayout {
    int S, L, G, n_tasks, vstride;
    long long nF;                 // factor elements
    unsigned off_F, off_bt, off_mu, off_ds, off_u0, off_u1, off_ct, off_lbt, off_ubt;
    unsigned off_seg, off_gk, off_pk, off_soff, off_sn, off_sf, off_smode, off_sfoff, off_tasks, off_sv;
    unsigned bytes;
};

}  // namespace opf
