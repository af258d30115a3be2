// Internal declarations of the ADMM library (host model, device layout,
// kernel launchers).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opf.h"

namespace opf {

// Message returned by opf_last_error() on the calling thread.
void set_last_error(const std::string &msg);

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

constexpr int RMAX = 8;   // entries per lane in the precompute (n <= 256)

// Arguments of one iteration, in precision T.  Pointers may address global or
// shared memory (generic addressing).
template <typename T>
struct IterArgs {
    // per subsystem (device order), S + 1 entries (entry S is a sentinel)
    const int4 *sub;      // (first slot, n, f, mode)  mode 0: M = I - F F^T, 1: M = F F^T
    const int4 *sub2;     // (factor offset, npad, padded-v prefix, f prefix)
    const T *F;           // factors: f columns of npad entries (zero-padded) each
    const int *items;     // per factor column: (subsystem << 8) | column
    // per slot (device order)
    const int *meta;      // (subsystem << 8) | row
    const int *segp;      // (start of the global's copies in u << 8) | number of copies
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
    const T *recip;       // recip[N] = 1 / (rho N), N < 256
    const int *tile_s0;   // first subsystem of each grid tile (n_tiles + 1 entries)
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
// at Bw + boff[s] are work copies, overwritten.  P + poff[s] is the scratch of
// subsystems too large for shared memory (n*n + 33*(m+n) + 64 doubles).
struct PreArgs {
    int S;
    int sh_m, sh_n;     // largest m, n handled in shared memory
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
    int S, L, G, nitems;
    long long nF;                 // factor elements
    unsigned off_F, off_sub, off_sub2, off_items, off_meta, off_segp, off_gk, off_pk;
    unsigned off_bt, off_mu, off_ds, off_u0, off_u1, off_ct, off_lbt, off_ubt, off_recip;
    unsigned off_xb, off_vb, off_tb;
    unsigned bytes;
};

}  // namespace opf
