// Internal declarations of the ADMM library (host model, device layout,
// kernel launchers).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/opf.h"
#include "batch_tables.h"

namespace opf {

// Message returned by opf_last_error() on the calling thread.
void set_last_error(const std::string &msg);

// Seconds of the steady clock (for deadlines shared between threads).
double steady_seconds();

// ---------------------------------------------------------------- host model
// One subsystem of Eq. OurModel: m x n block A (row-major), b, and the global
// index of each local slot (ascending for feeder models).
struct HostSub {
    int m = 0, n = 0;
    std::vector<int> vars;
    std::vector<double> A, b;
    // per row: which load value the right-hand side is proportional to
    // (-1: a constant; else 2 * (3 * load + phase) + 0 for a, 1 for b) and the factor
    std::vector<int> rsrc;
    std::vector<double> rcoef;
    // per row: column of the entry of A proportional to the same load value
    // (a ZIP exponent's w coefficient; -1: none) and its factor
    std::vector<int> acol;
    std::vector<double> acoef;
};

struct HostModel {
    int n = 0;
    int n_load = 0;               // feeder loads (0 for generic models)
    bool A_depends_on_loads = false;   // a ZIP exponent makes A_s a function of the load values
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
    // cluster engine records (offsets relative to the CTA's part); the grid
    // engine never reads these, the cluster engine never reads items / meta
    const int *citems;    // per factor column: (subsystem in part << 8) | column
    const int *cmeta;     // per slot: (subsystem in part << 8) | row
    const int4 *srec;     // per subsystem: (factor offset, padded-v offset, t offset, f<<10 | npad<<1 | mode)
    const int *gsegp;     // per global: (start of its copies in the owner's u part << 8) | copies
    const int *udst;      // per slot: (owner rank << 24) | position in the owner's u part
    const int *cdst;      // per u entry: (rank holding the copy << 24) | padded-v offset there
    // warp engine: factors of subsystems with n > 32 packed per CTA and each
    // one's offset; each subsystem's first local slot; per local slot the
    // replica segment ((start << 8) | copies) and destination list
    // ((offset << 8) | count) of its u; destinations ((rank << 24) | position);
    // replica list (local start, start in u, copies) per CTA
    const T *F2;
    const int *wmap;      // per (CTA, warp slot): (subsystem << 8) | (part << 4) | parts, or -1
    const int *fbig;
    const int *klb;
    const int *wrseg, *wdsp, *wdd;
    const int3 *wrep;
    T *u_prev_out;        // u of the previous iteration, written on tested iterations
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
    int fault;             // a bounded wait of an engine ran out (the iterates are not valid)
    int pad2;
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
    // optional (pinv != nullptr): the same row operations applied to the
    // identity give T with beta = T b; pinv = Q^T T_acc = A_s^+ (n x m,
    // row-major at pioff[s]) and the rejected rows' combinations T_rej
    // (rows 0 .. nrej[s]-1 of the m x m block at Tw + toff[s] + m*m), whose
    // products with b_s vanish exactly when A_s x = b_s is consistent
    double *Tw, *pinv;
    const long long *toff, *pioff;
    int *nrej;
    int *status;        // out: 0 ok, 1 inconsistent local system
};

// Shared-memory image of one CTA of the cluster engine (sizes are the maxima
// over the P parts), byte offsets.
struct ClusterLayout {
    int P, L, threads;
    unsigned off_F, off_srec, off_items, off_meta, off_udst, off_bt, off_ds, off_mu, off_vbx, off_vbw;
    unsigned off_tb, off_gsegp, off_ct, off_lbt, off_ubt, off_uloc, off_cdst, off_recip, off_red;
    unsigned off_xrg, off_cg, off_xrs, off_lrs;
    unsigned bytes;
};

// Shared-memory image of one CTA of the persistent grid engine, byte offsets.
constexpr int kPersistMaxThreads = 512;
struct PersistLayout {
    int P, L, threads;
    int split;                     // phase B: a factor column on 4 lanes (plans of small CTAs)
    unsigned off_F, off_srec, off_items, off_meta, off_segp, off_pk, off_bt, off_ds, off_mu;
    unsigned off_ct, off_lbt, off_ubt, off_vbx, off_vbw, off_tb, off_recip, off_xrs, off_lrs, off_cobj;
    unsigned off_misc;
    unsigned bytes;
};

// Device arrays of a persistent grid engine plan.
struct PersistPtrs {
    const int *pr;                 // part ranges, 5 fields x (P + 1)
    double *part;                  // Sec. III-C partial sums, P x 6
    unsigned long long *sync;      // grid barrier counter
};

// Shared-memory image of one CTA of the warp engine, byte offsets.
struct WarpLayout {
    int P, L, S, useg_len, fbig_len;
    int warps;                     // warps per CTA (subsystem s: CTA s % P, warp s / P)
    unsigned off_useg, off_dd, off_fbig, off_vbig, off_tpart, off_red;
    unsigned bytes;
};

// A second non-blocking stream on the same SMs as s (its green context, if any).
int stream_sibling(cudaStream_t s, cudaStream_t *out);
// SMs that kernels launched on s may use: its green context's, else the device's.
int stream_sm_count(cudaStream_t s, int device);

// ------------------------------------------------------------ batched engine
// One warp task of the batched engine.  Lanes are (member position jpos,
// instance column sc), lane = jpos * K + sc, J * K = 32.  A member subsystem
// spans p = 2^lp consecutive positions; position jpos holds chunks
// (part * nq + q), q < nq, of its member's slots, part = jpos % p, 4 slots
// per chunk.  Chunk (q, jpos) of the task is chunk ch0 + q * J + jpos of the
// CTA's chunk array.
// The iteration cap is applied at the tests of the Sec. III-C rule, which
// run every k iterations: max_iter rounded up to a multiple of k (at most the
// largest multiple of k in an int32).
inline int32_t cap_at_tests(int32_t max_iter, int32_t k) {
    const long long r = ((long long)max_iter + k - 1) / k * k;
    const long long top = (0x7fffffffLL / k) * k;
    return (int32_t)(r < top ? r : top);
}

constexpr int kBatchRecip = 256;   // copy counts of a global are below this (the 8-bit count field)


// Arguments of one batched-engine launch.  Instance column sc of CTA c holds
// instance inst[c * K + sc] (-1: empty).  Engine arrays (type T):
//   per slot      [c][NCH][K][4]   mu, ds, bt (+bbar~ if M = F^T F, else -bbar~), lref (lambda_ref)
//   per global    [c][G][K]        xrf (x_ref), xo (x~ at the end)
//   per bounded   [c][NB][K]       lbt, ubt (bounds - x_ref), cbt (c~)
// The reference lambda_ref of the shifted frame makes c~ = c + sum lambda_ref
// zero at every unbounded global, so this engine reads c~ of the bounded ones
// only (cbt; the lane engine reads the per-global c~).  Its slot array holds
// rho x between the phases, so a global with one copy and no bounds needs no
// global update: the u of its slot is that value.  The global update's table
// (gtab, Gs entries) holds the globals it computes, the bounded ones first;
// gx and gperm list every global for the test iterations' x output.
template <typename T>
struct BatchArgs {
    int K, kshift, J, NCH, G, L, NB, n_tasks, nF, Gs;
    unsigned off_u, off_gt, off_rc, off_task, off_useg, off_bnd, off_red, off_flag;   // shared-memory byte offsets
    // Tensor-memory plans (FP32): lambda and bbar~ of every task stay in
    // tensor memory for the launch; the tasks of lane quadrant q are
    // [qstart[q], qstart[q + 1]) and run only on warps w with w % 4 == q.
    int tm, tm_cols, qstart[5];
    const BatchTask *tasks;    // [n_tasks] in decreasing cost
    const int4 *chg;           // [NCH] g * K of each chunk's 4 slots (-1: padding)
    // slot-array row of a copy: (ch * 4 + (e ^ (ch & 3))) * K
    const int4 *gtab;          // [Gs] (row of copy 0, row of copy 1, copies | first later copy in uxt << 8,
                               //       bounded index or -1)
    const int *uxt;            // [n_uxt] rows of the third and later copies
    const int *gx;             // [G] row of copy 0 | copies << 24, every table entry
    const int *gperm;          // [G] global of table entry j
    int n_uxt;
    const T *Fpk;              // [nF] factors, task-interleaved
    const T *cost;             // [G] c_i
    T *mu, *ds, *xo;
    const T *bt, *lref, *xrf, *lbt, *ubt, *cbt;
    const int *inst;
    DevStatus *st;             // per instance
    T rho, inv_rho;
    double rho_d;
};

// Lane engine (FP32 batches): a tile of kLaneInst instances, one instance per
// lane (warp w serves instances 32 (w % 4) .. + 31, which are also the
// tensor-memory lanes it reaches), runs on a cluster of C CTAs; CTA r of the
// cluster holds part r of the subsystems for all the tile's instances.  The
// engine arrays are those of the batched engine with K = kLaneInst columns
// per tile and the tile's slot positions grouped by part (part r owns chunks
// [cb, cb + nslot / 4)).
constexpr int kLaneInst = 128;
constexpr int kLaneMaxGroups = 8;     // item groups (warps per lane quadrant)
constexpr int kLaneMaxF4 = 6;         // factor vectors per subsystem <= 4 kLaneMaxF4

struct LanePart {
    int nsub, sub0;       // subsystem records [sub0, sub0 + nsub)
    int nslot, cb;        // local slot positions (a multiple of 4); first chunk in the tile
    int nF, F0;           // packed factor floats (multiples of 4)
    int ng, g0;           // global items, the part's own (interior) globals first
    int ncp, cp0;         // copy entries
    int nux, pad;         // exchange rows (slots whose global has copies in other parts)
    // per item group g: subsystems [gsub[g], gsub[g + 1]), interior globals
    // [gint[g], gint[g + 1]) and the others [gcut[g], gcut[g + 1]) (local indices)
    int gsub[kLaneMaxGroups + 1], gint[kLaneMaxGroups + 1], gcut[kLaneMaxGroups + 1];
};

struct LaneArgs {
    int C, WG, G, NB, NCH;
    int nslm;             // tensor-memory column of bbar~ of local slot 0 (lambda of slot p at column p)
    int tm_cols, maxux;
    unsigned off_U, off_X, off_F, off_sub, off_gi, off_cp, off_ux, off_gk, off_rc, off_red, off_part, off_flag;
    const LanePart *parts;   // [C]
    const int4 *sub;      // (first local slot, rows n, factor offset, mode | has-exchange-rows << 1 | F4 << 8)
    const int4 *gi;       // (global, bounded index or -1, first copy entry, copies N | owner << 16)
    const int *cp;        // (part << 24) | row: local slot position in the own part, else exchange row
    const int *ux;        // per tile slot position: exchange row or -1
    const int *gk;        // per tile slot position: global or -1
    const float *F;       // factors: per subsystem n rows of 4 F4 floats, F[k][c] at k * 4 F4 + c
    const float *recip;   // [kBatchRecip] 1 / (rho N)
    const float *cost;    // [G]
    float *mu, *ds, *xo;
    const float *bt, *lref, *ct, *xrf, *lbt, *ubt;
    const int *inst;      // [tiles * kLaneInst]
    DevStatus *st;
    float rho, inv_rho;
    double rho_d;
};

}  // namespace opf
