/*
 * opf.h -- C ABI of the GB300 ADMM solver for the decomposed linearized
 * (LinDist3Flow) multi-phase OPF of Ryu, Byeon and Kim, "A GPU-based
 * Distributed Algorithm for Linearized Optimal Power Flow in Distribution
 * Systems" (PSCC 2024).
 *
 * The library builds the LP of Sec. II-A (Eq. LP_model) from feeder arrays,
 * splits it into bus, line and merged-leaf subsystems (Sec. V-A) to obtain the
 * consensus form of Eq. OurModel, computes each subsystem's closed-form
 * projector once (Eq. closed_2, Algorithm 1 precomputation) and runs the ADMM
 * iteration of Algorithm 1 on one CUDA device: global update (Eq. closed_1),
 * local update (Eq. closed_2), dual update (Eq. ADMM-3) and the residuals and
 * stopping test of Sec. III-C.
 *
 * Conventions
 *  - Every function returns an int status: OPF_OK (0), OPF_NOT_CONVERGED (1)
 *    or a negative OPF_E_* code; opf_strerror() names it.
 *  - Input arrays are host memory owned by the caller and are copied during
 *    the call; nothing is retained.  Output arrays are caller-allocated host
 *    memory with the stated lengths (checked where a length is passed).
 *  - The library allocates and owns all device memory of a handle.
 *  - A handle is not thread safe; use one handle per host thread.  All device
 *    work of a handle runs on its stream (opf_options.stream, or a stream the
 *    library creates); calls return after that work has finished.
 *  - Variable order ("canonical order") of x, the global vector of
 *    Eq. OurModel:  generators (for each gen, each phase a<b<c: p^g, q^g),
 *    buses (each bus, each phase: w), loads (each load, each phase:
 *    p^b, q^b, p^d, q^d), lines (each line, each phase: p_eij, q_eij, p_eji,
 *    q_eji).  Subsystem order: every non-leaf bus in bus order, then every
 *    line in line order (a line whose to-bus is a leaf also holds that bus).
 *    Local slots of a subsystem: ascending global index.  Stacked local
 *    vectors (x_s, lambda_s) are the subsystems' slots concatenated in
 *    subsystem order.
 */
#ifndef OPF_H
#define OPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OPF_OK                  0
#define OPF_NOT_CONVERGED       1   /* max_iter reached; results are readable */
#define OPF_E_INVALID          -1   /* malformed input (message: opf_last_error) */
#define OPF_E_INFEASIBLE_LOCAL -2   /* a local system A_s x_s = b_s is inconsistent */
#define OPF_E_STATE            -3   /* call out of order (e.g. solve before precompute) */
#define OPF_E_OOM              -4   /* device or host allocation failed */
#define OPF_E_NUMERIC          -5   /* NaN or Inf in the residual reductions */
#define OPF_E_TIMEOUT          -6   /* a bounded device wait gave up */
#define OPF_E_CUDA             -7   /* CUDA runtime error */
#define OPF_E_CAPACITY         -8   /* size beyond a documented limit */

/* Precision of the iterations (Sec. IV runs the GPU in single precision). */
#define OPF_PREC_FP64   0   /* plain FP64 iterations */
#define OPF_PREC_FP32   1   /* FP32 iterations, FP64 reductions, no refinement */
#define OPF_PREC_MIXED  2   /* FP32 iterations re-centred in FP64, then FP64 polish */

/* Largest subsystem size n_s the iteration kernels accept. */
#define OPF_MAX_NS 256

/* Radial three-phase feeder (Table I nomenclature).  Phase sets are bit masks
 * (bit 0 = a, 1 = b, 2 = c).  Per-phase arrays have 3 entries per component
 * (index = phase), entries of absent phases are ignored.  Bus 0 is the
 * substation; every other bus has exactly one incoming line (line_to), its
 * phases equal that line's, and a line's phases are a subset of its from-bus
 * phases.  Units: powers in p.u., impedances in p.u., voltage squared in p.u.
 * Infinite bounds are IEEE +-INFINITY. */
typedef struct opf_feeder {
    int32_t n_bus;
    const uint8_t *bus_phases;      /* [n_bus] */
    const double *bus_wmin;         /* [n_bus*3] bounds on w (Eq. operational) */
    const double *bus_wmax;         /* [n_bus*3] */
    const double *bus_gsh;          /* [n_bus*3] shunt conductance g^sh (Eq. balance_eqns) */
    const double *bus_bsh;          /* [n_bus*3] shunt susceptance b^sh */

    int32_t n_line;                 /* must be n_bus - 1 */
    const int32_t *line_from;       /* [n_line] from bus i (towards the substation) */
    const int32_t *line_to;         /* [n_line] to bus j */
    const uint8_t *line_phases;     /* [n_line] */
    const double *line_r;           /* [n_line*9] 3x3 resistance, row-major */
    const double *line_x;           /* [n_line*9] 3x3 reactance, row-major */
    const double *line_gs_from;     /* [n_line*3] g^s_eij (Eq. power_flow_eqns) */
    const double *line_bs_from;     /* [n_line*3] b^s_eij */
    const double *line_gs_to;       /* [n_line*3] g^s_eji */
    const double *line_bs_to;       /* [n_line*3] b^s_eji */
    const double *line_tap;         /* [n_line*3] tap ratio tau */

    int32_t n_load;
    const int32_t *load_bus;        /* [n_load] */
    const uint8_t *load_phases;     /* [n_load] equal to its bus's phases */
    const uint8_t *load_delta;      /* [n_load] 0 = wye, 1 = delta (three-phase only) */
    const double *load_a;           /* [n_load*3] a (Eq. VDLM-1) */
    const double *load_b;           /* [n_load*3] b (Eq. VDLM-2) */
    const double *load_alpha;       /* [n_load*3] alpha >= 0 */
    const double *load_beta;        /* [n_load*3] beta >= 0 */

    int32_t n_gen;
    const int32_t *gen_bus;         /* [n_gen] */
    const uint8_t *gen_phases;      /* [n_gen] subset of its bus's phases */
    const double *gen_pmin;         /* [n_gen*3] */
    const double *gen_pmax;
    const double *gen_qmin;
    const double *gen_qmax;
    const double *gen_cost;         /* [n_gen] linear cost on every phase's p^g */
} opf_feeder;

typedef struct opf_options {
    int32_t device;                 /* CUDA device ordinal */
    void *stream;                   /* cudaStream_t to run on, or NULL */
} opf_options;

typedef struct opf_solve_opts {
    double rho;                     /* penalty (the paper's default is 100) */
    double eps_rel;                 /* epsilon_rel of the Sec. III-C test */
    double eps_abs_pres;            /* absolute gate: also require pres <= this */
    int32_t max_iter;               /* iteration cap (counts every iteration), applied at the
                                       tests: rounded up to a multiple of check_every */
    int32_t check_every;            /* iterations between tests; even, >= 2 */
    int32_t precision;              /* OPF_PREC_* */
    int32_t recenter_every;         /* OPF_PREC_MIXED: iterations between FP64 re-centrings (0 = default) */
    int32_t engine;                 /* 0 = automatic, 1 = whole-grid kernels, 2 = cluster resident,
                                       3 = warp per subsystem (one cluster of at most 16 CTAs: at
                                           most 192 subsystems of at most 64 slots; FP32 factors
                                           of at most 32 slots in registers, FP64 factors in
                                           shared memory),
                                       4 = persistent grid (cooperative launch, instance resident in
                                       the shared memory of all CTAs, one grid barrier per iteration) */
    int32_t flags;                  /* OPF_SOLVE_* bits */
    int32_t cluster;                /* engine 2: CTAs per cluster (1, 2, 4, 8, 16; 0 = automatic);
                                       engine 3: CTAs of the cluster (1 .. 16, at most 12
                                       subsystems per CTA; 0 = automatic);
                                       engine 4: CTAs of the grid (1 .. 2048, at most the resident
                                       count; 0 = automatic) */
} opf_solve_opts;

/* opf_solve_opts.flags: drive the iteration chunks from the host (one plain
 * CUDA graph per chunk and a status read after each) instead of one graph
 * with a device-side WHILE node; same arithmetic, slower, profiler-visible. */
#define OPF_SOLVE_HOST_LOOP 1
/* Test hook for the failure path of the persistent grid engine (engine 4):
 * its grid barriers expect one CTA more than the launch has, so the first
 * bounded wait runs out (about 1 s), every CTA leaves, and the solve returns
 * OPF_E_TIMEOUT with the handle still usable (reset or re-solve). */
#define OPF_SOLVE_TEST_BARRIER_TIMEOUT 2

typedef struct opf_sizes {
    int64_t n_global;               /* n: length of x */
    int64_t n_sub;                  /* S */
    int64_t n_slots;                /* L = sum n_s */
    int64_t n_rows;                 /* sum m_s */
    int64_t sum_nf;                 /* sum n_s * f_s of the stored factors (after precompute) */
    int64_t max_ns;
    int64_t h2d_bytes;              /* bytes copied host -> device by opf_create */
} opf_sizes;

typedef struct opf_handle opf_handle;

/* Build the LP of Eq. LP_model from a feeder, decompose it (Sec. V-A) and
 * upload the subsystems.  Errors: OPF_E_INVALID (malformed feeder),
 * OPF_E_CAPACITY (a subsystem larger than OPF_MAX_NS), OPF_E_CUDA, OPF_E_OOM. */
int opf_create(const opf_feeder *f, const opf_options *o, opf_handle **out);

/* Consensus form of Eq. OurModel given directly: n globals with cost c,
 * bounds lb/ub and an optional is_voltage flag (start value 1, Sec. V-A);
 * S subsystems with m_s rows and n_s slots; A (row-major m_s x n_s blocks
 * concatenated), b (m_s entries each) and idx (n_s distinct global indices
 * each, in the subsystem's slot order) concatenated over s.  Every global
 * must appear in some subsystem. */
int opf_create_generic(int32_t n, const double *c, const double *lb, const double *ub,
                       const uint8_t *is_voltage, int32_t S, const int32_t *m_s,
                       const int32_t *n_s, const double *A, const double *b,
                       const int32_t *idx, const opf_options *o, opf_handle **out);

/* Algorithm 1 precomputation (Sec. III-B) on the device in FP64: for each
 * subsystem an orthonormal basis of row(A_s) by Gram-Schmidt with
 * re-orthogonalisation (dependent rows dropped after a consistency check),
 * the projector -Abar_s kept as the smaller of Q Q^T-complement or a null-space
 * basis, and bbar_s = A_s^+ b_s.  Resets the iterate to the Sec. V-A start.
 * Idempotent.  Errors: OPF_E_INFEASIBLE_LOCAL, OPF_E_CUDA. */
int opf_precompute(opf_handle *h);

/* Run Algorithm 1 from the current state until the Sec. III-C test holds with
 * epsilon_rel = eps and pres <= 1e-4, or max_iter iterations (FP64).
 * Returns OPF_OK, OPF_NOT_CONVERGED, OPF_E_STATE, OPF_E_NUMERIC, OPF_E_CUDA. */
int opf_solve(opf_handle *h, double rho, double eps, int32_t max_iter);

/* Same with every option (NULL = defaults: rho 100, eps_rel 1e-8,
 * eps_abs_pres 1e-4, max_iter 1e6, check_every 50, FP64).  Automatic engine
 * choice: FP32 / mixed iterations on the warp engine, else the cluster
 * engine, else the persistent grid engine, else whole-grid kernels; FP64
 * iterations (and the polish) on the warp engine when the instance fits it
 * with at most 4 warps per CTA (at most 64 subsystems), else on the
 * persistent grid engine when its plan fits, else whole-grid kernels.  The persistent engine's grid
 * barrier waits at most 1 s; past that the solve returns OPF_E_TIMEOUT. */
int opf_solve_ex(opf_handle *h, const opf_solve_opts *opts);

/* Exactly n_iters FP64 iterations with penalty rho, no stopping test. */
int opf_step(opf_handle *h, double rho, int32_t n_iters);

/* Reset the iterate to the Sec. V-A start (lambda = 0). */
int opf_reset(opf_handle *h);

/* Global solution x (n entries, canonical order) and c^T x of the last
 * iteration.  x may be NULL. */
int opf_get_solution(opf_handle *h, double *x, size_t n, double *objective);

/* Residuals of the last tested iteration (Sec. III-C); eps_prim and eps_dual
 * are given for epsilon_rel = 1, i.e. the two norms the test scales.  Any
 * pointer may be NULL. */
int opf_get_residuals(opf_handle *h, double *pres, double *dres, double *eps_prim,
                      double *eps_dual, int64_t *iters);

/* Stacked local copies x_s and duals lambda_s (L entries each, canonical
 * order); either may be NULL.  opf_set_locals restores them (warm start or
 * checkpoint); the global x is recomputed by the next iteration. */
int opf_get_locals(opf_handle *h, double *xs, double *lam, size_t L);
int opf_set_locals(opf_handle *h, const double *xs, const double *lam, size_t L);

/* Sizes of the handle's model (opf_sizes above; sum_nf after opf_precompute).
 * OPF_E_INVALID for a NULL handle or output. */
int opf_get_sizes(opf_handle *h, opf_sizes *out);

/* New load values for a feeder handle (host arrays [n_load*3] like
 * opf_feeder.load_a / load_b): the right-hand sides of the load rows change,
 * and with a ZIP exponent (alpha or beta > 0) also their w coefficients
 * (VDLM-1..5), so M_s depends on the scenario; call opf_precompute again
 * before iterating (OPF_E_STATE until then).  A batch created from the handle
 * must be destroyed first.  OPF_E_INVALID for generic handles. */
int opf_set_loads(opf_handle *h, const double *load_p, const double *load_q);

/* Statistics of the last precompute/solve (device times from CUDA events on
 * the handle's stream): [0] precompute ms, [1] main iteration phase ms,
 * [2] FP64 polish ms, [3] iterations in the main phase, [4] iterations in the
 * polish, [5] re-centrings.  n = number of entries wanted (<= 6). */
int opf_get_timing(opf_handle *h, double *ms, int n);

/* Allocation-free global update, for callers that cannot allocate device
 * memory: control loops that forbid allocation once they run (an allocation
 * may block, or fail when memory is short, at any moment), and hosts whose
 * device memory is handed out only by their own allocator (a framework's
 * caching allocator that owns the whole device).  The paper has no
 * counterpart: this is the global update and the objective c^T x (what
 * opf_get_solution returns) over caller device arrays, without a handle.
 *   n          number of globals, 1 <= n <= OPF_STATIC_MAX_GLOBALS
 *   seg_off    device, n + 1 int32 offsets: the local copies of global i are
 *              u[seg_off[i] .. seg_off[i+1]) (at least one each)
 *   u          device, seg_off[n] doubles: rho x_k - lambda_k of every copy,
 *              grouped by global (summed in that order)
 *   c, lb, ub  device, n doubles each (bounds may be +-INFINITY)
 *   rho        > 0
 *   x          device, n doubles out: clip((sum u - c_i) / (rho N_i), lb_i, ub_i)
 *   objective  device, 1 double out: c^T x
 *   stream     cudaStream_t (NULL = legacy default stream); the call only
 *              enqueues work, synchronise the stream before reading outputs.
 * Scratch is a fixed device array of OPF_STATIC_MAX_BLOCKS doubles, one per
 * block of 256 globals, held by every device that loads the library until
 * the process exits.  The first call in a CUDA context (the stream's; a
 * stream of an SM partition has its own) is the set-up: it looks up the
 * array's address in that context, and the CUDA driver may load the
 * library's device code into the context then; later calls in the context
 * allocate nothing.  Make that first call before any stream capture.  Every call in a context shares the array: calls that may
 * overlap on the GPU (different streams without ordering) race and must be
 * serialised by the caller.  Each call writes every entry it reads, so stale
 * contents from an earlier call are never used.
 * Returns OPF_OK, OPF_E_INVALID (null pointer, n < 1, rho <= 0),
 * OPF_E_CAPACITY (n above the limit; message in opf_last_error), OPF_E_CUDA. */
#define OPF_STATIC_MAX_BLOCKS 8192
#define OPF_STATIC_MAX_GLOBALS (256 * OPF_STATIC_MAX_BLOCKS)
int opf_global_update_static(int32_t n, const int32_t *seg_off, const double *u, const double *c,
                             const double *lb, const double *ub, double rho, double *x,
                             double *objective, void *stream);

/* ------------------------------------------------------------------ batches
 * Many instances of one model solved together.  Every instance shares the
 * handle's A_s, c and bounds (the local systems of Sec. III-B, hence M_s =
 * -Abar_s) and has its own right-hand side b, so its own bbar = A_s^+ b.
 * Load scenarios of one feeder are such instances when every load has
 * constant power (alpha = beta = 0 in VDLM-1..5): the loads enter only the
 * rhs of the p^d, q^d rows.  Each instance runs Algorithm 1 with its own
 * Sec. III-C test and stops on its own; the iterations of all instances are
 * advanced together by one persistent kernel per re-centring interval (a CUDA
 * graph loops until every instance stopped).
 * The batch keeps a pointer to the handle: destroy the batch first.  Not
 * thread-safe; the handle's stream orders all work. */
typedef struct opf_batch opf_batch;

/* n_inst >= 1 instances, each starting as a copy of the handle's own rhs and
 * at the start point of Sec. V-A.  Needs a precomputed handle (OPF_E_STATE);
 * computes A_s^+ once per handle (FP64).  OPF_E_OOM if device memory is short. */
int opf_batch_create(opf_handle *h, int32_t n_inst, opf_batch **out);

/* rhs of instances [first, first + count): host array of count * n_rows
 * doubles, instance-major, rows in canonical order (subsystems in creation
 * order, each subsystem's rows in its own order; n_rows from opf_get_sizes).
 * The instances restart from the start point.  OPF_E_INFEASIBLE_LOCAL if some
 * A_s x_s = b_s has no solution for an instance (message names it). */
int opf_batch_set_rhs(opf_batch *b, int32_t first, int32_t count, const double *rhs);

/* Same from load values (feeder handles): load_p, load_q are host arrays of
 * count * n_load * 3 doubles, [instance][load][phase] like opf_feeder.load_a /
 * load_b (entries of absent phases are ignored).  OPF_E_INVALID for generic
 * handles or when a load has a ZIP exponent (then A_s depends on the loads). */
int opf_batch_set_loads(opf_batch *b, int32_t first, int32_t count, const double *load_p,
                        const double *load_q);

/* As opf_batch_set_loads with load_p, load_q in device memory of the
 * handle's device (no host transfer); the caller keeps them alive until the
 * handle's stream has passed this call. */
int opf_batch_set_loads_device(opf_batch *b, int32_t first, int32_t count, const double *load_p,
                               const double *load_q);

/* Runs every instance to its own stopping test (options as opf_solve_ex;
 * engine and cluster ignored).  OPF_PREC_MIXED: FP32 iterations re-centred
 * every recenter_every iterations (0: 4000) on an FP64 reference, then FP64 iterations
 * until the test holds in FP64 (this polish tests every 2 iterations, for at
 * most 2 check_every iterations).  Returns OPF_OK when every instance
 * converged, OPF_NOT_CONVERGED when some hit max_iter (per-instance results in
 * opf_batch_get_status), OPF_E_NUMERIC on NaN/Inf. */
int opf_batch_solve(opf_batch *b, const opf_solve_opts *opts);

/* n_iters FP64 iterations of every instance without the test (for checking
 * against a reference implementation iteration by iteration). */
int opf_batch_step(opf_batch *b, double rho, int32_t n_iters);

/* Engine shape for one precision (OPF_PREC_FP32 or OPF_PREC_FP64): k_inst
 * instances per CTA (power of two <= 32) and warps per CTA (<= 16); 0 = pick
 * (FP32: the fastest of the candidate shapes timed on the batch; FP64: the
 * largest k_inst <= 4 that fits).  FP32 k_inst = 128 selects the lane engine
 * (never picked automatically; several times slower than the other shapes on
 * the feeders measured): one instance per lane, tiles of 128 instances, each
 * on a cluster of up to 16 CTAs that split the subsystems; warps 4, 8, 12 or
 * 16 per CTA (OPF_E_CAPACITY at the solve when the model needs more than 16
 * parts of at most 256 slots).  out (get): ok, k_inst, warps, chunks per lane, tasks,
 * chunks per CTA (lane engine: per tile), shared bytes, CTAs (lane engine:
 * tiles), lambda and bbar~ in tensor memory (1/0), tensor-memory columns per
 * CTA, CTAs per cluster (lane engine, else 0). */
int opf_batch_set_shape(opf_batch *b, int32_t precision, int32_t k_inst, int32_t warps);
int opf_batch_get_shape(opf_batch *b, int32_t precision, int32_t *out, int32_t n_out);

/* FP32 engine storage, an implementation choice with no counterpart in the
 * paper (default 1): with 1, a plan whose warp count is a
 * multiple of 4 keeps lambda and bbar~ of its CTA's instances in tensor
 * memory (tcgen05 TMEM, allocated per CTA for each launch) when they fit in
 * 512 columns per lane quadrant, instead of streaming them from L2 every
 * iteration; 0 streams them.  The arithmetic and the iterates are the same
 * either way.  The FP32 plan is rebuilt at the next solve. */
int opf_batch_set_tmem(opf_batch *b, int32_t enable);

/* Global x (count * n_global doubles, canonical order) and objective c^T x of
 * instances [first, first + count) after the last solve or step; either
 * output may be NULL. */
int opf_batch_get_solution(opf_batch *b, int32_t first, int32_t count, double *x, double *objective);

/* Per instance: res[4 i ..] = pres, dres, eps_prim, eps_dual of its last
 * test (eps_prim and eps_dual for epsilon_rel = 1, i.e. the two norms the
 * test scales, as opf_get_residuals), iterations, converged flag (any output
 * may be NULL). */
int opf_batch_get_status(opf_batch *b, int32_t first, int32_t count, double *res, int32_t *iters,
                         int32_t *converged);

/* x_s and lambda of one instance, canonical slot order (n_slots each). */
int opf_batch_get_locals(opf_batch *b, int32_t inst, double *xs, double *lam);

/* Warm start, an opt-in acceleration (the paper starts every solve from the
 * point of Sec. V-A): instances whose rhs or loads are set after this call
 * start from x_s = xs and lambda = lam (host arrays of n_slots doubles,
 * canonical slot order, e.g. opf_get_locals of a converged solve of the
 * same feeder at base load) instead of that point.  ADMM converges to the
 * same LP optimum from any start; the iterates differ from the paper's.
 * xs = lam = NULL returns to the Sec. V-A start.  OPF_E_INVALID for one
 * NULL array or a non-finite entry, OPF_E_OOM. */
int opf_batch_set_start(opf_batch *b, const double *xs, const double *lam);

/* Last solve: [0] FP32 phase ms, [1] FP64 phase ms, [2] autotune ms (0 when
 * the shape was known), [3] mean iterations, [4] converged instances,
 * [5] FP32 loop passes (engine launches), [6] FP64 loop passes, [7] FP32
 * engine-kernel ms alone (timed only with OPF_SOLVE_HOST_LOOP, else 0). */
int opf_batch_get_timing(opf_batch *b, double *out, int32_t n_out);

/* (k_inst, warps, ms) triples timed by the last FP32 autotune; returns how
 * many values exist (out may be NULL). */
int opf_batch_get_tune_log(opf_batch *b, double *out, int32_t n_out);

void opf_batch_destroy(opf_batch *b);

/* ------------------------------------------------------------------ server
 * OPF solves of several feeders and load scenarios that arrive over time,
 * served with continuous batching: each model (feeder topology) keeps the
 * ADMM state of its running requests resident on the device, admits queued
 * requests into free slots as earlier ones finish, and advances all of them
 * together; models run on separate streams.  Every request runs Algorithm 1
 * in FP32 (re-centred every chunk_iters iterations) until its Sec. III-C
 * test holds, then in FP64 until the test holds there (or max_iter).  A
 * request's result does not depend on the other requests in flight.  Not
 * thread-safe: one host thread drives a server. */
typedef struct opf_server opf_server;

typedef struct opf_server_opts {
    double rho, eps_rel, eps_abs_pres;  /* the stopping test, as opf_solve_opts */
    int32_t max_iter;               /* per request (rounded up to a multiple of check_every) */
    int32_t check_every;            /* iterations between tests; even, >= 2 */
    int32_t chunk_iters;            /* iterations per pass (a multiple of check_every) */
    int32_t keep_solutions;         /* 1: keep x of finished requests for opf_server_take_solution */
    int64_t mem_budget;             /* device bytes for request slots over all models (0: no limit) */
    int32_t polish_chunk_iters;     /* FP64 iterations per pass for slots in the polish (a multiple of
                                       check_every; 0 = 2 x check_every): FP64 iterations cost several
                                       times FP32 ones, and a model's next pass waits for both */
    int32_t reserved;               /* 0 */
} opf_server_opts;

int opf_server_create(const opf_server_opts *o, opf_server **out);

/* Adds a model served from n_handles precomputed feeder handles of the same
 * topology (the server keeps the pointers; destroy the server first).  When
 * the batched engine holds the model, handles[0] carries a batch of up to
 * `capacity` request slots (fewer if the memory budget is short); otherwise
 * each handle serves one request at a time on a worker thread (single-
 * instance engines; also for loads with ZIP exponents, where every request
 * needs its own factorization).  model_id receives the model's index.  OPF_E_STATE if
 * handles[0] is not precomputed, OPF_E_CAPACITY if the budget admits no slot. */
int opf_server_add_model(opf_server *s, opf_handle *const *handles, int32_t n_handles, int32_t capacity,
                         int32_t *model_id);

/* Stopping test of one model's requests (default: the server's eps_rel and
 * eps_abs_pres), for requests admitted after the call; e.g. a tighter
 * eps_rel for a feeder whose norms run over many more slots.  OPF_E_INVALID
 * for an unknown model or a negative or NaN tolerance. */
int opf_server_set_model_tolerance(opf_server *s, int32_t model, double eps_rel, double eps_abs_pres);

/* FP32 engine shape of a batched model (as opf_batch_set_shape: k_inst
 * instances per CTA, warps per CTA; 0, 0 = the shape timed fastest on a full
 * batch of the model's slots), for passes started after the call.  The
 * default favours throughput when every slot runs; a model whose requests
 * keep only part of its slots busy is served with lower latency by a smaller
 * k_inst (more CTAs, less work each, on otherwise idle SMs): on the 123-bus
 * feeder an iteration takes about 8.4 us with 8 instances per CTA and 6 us
 * with 2.  The shape stays fixed until the next call, so a request's result
 * does not depend on the other requests.  The paper has no serving layer, so
 * no passage defines this.  OPF_E_INVALID for an unknown model, a model
 * served by worker threads or an invalid shape; OPF_E_STATE while a pass of
 * the model is in flight; OPF_E_CAPACITY when the shape does not hold the
 * model. */
int opf_server_set_model_shape(opf_server *s, int32_t model, int32_t k_inst, int32_t warps);

/* Warm start of one model's requests (opt-in, as opf_batch_set_start): every
 * request admitted after the call starts from x_s = xs, lambda = lam
 * (n_slots doubles each, canonical slot order) instead of the Sec. V-A
 * point; the start is fixed per model, so a result still does not depend on
 * the other requests.  NULL, NULL returns to the Sec. V-A start. */
int opf_server_set_model_start(opf_server *s, int32_t model, const double *xs, const double *lam);

/* Admission policy of one model (default: no bounds; 0 = no bound); the
 * paper has no serving layer, so no passage defines it.
 * max_queue bounds the requests waiting for a slot.  max_wait_s bounds the
 * seconds a request may wait for one: at submit the wait is predicted from
 * the requests ahead (queued and running, served `slots` at a time) and the
 * model's mean service time so far (before any of its requests finished:
 * the longest time a running one has run, a lower bound on the service
 * time), and a queued request that has waited
 * longer is shed by opf_server_step.  max_service_s bounds the seconds a
 * request may run once admitted: a batched slot past it is retired at the
 * end of a pass, a worker's solve stops at its next chunk.  Shed and stopped
 * requests are reported by opf_server_poll_ex with status OPF_E_TIMEOUT
 * (objective NaN), refused ones get OPF_E_CAPACITY from opf_server_submit,
 * so with the bounds set no request stays pending without a status when the
 * arrivals exceed what the model can serve.  OPF_E_INVALID for an unknown
 * model or a negative bound. */
int opf_server_set_admission(opf_server *s, int32_t model, int32_t max_queue, double max_wait_s,
                             double max_service_s);

/* Queues a request of model `model` with its loads (host arrays [n_load*3],
 * copied) and a caller tag that identifies it in opf_server_poll.  Returns
 * OPF_E_CAPACITY, with the request counted as refused and not queued, when
 * the model's admission policy turns it away (message in opf_last_error). */
int opf_server_submit(opf_server *s, int32_t model, const double *load_p, const double *load_q, int64_t tag);

/* Progress without blocking: for each model whose previous pass finished,
 * retire finished requests, admit queued ones and start the next pass (every
 * running request advances by chunk_iters iterations per pass); worker
 * threads of single-instance models start queued requests.  Call it in a
 * loop; models progress independently of one another. */
int opf_server_step(opf_server *s);

/* Up to max_n finished requests (in finishing order): tag, converged flag,
 * objective c^T x, iterations and latency in seconds from submit to finish
 * (any array may be NULL).  Returns how many were written (>= 0). */
int opf_server_poll(opf_server *s, int64_t *tags, int32_t *converged, double *objective, int32_t *iters,
                    double *latency_s, int32_t max_n);
/* Same with each request's status: OPF_OK (served; converged or not as the
 * flag says), OPF_E_NUMERIC, OPF_E_TIMEOUT (shed or stopped by the admission
 * policy, objective NaN) or the error of a failed single-instance solve. */
int opf_server_poll_ex(opf_server *s, int64_t *tags, int32_t *status, int32_t *converged, double *objective,
                       int32_t *iters, double *latency_s, int32_t max_n);

/* x (n_global doubles) of a finished request when keep_solutions is set. */
int opf_server_take_solution(opf_server *s, int64_t tag, double *x, int32_t n);

/* [0] submitted (refused ones included), [1] polled, [2] queued,
 * [3] running, [4] slots, [5] passes, [6] device bytes held for slots. */
int opf_server_stats(opf_server *s, int64_t *out, int32_t n);
/* Serving statistics (no counterpart in the paper).  Per model: [0]
 * submitted, [1] served (finished after running, stopped
 * ones included), [2] of those converged, [3] refused at submit, [4] shed
 * from the queue, [5] queued, [6] running, [7] slots, [8] mean service time
 * in microseconds, [9] stopped by the service bound (part of [1]).
 * submitted = served + refused + shed + queued + running. */
int opf_server_model_stats(opf_server *s, int32_t model, int64_t *out, int32_t n);

void opf_server_destroy(opf_server *s);

/* ------------------------------------------------------------------ shards
 * One instance split over several GPUs (one shard per GPU), the multi-GPU
 * form of the server/agent exchange of Sec. IV reduced to what Algorithm 1
 * needs: a shard holds a subset of the subsystems; the global update of
 * Eq. closed_1 for a global whose copies lie on several shards (a cut
 * global) needs the sum over all shards of sigma_i = sum_k (rho x_k -
 * lambda_k), which the caller exchanges (an all-reduce over the cut) between
 * opf_shard_partial and opf_shard_step.  The cut is the same list on every
 * shard (every global with copies on more than one part, ascending), so the
 * exchange is a plain sum of equal-length arrays.  Every shard then computes the same
 * x_i, so the iterates equal the unsharded instance's.  FP64 iterations.
 * A shard is not thread-safe; all its work is ordered on its stream. */
typedef struct opf_shard opf_shard;

/* Part of every subsystem (n_sub = subsystem count of the feeder's model,
 * canonical order): the buses in depth-first order from the substation cut
 * into n_parts contiguous ranges of balanced work (n_s^2 summed over the
 * subsystems anchored at a bus: a bus subsystem at its bus, a line subsystem
 * at its to-bus), so each part is a run of whole subtrees.  Host only.
 * OPF_E_INVALID for a malformed feeder or a wrong n_sub. */
int opf_partition(const opf_feeder *f, int32_t n_parts, int32_t *sub_part, int32_t n_sub);

/* Shard `part` of the feeder under the partition sub_part (n_sub entries):
 * its subsystems over the globals they touch (local globals, ascending global
 * index); the cut (n_cut entries, the same on every shard) lists the globals
 * with copies on more than one part; the objective counts a global on the
 * lowest part holding it.  The feeder arrays are
 * copied.  OPF_E_INVALID if the part is empty. */
int opf_shard_create(const opf_feeder *f, const int32_t *sub_part, int32_t n_sub, int32_t part,
                     const opf_options *o, opf_shard **out);
/* FP64 precompute of the shard's subsystems; the iterate goes to the
 * Sec. V-A start. */
int opf_shard_precompute(opf_shard *sh);
/* Local globals, cut globals (of all shards), local copies (slots). */
int opf_shard_sizes(opf_shard *sh, int32_t *n_global, int32_t *n_cut, int32_t *n_slots);
/* Global index (whole instance) of every local global, and of every cut
 * global in the order of the sigma arrays (host arrays; either may be NULL). */
int opf_shard_maps(opf_shard *sh, int32_t *global_of_local, int32_t *cut_global);
/* Enqueues on the shard's stream: sig[j] = this shard's part of sigma of cut
 * global j from the current iterate, 0 where it holds no copy (device array
 * of n_cut doubles). */
int opf_shard_partial(opf_shard *sh, double rho, double *sig);
/* Enqueues one FP64 iteration with sig_tot (device, n_cut doubles: sigma
 * summed over all shards, as opf_shard_partial produced before this step).
 * sums (device, 6 doubles, or NULL): this shard's part of the Sec. III-C sums
 * of the iteration, |x_g(k) - x_s,k|^2, |x_s - x_s,old|^2, |x_g(k)|^2,
 * |x_s|^2 over its slots, |lambda|^2 and its share of c^T x; add them over
 * the shards and apply opf_test_rule.  OPF_E_STATE without a preceding
 * opf_shard_partial at the same rho. */
int opf_shard_step(opf_shard *sh, double rho, const double *sig_tot, double *sums);
/* x per local global after the last step (host array), and x_s, lambda of the
 * shard's slots (as opf_get_locals on its subsystems). */
int opf_shard_get_x(opf_shard *sh, double *x);
int opf_shard_get_locals(opf_shard *sh, double *xs, double *lam, size_t n);
/* The cudaStream_t the shard's work is ordered on. */
void *opf_shard_stream(opf_shard *sh);
void opf_shard_destroy(opf_shard *sh);

/* The Sec. III-C test on summed squares (host): sums as opf_shard_step,
 * out (may be NULL) = pres, dres, eps_prim / eps_rel, eps_dual / eps_rel,
 * objective.  Returns 1 when pres <= eps_rel eps_prim, dres <= eps_rel
 * eps_dual and pres <= eps_abs_pres, 0 when not, OPF_E_NUMERIC on NaN. */
int opf_test_rule(const double *sums, double rho, double eps_rel, double eps_abs_pres, double *out);

/* Measurement helper, not part of the method: enqueues a kernel of
 * `blocks` x `threads` threads (threads a multiple of 32, at most 1024) in
 * which every thread runs 8 independent FP32 FMA chains for 16 * iters steps,
 * writing one float per thread to the device buffer out (blocks * threads
 * floats, caller-owned).  *flops (may be NULL) receives the launch's flop
 * count (2 per FMA); time the launch with events on `stream` for the FP32
 * FMA throughput of the device at its current clocks, the denominator of the
 * batched engine's roofline.  OPF_E_INVALID for bad sizes, OPF_E_CUDA. */
int opf_probe_fma(int32_t blocks, int32_t threads, int32_t iters, float *out, void *stream, double *flops);
/* The same with FP64 chains (out: blocks * threads doubles), for the FP64
 * FMA rate, the denominator of FP64 iterations. */
int opf_probe_dfma(int32_t blocks, int32_t threads, int32_t iters, double *out, void *stream, double *flops);

/* A CUDA stream whose kernels run only on a partition of the device's SMs
 * (a green context), e.g. to keep the long single-instance solves of large
 * feeders from taking the SMs the batched engine's resident CTAs need.
 * n_sm > 0: a partition of n_sm SMs (rounded up to the device's partition
 * granularity); n_sm < 0: the SMs left after setting -n_sm aside.  The
 * stream is non-blocking with the given priority; *sm_count receives the
 * partition's SM count.  Memory of the device is shared as usual.  Solves
 * on such a stream need OPF_SOLVE_HOST_LOOP (their while-loop graph cannot be
 * instantiated there).  Release with opf_stream_destroy_partition after the
 * work on it finished.
 * OPF_E_CUDA if the driver offers no green contexts. */
int opf_stream_create_partition(int32_t device, int32_t n_sm, int32_t priority, void **stream,
                                int32_t *sm_count);
/* Destroys a stream made by opf_stream_create_partition and its green
 * context; OPF_E_INVALID for any other stream. */
int opf_stream_destroy_partition(void *stream);

/* Frees the handle and all its device memory (NULL is a no-op); destroy its
 * batches and any server using it first. */
void opf_destroy(opf_handle *h);
/* Static name of a status code. */
const char *opf_strerror(int code);
/* Message of the last OPF_E_INVALID / OPF_E_CUDA on this thread. */
const char *opf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OPF_H */
