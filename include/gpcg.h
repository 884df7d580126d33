/*
 * gpcg.h -- C ABI of the GB300 N-1 contingency screen.
 *
 * The library solves the fast-decoupled power flow (Sec. III.B, eqs. (4)-(5))
 * of every single-branch outage scenario (Sec. IV.A) with conjugate gradient
 * preconditioned by a factorisation of the base-case matrix (Sec. IV.B,
 * eqs. (6)-(7)), after islanding detection and proportional re-dispatch
 * (Sec. IV.C).  Beyond branch outages: generator outages
 * (gpcg_n1_gen_screen), transformer turns ratios and PV reactive limits
 * (gpcg_grid), the P-theta quick screen (gpcg_n1_dc_screen) and the adjoint
 * of an overload penalty (gpcg_n1_adjoint).  All numerical work runs in CUDA
 * kernels on the current device; the host code only validates arguments,
 * analyses the sparsity structure once per grid, and enqueues work.
 *
 * Conventions
 *  - Buses and branches are 0-based.  Per-unit quantities.
 *  - Every function returns a gpcg_status; GPCG_OK is 0.  On error
 *    gpcg_last_error() returns a message for the calling thread, valid until
 *    that thread's next call into the library.
 *  - A context belongs to the device that was current at gpcg_create and
 *    must be used with that device current.  Calls on one context must not
 *    overlap (one host thread at a time).
 *  - Input arrays are borrowed for the duration of the call and copied.
 *    Output arrays are owned by the caller.  A NULL output pointer skips
 *    that output.
 *  - mem = GPCG_MEM_HOST: every array argument is host memory (pageable or
 *    pinned); the call returns after the results are in host memory.
 *    mem = GPCG_MEM_DEVICE: every array argument is device memory of the
 *    context's device; the work is ordered on `stream` (a cudaStream_t, or
 *    NULL for the legacy default stream) and the call returns once it is
 *    enqueued, except where a function says otherwise.
 */
#ifndef GPCG_H_
#define GPCG_H_

#include <stdint.h>

#if defined(__GNUC__)
#define GPCG_API __attribute__((visibility("default")))
#else
#define GPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPCG_OK = 0,
  GPCG_ERR_INVALID_ARG = 1,     /* bad size, index, pointer or option */
  GPCG_ERR_CUDA = 2,            /* a CUDA runtime call failed */
  GPCG_ERR_BASE_NOT_CONVERGED = 3, /* also: the base case needs PV generators
                                     outside their reactive limits */
  GPCG_ERR_BASE_ISLANDED = 4,   /* the intact grid is not connected */
  GPCG_ERR_TIMEOUT = 5,         /* a bounded device wait gave up (the grid-wide
                                   barriers of the plain FP64 path; see
                                   gpcg_options.wait_limit) */
  GPCG_ERR_OOM = 6,             /* a device allocation failed */
  GPCG_ERR_NOT_READY = 7        /* gpcg_base_solve has not succeeded yet */
} gpcg_status;

/* Per-scenario outcome written to status[] by the screens. */
enum {
  GPCG_SCEN_OK = 0,             /* converged to the mismatch tolerance */
  GPCG_SCEN_MAXITER = 1,        /* outer iteration cap reached */
  GPCG_SCEN_DIVERGED = 2,       /* non-finite or > 1e4 p.u. mismatch */
  GPCG_SCEN_ISLAND_NO_GEN = 3,  /* converged, but the main island had no
                                   generator to take the re-dispatch: the
                                   slack absorbed it */
  GPCG_SCEN_QLIM_OVERFLOW = 4   /* reactive limits: more buses had to be
                                   held at a limit at once than a scenario
                                   can hold (GPCG_MAX_EXT_ROWS rows, a tripped
                                   generator's bus included) */
};

/* B'' rows a scenario can add beyond the base case's PQ buses: a tripped
 * generator's bus and PV buses held at a reactive limit. */
#define GPCG_MAX_EXT_ROWS 8

enum { GPCG_PQ = 0, GPCG_PV = 1, GPCG_SLACK = 2 };        /* bus_type */

/* 32-bit words of one scenario's row of the branch overload mask. */
#define GPCG_MASK_WORDS(n_branch) (((n_branch) + 31) / 32)

enum { GPCG_MEM_HOST = 0, GPCG_MEM_DEVICE = 1 };

/* Precision of the inner PCG (the mismatch, state update and flows are
 * always FP64, Sec. II.C eqs. (1)-(3)). */
enum {
  GPCG_PLAIN_FP64 = 0,    /* one scenario at a time, FP64 vectors: the
                             unbatched comparison path */
  GPCG_BATCHED_FP32 = 1,  /* batched, FP32 vectors and factors; the FP64
                             outer loop acts as iterative refinement */
  GPCG_BATCHED_FP64 = 2,  /* batched, FP64 vectors and factors */
  GPCG_BATCHED_FP32_F16 = 3 /* batched, FP32 vectors; the base-case factor
                               stored scaled to a unit diagonal in FP16
                               (L = Ls D, Ls in FP16, D^-2 in FP32) */
};

/* Preconditioner built from the base-case matrix (Sec. IV.B, eq. (6)). */
enum {
  GPCG_PRECOND_IC0 = 0,    /* incomplete Cholesky, zero fill */
  GPCG_PRECOND_JACOBI = 1, /* diagonal of the contingency matrix, as in the
                              vertex update of the listing in Sec. III.B */
  GPCG_PRECOND_EXACT = 2   /* complete Cholesky of the base-case matrix:
                              eq. (6) read literally */
};

/* Bus/branch model of Sec. II.B (vertex and edge attributes).  Host
 * pointers.  Exactly one slack bus.  from[l] != to[l], x[l] > 0.
 * A transformer is a branch with an off-nominal turns ratio tap[l] (the
 * edge attribute "transformer turns ratio" of Sec. II.B): an ideal
 * tap[l]:1 transformer at the from end in series with the pi-model, no
 * phase shift, so with c = 1/tap[l]: Y_ff += c^2 (y + j b_sh/2),
 * Y_tt += y + j b_sh/2, Y_ft = Y_tf = -c y.  B'' takes the turns ratios
 * (w v v^T, v = c e_from - e_to), B' leaves them out (the XB scheme).
 * Outaging a transformer is a branch outage like any other.
 * Reactive limits (Q_min, Q_max; the paper models none): a PV generator's
 * output is Q(V) - Q_sched at its bus.  When a scenario has converged, every
 * PV bus whose generator is outside its limits turns PQ with the generator
 * held at the violated limit (Q_sched + Q_max or Q_min), B'' gains its row;
 * at the same check every held bus whose |V| has passed its set point (above
 * it at Q_max, below it at Q_min) turns back PV at the set point; the
 * iteration then goes on from the mismatch of that state.  At the result
 * every PV generator is within its limits and every held one on its side of
 * the set point.  A scenario holds at most GPCG_MAX_EXT_ROWS such rows at
 * once (GPCG_SCEN_QLIM_OVERFLOW beyond).  The base case must be within the
 * limits (gpcg_base_solve fails otherwise). */
typedef struct {
  int32_t n_bus;
  int32_t n_branch;
  const int8_t *bus_type;   /* [n_bus] GPCG_PQ / GPCG_PV / GPCG_SLACK */
  const double *P_sched;    /* [n_bus] scheduled net active injection */
  const double *Q_sched;    /* [n_bus] scheduled net reactive injection (PQ) */
  const double *P_gen;      /* [n_bus] scheduled generation: re-dispatch weights */
  const double *V_set;      /* [n_bus] |V| set point (PV, slack); start (PQ) */
  const int32_t *from;      /* [n_branch] */
  const int32_t *to;        /* [n_branch] */
  const double *r;          /* [n_branch] series resistance */
  const double *x;          /* [n_branch] series reactance, > 0 */
  const double *b_sh;       /* [n_branch] total line charging */
  const double *rating;     /* [n_branch] flow limit, > 0 */
  const double *tap;        /* [n_branch] turns ratio at the from end, > 0;
                               NULL: every branch is a line (ratio 1) */
  const double *Q_min;      /* [n_bus] reactive limits of the PV buses'    */
  const double *Q_max;      /* generators (Q_min <= Q_max); both NULL: none */
} gpcg_grid;

typedef struct {
  double tol;          /* outer tolerance on max |dP|, |dQ| (p.u.); 1e-4 */
  double base_tol;     /* tolerance of gpcg_base_solve; 1e-10 */
  double inner_rtol;   /* PCG stops at ||r|| <= inner_rtol ||b||; 3e-3 */
  int32_t max_outer;   /* outer FDPF iteration cap; 50 */
  int32_t max_inner;   /* PCG iteration cap per solve; 500 */
  int32_t precision;   /* GPCG_PLAIN_FP64 / _BATCHED_FP32 / _BATCHED_FP64 /
                          _BATCHED_FP32_F16 */
  int32_t precond;     /* GPCG_PRECOND_*; default GPCG_PRECOND_EXACT */
  int32_t tile;        /* scenarios per tile (the scenario chunk a CTA solves
                          together): 2, 4, 8, 16 or 32; 0 = autotuned */
  int32_t ctas_per_sm; /* resident tiles per SM, which sets the scenarios in
                          flight (tile x ctas_per_sm x SMs); 0 = autotuned
                          among the occupancy maximum and the two counts below
                          it */
  int32_t tail_rows;   /* level-tile shape of the substitutions: the factor's
                          last levels, together at most this many rows, are
                          solved with the dense inverse of their block
                          (1 ... GPCG_MAX_TAIL_ROWS), the levels before it one
                          block barrier each; -1 = no dense tail; 0 = autotuned */
  int32_t wait_limit;  /* bounded device waits: the polls (about 64 ns apart)
                          a grid-wide barrier of the plain FP64 path makes
                          before it gives up, which ends the call with
                          GPCG_ERR_TIMEOUT and leaves the context usable;
                          0 = 2^25 (about 2 s) */
} gpcg_options;

/* Largest dense tail of a factor (rows); the tail's right-hand side is kept
 * in shared memory. */
#define GPCG_MAX_TAIL_ROWS 248

/* The autotuner (options left at 0) runs on the first batched screen of a
 * context, and again when the number of scenarios of a call moves to another
 * power of two.  Every candidate screens the same probe: all of the call's
 * outages, or for calls of more than 16,384 (and more than eight times the
 * most scenarios a candidate keeps in flight) that many taken at an even
 * stride from the call's scheduling order; the fastest is kept, a candidate
 * replacing the one before it only when 3 % faster: first the tile width
 * (2, 4, 8), then the tiles per SM, then the dense tail (248, 128, 64 rows
 * or none).  Choices are cached
 * for the process, keyed by the device (SM count, compute capability), the
 * grid's sizes (buses, branches, nonzeros of B', B'' and their factors),
 * precision, preconditioner, kernel kind and the power of two of the
 * scenario count; a context whose key is cached takes the cached choice
 * without probing.  Every choice gives the same results up to the rounding
 * of the inner solve. */

/* Sizes of the structures built by gpcg_create. */
typedef struct {
  int32_t n_bus, n_branch, slack;
  int32_t n_p, n_q;            /* rows of B' (non-slack) and B'' (PQ) */
  int32_t nnz_p, nnz_q;        /* nonzeros of B', B'' */
  int32_t nnz_lp, nnz_lq;      /* nonzeros of the factors (lower, with diag) */
  int32_t levels_p, levels_q;  /* forward level-schedule depths */
  int32_t blevels_p, blevels_q;/* backward level-schedule depths */
  int32_t n_bridges;           /* branches whose outage islands buses */
  int32_t tile;                /* tile width in use (0 until chosen) */
  int32_t num_sms;
  int32_t base_outer;          /* outer iterations of the base solve, -1 if none */
  int32_t ctas_per_sm;         /* tiles per SM in use (0 until chosen) */
  int32_t tail_rows_p;         /* rows of the B' factor solved by the dense tail */
  int32_t tail_rows_q;         /* rows of the B'' factor solved by the dense tail */
  int32_t tuned;               /* 0: not tuned (or every knob fixed by options);
                                  1: chosen by probes; 2: taken from the cache */
} gpcg_info;

/* Fill *opt with the defaults listed above. */
GPCG_API gpcg_status gpcg_default_options(gpcg_options *opt);

typedef struct gpcg_ctx gpcg_ctx;   /* opaque; owned by the library */

/* Create a context for one grid (Sec. II.B).  Validates the grid, copies it
 * to the device, orders B' and B'' (minimum degree, then by level), builds
 * their CSR values in a kernel (Sec. III.B: diagonal on the vertex,
 * off-diagonal on the edge) and factorises the base-case matrices with a
 * level-scheduled kernel (Sec. IV.B, eq. (6)).  opt may be NULL (defaults);
 * it is copied.  Errors: INVALID_ARG (bad grid or options), BASE_ISLANDED,
 * OOM, CUDA.  On error *out is set to NULL.  Synchronous. */
GPCG_API gpcg_status gpcg_create(const gpcg_grid *grid, const gpcg_options *opt,
                        gpcg_ctx **out);

/* Release every device and host resource of the context.  NULL is a no-op. */
GPCG_API void gpcg_destroy(gpcg_ctx *ctx);

/* Replace the options of a live context (same rules as gpcg_create).
 * Changing `precond` re-factorises the base-case matrices. */
GPCG_API gpcg_status gpcg_set_options(gpcg_ctx *ctx, const gpcg_options *opt);

GPCG_API gpcg_status gpcg_get_info(const gpcg_ctx *ctx, gpcg_info *info);

/* Fast-decoupled power flow of the intact grid from a flat start
 * (theta = 0, |V| = V_set), FP64, to opt.base_tol (Sec. III.B eqs. (4)-(5)).
 * The result is kept in the context as the warm start of every N-1
 * scenario (Sec. III.B: convergence depends on the initial vector).
 * Host outputs, each optional: theta[n_bus], vm[n_bus], flow[n_branch]
 * (active power at the from end), iters[3] = {outer, inner P, inner Q}.
 * Errors: BASE_NOT_CONVERGED, CUDA.  Synchronous. */
GPCG_API gpcg_status gpcg_base_solve(gpcg_ctx *ctx, double *theta, double *vm,
                            double *flow, int32_t *iters);

/* The N-1 screen (Sec. IV.A): for each outage l = outages[s] (a branch
 * index) remove the branch, detect islands by connected components
 * (Sec. IV.C), re-dispatch the islands' net injection over the main island's
 * PV generators in proportion to P_gen (Sec. IV.C), solve the FDPF of the
 * main island from the base-case state with base-preconditioned CG
 * (Sec. IV.B), and screen the branch flows against their ratings (Sec. I).
 * The FDPF loop (Sec. III.B, eqs. (4)-(5)): evaluate dP and dQ; stop when
 * max|dP| (non-slack buses) and max|dQ| (PQ buses) are both within tol;
 * take the P-theta step unless max|dP| is already within tol; evaluate dQ;
 * take the Q-V step unless max|dQ| is then within tol; one outer iteration
 * per pass.
 * Islanded buses report theta = vm = 0; branches touching them, and the
 * outaged branch, report zero flow.
 *
 * Outputs, row-major per scenario, each optional except where noted:
 *   theta[n_out][n_bus], vm[n_out][n_bus]     FP64 state
 *   flow[n_out][n_branch]                     active power at the from end
 *   island_label[n_out][n_bus]                min bus index of each bus's
 *                                             component after the outage
 *   iters[n_out][3]                           {outer, inner P, inner Q}
 *   status[n_out]                             GPCG_SCEN_*
 *   max_loading[n_out]                        max over branches of
 *                                             max(|P_ij|,|P_ji|)/rating
 *   n_overload[n_out]                         branches whose loading
 *                                             max(|P_ij|,|P_ji|)/rating
 *                                             exceeds 1 (the violations
 *                                             the screen flags, Sec. I)
 *   overload[n_out][GPCG_MASK_WORDS(n_branch)] the same branches as a bit
 *                                             mask: bit k % 32 of word
 *                                             k / 32 is set for branch k
 * n_out may be 0.  An outage index outside [0, n_branch) is INVALID_ARG.
 * Requires a successful gpcg_base_solve (else NOT_READY).  A scenario that
 * fails to converge never fails the call: see status[].
 *
 * mem = 0: every pointer is host memory; the call returns with the results
 * written.  Outputs in page-locked host memory (cudaHostAlloc,
 * cudaHostRegister) are written by the kernels in place, through their
 * device-visible addresses, while the solve runs; other host outputs go
 * through device buffers copied back at the end.  mem = 1: every pointer
 * is device memory; the outage list is read
 * back to validate it and order the scenarios (a synchronisation of
 * `stream`), and the call returns once the solve is enqueued on `stream`.
 * In device mode the islanding and solve launches are captured once as a
 * CUDA graph, keyed on n_out, the output pointers and the options, and
 * replayed while that key holds (gpcg_set_options drops it).
 * Knobs left at 0 in the options (tile width, tiles per SM, dense tail) are
 * chosen by the autotuner described with gpcg_options on the first batched
 * screen of the context and whenever n_out moves to another power of two
 * (gpcg_info reports the choice and whether it came from the cache). */
GPCG_API gpcg_status gpcg_n1_screen(gpcg_ctx *ctx, const int32_t *outages, int32_t n_out,
                           int32_t mem, void *stream, double *theta, double *vm,
                           double *flow, int32_t *island_label, int32_t *iters,
                           int32_t *status, double *max_loading, int32_t *n_overload,
                           uint32_t *overload);

/* N-1 screen of generator outages (Sec. IV.A: the loss of a single
 * component).  Scenario s trips the generator of PV bus gen_buses[s]
 * (caller's numbering): that bus keeps its load -- P_sched - P_gen and
 * Q_sched, Q_sched being the reactive injection without the generator --
 * and no longer holds |V|, so it becomes a PQ bus; its P_gen is taken up by
 * the other PV generators with P_gen > 0 in proportion to theirs (the
 * re-dispatch rule of Sec. IV.C; with none left the slack absorbs it and
 * the status is GPCG_SCEN_ISLAND_NO_GEN).  No branch leaves service and
 * nothing is islanded (labels all 0).  The P-theta half-step solves with
 * the base-case B' itself; the Q-V half-step's B'' gains the bus's row, and
 * the base-case factor preconditions the other rows while that row is
 * preconditioned by its diagonal.  Outputs, modes, the graph replay and the
 * tile autotuner as gpcg_n1_screen.  A bus that is not PV (or out of range)
 * is INVALID_ARG; the slack's generator cannot be tripped. */
GPCG_API gpcg_status gpcg_n1_gen_screen(gpcg_ctx *ctx, const int32_t *gen_buses, int32_t n_out,
                               int32_t mem, void *stream, double *theta, double *vm,
                               double *flow, int32_t *island_label, int32_t *iters,
                               int32_t *status, double *max_loading, int32_t *n_overload,
                               uint32_t *overload);

/* Loss and gradients of a smooth overload penalty summed over the N-1
 * scenarios of the P-theta (DC) model (eq. (4) with |V| = 1, Sec. IV.A's
 * quick screen).  For outage l = outages[s]:
 *   theta_s = B'_s^{-1} R_s P,   f_s = diag(b_s) A theta_s,
 *   loss = sum_s sum_k softplus(|f_ks| / rating_k - 1)^2,
 * where B'_s is the base matrix built from the susceptances b with the
 * outage's four-element change (Sec. IV.B), islands removed and their
 * injection re-dispatched with frozen weights (Sec. IV.C), R_s that
 * re-dispatch map.  The gradients take one more batched PCG solve per
 * scenario with the symmetric B'_s:
 *   dL/dP = sum_s R_s^T lambda_s,  lambda_s = B'_s^{-1} A^T diag(b_s) g_s,
 *   dL/db_k = sum_s [g_ks (A theta_s)_k - (A lambda_s)_k (A theta_s)_k],
 * with g = dloss/df.  The base case is factorised for the given b, and the
 * solves run in FP64.
 * Inputs: P[n_bus] bus injections (NULL: the grid's P_sched), b[n_branch]
 * branch susceptances, > 0 (NULL: 1/x).  Outputs: loss[1]; dL_dP[n_bus] and
 * dL_db[n_branch], each optional.  mem and stream as in gpcg_n1_screen; the
 * call returns when the results are written.  Sums over scenarios are taken
 * in a fixed order (deterministic).  Errors: INVALID_ARG, OOM, CUDA. */
GPCG_API gpcg_status gpcg_n1_adjoint(gpcg_ctx *ctx, const int32_t *outages, int32_t n_out,
                                     int32_t mem, void *stream, const double *P,
                                     const double *b, double *loss, double *dL_dP,
                                     double *dL_db);

/* The N-1 quick screen of the P-theta equation alone (Sec. IV.A: eq. (4)
 * with |V| = 1, the DC power flow).  For each outage l = outages[s]: remove
 * the branch, detect islands (Sec. IV.C), re-dispatch the islands' net
 * injection over the main island's PV generators in proportion to P_gen
 * (Sec. IV.C), and solve
 *   B'_s theta_s = R_s P      (slack angle 0, islanded buses 0)
 * with base-preconditioned CG (Sec. IV.B, eq. (6)); B'_s is B' (weights
 * 1/x) with the outage's four-element change.  Then
 *   flow[s][k] = (theta_i - theta_j) / x_k on branches k = (i, j) in service
 *                between main-island buses, else 0,
 *   max_loading[s] = max_k |flow[s][k]| / rating_k,
 *   n_overload[s]  = the number of branches with |flow[s][k]| / rating_k > 1,
 *   overload[s]    = those branches as a bit mask (as in gpcg_n1_screen).
 * Inputs: P[n_bus] bus injections (NULL: the grid's P_sched), host or device
 * memory as mem says.  Outputs, each optional: theta[n_out][n_bus],
 * flow[n_out][n_branch], iters[n_out] (PCG iterations), status[n_out]
 * (GPCG_SCEN_OK, or GPCG_SCEN_ISLAND_NO_GEN when an island's injection has
 * no main-island generator to go to and the slack takes it), max_loading,
 * n_overload[n_out], overload[n_out][GPCG_MASK_WORDS(n_branch)].
 * The solve runs in the context's precision: GPCG_BATCHED_FP64 to a 1e-12
 * relative residual; GPCG_BATCHED_FP32 and _FP32_F16 with FP32 vectors and
 * factors to 1e-6, then one step of iterative refinement (FP64 residual,
 * FP32 correction); GPCG_PLAIN_FP64 is INVALID_ARG.  mem and
 * stream as in gpcg_n1_screen (device mode returns once the work is
 * enqueued; host mode when the results are written).  It does not need
 * gpcg_base_solve.  Errors: INVALID_ARG, OOM, CUDA. */
GPCG_API gpcg_status gpcg_n1_dc_screen(gpcg_ctx *ctx, const int32_t *outages, int32_t n_out,
                                       int32_t mem, void *stream, const double *P,
                                       double *theta, double *flow, int32_t *iters,
                                       int32_t *status, double *max_loading,
                                       int32_t *n_overload, uint32_t *overload);

/* Batched operators of the hot path, for verification: each applies, for
 * S scenarios at once, one step of the inner solve to S vectors stored
 * row-major per scenario in the matrix's own row order (gpcg_export_matrix
 * gives that order).  which = 0: B' (eq. (4)), 1: B'' (eq. (5)).
 *   op = 0: Y = B_s X, the base-case matrix with the outaged branch's
 *           four-element change (Sec. IV.B) applied on the fly.
 *   op = 1: Y = M^{-1} X with the base-case preconditioner (eq. (6)):
 *           level-scheduled forward and backward substitution.
 * precision: GPCG_BATCHED_FP32 (vectors and factors in FP32),
 * GPCG_BATCHED_FP64, or GPCG_BATCHED_FP32_F16 (scaled FP16 factor).
 * X, Y are [S][rows] FP64 host arrays.  Synchronous. */
GPCG_API gpcg_status gpcg_apply(gpcg_ctx *ctx, int32_t which, int32_t op,
                       const int32_t *outages, int32_t S, int32_t precision,
                       const double *X, double *Y);

/* Copy out the structures built by gpcg_create for matrix `which`
 * (0: B', 1: B'').  Host arrays, each optional:
 *   bus_of_row[rows]      bus index of each matrix row
 *   rowptr[rows+1], col[nnz], val[nnz]        the matrix (CSR, FP64)
 *   lrowptr[rows+1], lcol[nnz_l], lval[nnz_l] the factor L (CSR, lower,
 *                                             diagonal last in each row)
 *   level[rows]           forward level of each row
 * Sizes are in gpcg_info.  Synchronous. */
GPCG_API gpcg_status gpcg_export_matrix(const gpcg_ctx *ctx, int32_t which,
                               int32_t *bus_of_row, int32_t *rowptr,
                               int32_t *col, double *val, int32_t *lrowptr,
                               int32_t *lcol, double *lval, int32_t *level);

/* Device time of the kernels of the context's last gpcg_n1_screen, from
 * CUDA events recorded on that call's stream: ms[0] = islanding kernel,
 * ms[1] = N-1 solve kernel (sum over its launches).  Waits for those events.
 * Returns NOT_READY when no screen has run. */
GPCG_API gpcg_status gpcg_last_timings(gpcg_ctx *ctx, float *ms /*[2]*/);

/* Size of the device array gpcg_n1_screen_noalloc works in (64 MiB). */
#define GPCG_NOALLOC_SCRATCH_BYTES (64u << 20)

/* The N-1 screen of gpcg_n1_screen with device memory (mem = 1), for
 * callers that must not allocate GPU memory while they run: a control loop
 * or service with a fixed memory budget, a process whose GPU memory is
 * already held by another allocator, or code that cannot afford the device
 * synchronisation that cudaMalloc and cudaFree may cause.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *
 * It allocates nothing: all scratch (island data, the solve's per-tile
 * vectors and state, the scenario queue) comes from one static device array
 * of GPCG_NOALLOC_SCRATCH_BYTES that every CUDA context which loads the
 * library holds until it is destroyed or the process exits.  Each call looks
 * up that array's address in the current context (cudaGetSymbolAddress).
 * The caller provides the context (built earlier by gpcg_create and
 * gpcg_base_solve, which do allocate) and every input and output, all in
 * device memory; outputs as in gpcg_n1_screen.  The outage list is checked
 * through a fixed host buffer, which synchronises `stream`: the call cannot
 * be made while `stream` is being captured into a CUDA graph.  The rest is
 * enqueued on `stream`.
 *
 * Scheduling differs from gpcg_n1_screen, results do not: scenarios are
 * taken in the order given (gpcg_n1_screen starts the outages of heavily
 * loaded branches first); the tile width and the tiles per SM are the
 * context's options, else the ones gpcg_n1_screen's autotuner chose last,
 * else 2 and the occupancy maximum; the dense tails are the factors' own.
 *
 * Every call shares the one array of its context, which keeps the previous
 * call's contents (the call resets what must start at zero): calls that
 * overlap on the GPU -- from two streams or threads in the same context --
 * race and give wrong results.  The solve runs as many scenario tiles at
 * once as fit in the array, so large grids run with fewer tiles than
 * gpcg_n1_screen.
 * Errors: INVALID_ARG when the scenarios and one tile of the grid do not
 * fit in the array (the message gives the bytes needed), when an outage is
 * not a branch index, or when the context's precision is
 * GPCG_PLAIN_FP64 (only the batched solve is offered here); NOT_READY
 * before a successful gpcg_base_solve; CUDA. */
GPCG_API gpcg_status gpcg_n1_screen_noalloc(gpcg_ctx *ctx, const int32_t *outages,
                                            int32_t n_out, void *stream, double *theta,
                                            double *vm, double *flow, int32_t *island_label,
                                            int32_t *iters, int32_t *status,
                                            double *max_loading, int32_t *n_overload,
                                            uint32_t *overload);

/* Sizes of a structural plan (gpcg_analyze). */
typedef struct {
  int32_t n_rows, nnz_a, nnz_l, levels, blevels, n_bridges;
} gpcg_plan_info;

/* The host-side structural analysis of gpcg_create alone, without a GPU:
 * the internal bus numbering (a reverse Cuthill-McKee order of the bus
 * graph), and for matrix `which` (0: B', 1: B'') the row order, the factor
 * pattern for `precond` (GPCG_PRECOND_EXACT: the complete symbolic
 * Cholesky pattern under the minimum-degree order; otherwise the lower
 * triangle of the matrix, i.e. IC(0)) and its forward level schedule
 * (Sec. IV.B), plus the branches whose outage splits the grid (Sec. IV.C).
 * Call with NULL arrays to get the sizes in *info, then again with:
 *   bus_order[n_bus]      internal position -> bus
 *   bus_of_row[n_rows]    matrix row -> bus
 *   lrowptr[n_rows+1], lcol[nnz_l]  the factor pattern (CSR, lower, diagonal last)
 *   level[n_rows]         forward level of each row
 *   bridge[n_branch]      1 where the branch is a bridge
 * Errors: INVALID_ARG (as gpcg_create), BASE_ISLANDED. */
GPCG_API gpcg_status gpcg_analyze(const gpcg_grid *grid, int32_t precond, int32_t which,
                                  gpcg_plan_info *info, int32_t *bus_order,
                                  int32_t *bus_of_row, int32_t *lrowptr, int32_t *lcol,
                                  int32_t *level, uint8_t *bridge);

/* Message of the last error on the calling thread ("" if none). */
GPCG_API const char *gpcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GPCG_H_ */
