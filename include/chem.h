/*
 * chem.h -- C ABI of libchem: batched implicit chemistry step on sm_103a.
 *
 * The operation is the chemistry half of the operator-split reacting-flow
 * step of Le & Cambier, "Development of a Flow Solver with Complex Kinetics
 * on the Graphic Processing Units" (arXiv 1110.4903): Eq. 4 splits the time
 * derivative into convection and chemistry; the chemistry half advances,
 * independently in every finite-volume cell, the species densities rho_s and
 * the energy e (Eq. 3, formation energy excluded) over one fluid time step
 * dt at constant volume, with the sources of Sec. 3.2 (Eqs. 23-27) and the
 * implicit system of Eq. 29 solved by Gaussian elimination.  Here Eq. 29 is
 * iterated to the full backward-Euler solution by Newton's method, on
 * substeps dt 2^-level.  Each Newton system is reduced exactly to the N_s
 * species unknowns (the energy unknown follows from the conservation of
 * total energy) and solved by LU with row partial pivoting.
 *
 * Conventions
 *  - Units SI (kg, m, s, mol, K, J), except the Arrhenius factor A, given in
 *    CGS mol-cm-s units for the forward order of its reaction (incl. +M).
 *  - Cell state is structure-of-arrays in device memory: rho_s[s*ld + cell]
 *    (kg/m^3), e[cell] (J/m^3, sensible energy sum_s rho_s (e_s(T) -
 *    e_s(298.15 K))).  ld >= n_cells; the caller owns all state buffers.
 *  - Every function returns CHEM_OK (0) or a negative CHEM_E_* code; no
 *    function aborts the process.  Per-cell outcomes are CHEM_CELL_* codes.
 *  - Launching calls are asynchronous and stream-ordered on the cudaStream_t
 *    passed as `stream` (NULL = legacy default stream); they never
 *    synchronize, except chem_advance_host, which is synchronous.
 *  - A cell whose step fails keeps its input values.
 *  - All pointers are plain addresses; no PyTorch type crosses this ABI.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define CHEM_OK               0
#define CHEM_E_INVALID_ARG   (-1)   /* NULL pointer, bad size, bad option     */
#define CHEM_E_BAD_MECHANISM (-2)   /* mechanism fails validation             */
#define CHEM_E_OOM           (-3)   /* device or host allocation failed       */
#define CHEM_E_OVER_BUDGET   (-4)   /* request larger than the HBM budget     */
#define CHEM_E_CUDA          (-5)   /* a CUDA call failed (see chem_last_error_message) */
#define CHEM_E_TIMEOUT       (-6)   /* a bounded wait ran out                 */
#define CHEM_E_UNSUPPORTED   (-7)   /* size beyond the kernels' limits        */
#define CHEM_E_NOT_FOUND     (-8)   /* unknown ticket                         */

/* ---- per-cell status ----------------------------------------------------- */
#define CHEM_CELL_OK             0
#define CHEM_CELL_NEWTON_FAILED  1  /* substep halving limit reached          */
#define CHEM_CELL_T_FAILED       2  /* T of the input state not in [200, 6000] K */
#define CHEM_CELL_BAD_INPUT      3  /* non-finite value or total density <= 0 */
#define CHEM_CELL_TOO_MANY_STEPS 4  /* substep attempt budget spent           */

/* ---- limits -------------------------------------------------------------- */
#define CHEM_MAX_SPECIES    64
#define CHEM_MAX_REACTIONS  4096

#define CHEM_FP64   0   /* everything in FP64                                  */
#define CHEM_MIXED  1   /* Jacobian and LU in FP32, residual/rates/T in FP64   */

typedef struct chem_handle_s *chem_handle_t;

/* Reaction mechanism (Sec. 3.2; Appendix A gives one such table).  All
 * arrays are host memory, read during chem_create and not kept. */
typedef struct chem_mech_desc {
    int32_t n_species;            /* N_s, 1..CHEM_MAX_SPECIES                  */
    int32_t n_reactions;          /* reversible reactions, 0..CHEM_MAX_REACTIONS */
    int32_t n_elements;           /* 0 disables the element-balance check      */
    const double  *molar_mass;    /* [N_s] kg/mol, > 0                         */
    const int32_t *elem_comp;     /* [N_s*n_elements] atoms, may be NULL if n_elements == 0 */
    const double  *nasa7;         /* [N_s][2][7] NASA-7 a1..a7, low then high range */
    const double  *t_mid;         /* [N_s] range switch, K (T <= t_mid: low)   */
    const double  *arr_A;         /* [R] Arrhenius factor, CGS, >= 0 (Eq. 23)  */
    const double  *arr_beta;      /* [R] temperature exponent                  */
    const double  *arr_Ea;        /* [R] activation energy, J/mol              */
    const int32_t *reac_sp;       /* [R*3] reactant species, -1 = unused slot  */
    const int32_t *reac_nu;       /* [R*3] stoichiometric coefficients 1..3    */
    const int32_t *prod_sp;       /* [R*3] product species, -1 = unused slot   */
    const int32_t *prod_nu;       /* [R*3]                                     */
    const int32_t *third_body;    /* [R] 1 = "+M" reaction (Eq. 25 factor)     */
    const double  *tb_eff;        /* [R*N_s] efficiencies alpha_rs; NULL = all 1 */
} chem_mech_desc;

typedef struct chem_options {
    int32_t precision;        /* CHEM_FP64 or CHEM_MIXED                        */
    double  rtol;             /* Newton: max_i |dx_i|/(rtol|x_i| + atol_i) <= 1 */
    double  atol_rel;         /* atol = atol_rel * rho (species), atol_rel * E_scale (energy) */
    int32_t max_newton;       /* Newton iterations per substep attempt, 1..1000 */
    int32_t max_halvings;     /* deepest substep level, 0..40                   */
    int32_t max_attempts;     /* substep attempts per cell, 1..1e6              */
    int32_t point_implicit;   /* 1: one linearised step per substep (Eq. 29 as printed) */
    int32_t div_check;        /* 1: abandon a substep whose Newton norm stops falling */
    int32_t lanes_per_cell;   /* 0 = chosen by the library; else 2, 4, 8, 16 or 32 */
    int32_t autotune;         /* 1: time the lane choices once and keep the best */
    int64_t hbm_budget_bytes; /* not used by the step calls (validated: >= 0); the request
                                 server's budget is chem_server_options.hbm_budget_bytes */
    int32_t max_newton_mixed; /* Newton iterations per attempt on the CHEM_MIXED path, whose
                                 FP32 LU makes convergence linear; 1..1000 */
    double  conv_kappa;       /* > 0: also converged when the contraction theta = norm_k/norm_k-1 < 1
                                 bounds the remaining error, theta/(1-theta) norm_k <= conv_kappa
                                 (Hairer & Wanner's stopping estimate); 0 = off; 0..1.  CHEM_FP64 */
    double  conv_kappa_mixed; /* the same for the CHEM_MIXED path */
} chem_options;

/* Fills *o with the defaults: FP64, rtol 1e-10, atol_rel 1e-12,
 * max_newton 12, max_halvings 20, max_attempts 1000, point_implicit 0,
 * div_check 1, lanes_per_cell 0, autotune 0, hbm_budget_bytes 0,
 * max_newton_mixed 12, conv_kappa 0 (the FP64 path stops on the norm test alone: an
 * accepted update well above the tolerance carries its rounding into the result),
 * conv_kappa_mixed 0.01. */
int chem_default_options(chem_options *o);

/* Validates the mechanism (index ranges, 1..3 species per side with
 * coefficients 1..3, element balance when n_elements > 0, cp/R > 1 on
 * [200, 6000] K so temperature recovery is monotone), builds the derived
 * device tables and returns a handle.  opts may be NULL (defaults).  Uses the
 * current CUDA device.  Errors: INVALID_ARG, BAD_MECHANISM, UNSUPPORTED, OOM,
 * CUDA. */
int chem_create(const chem_mech_desc *mech, const chem_options *opts, chem_handle_t *out);

/* Waits for the handle's own work, then frees everything the handle owns. */
int chem_destroy(chem_handle_t h);

/* Advances n_cells cells over dt >= 0 in place (Eq. 4, chemistry half):
 * rho_s [N_s*n_cells] and e [n_cells], device, ld = n_cells.  n_cells == 0 is
 * a no-op.  Asynchronous on `stream`. */
int chem_advance(chem_handle_t h, int64_t n_cells, double *rho_s, double *e, double dt,
                 void *stream);

typedef struct chem_advance_args {
    int64_t  n_cells;
    int64_t  ld;              /* leading dimension of rho_s, >= n_cells (0 = n_cells) */
    double  *rho_s;           /* device, in/out                                */
    double  *e;               /* device, in/out                                */
    double   dt;              /* s, >= 0                                       */
    const double *T_in;       /* device [n_cells] temperature guesses, or NULL (1500 K) */
    double  *T_out;           /* device [n_cells] temperature of the result, or NULL */
    int32_t *status;          /* device [n_cells] CHEM_CELL_* codes, or NULL   */
    int32_t *newton_iters;    /* device [n_cells] Newton iterations, all attempts, or NULL */
    int32_t *substeps;        /* device [n_cells] accepted substeps, or NULL   */
    int32_t *failures;        /* device [n_cells] failed substep attempts, or NULL */
    void    *stream;          /* cudaStream_t                                  */
    int32_t  precision;       /* -1 = the handle's; else CHEM_FP64 / CHEM_MIXED */
    int32_t  lanes_per_cell;  /* 0 = the handle's choice                        */
    uint32_t *schedule;       /* diagnostics, device [n_cells*CHEM_SCHEDULE_WORDS], or NULL:
                                 cell c's substep attempts, bit a (word a/32, bit a%32 of
                                 schedule[c*CHEM_SCHEDULE_WORDS ..]) set when attempt a was
                                 accepted.  While recording, the attempt budget is at most
                                 32*CHEM_SCHEDULE_WORDS (cells beyond it end with
                                 CHEM_CELL_TOO_MANY_STEPS).  With the counts in substeps and
                                 failures it fixes the sequence of substep sizes the cell
                                 took, so a reference integrator can follow the same one. */
    double  *substep_states;  /* diagnostics, device [n_cells*CHEM_SUBSTEP_STATES*(N_s+1)], or
                                 NULL: the state (rho_1..rho_Ns, e) after each of cell c's first
                                 CHEM_SUBSTEP_STATES accepted substeps, at
                                 [(c*CHEM_SUBSTEP_STATES + j)*(N_s+1) ..]; rows past the cell's
                                 accepted substeps are left untouched.  Where a substep's
                                 backward-Euler system has several roots, it tells a reference
                                 integrator which one the cell took. */
} chem_advance_args;

/* Words of the per-cell substep-schedule record (256 attempts). */
#define CHEM_SCHEDULE_WORDS 8
/* Accepted substeps whose states chem_advance_args.substep_states records. */
#define CHEM_SUBSTEP_STATES 32

/* chem_advance with strides, temperature guesses and per-cell outputs.
 * Each launch takes one of the handle's 4096 work counters in turn (zeroed
 * in-stream before it): at most 4096 launches of one handle may be in flight
 * at once, across all the streams it is used on. */
int chem_advance_ex(chem_handle_t h, const chem_advance_args *a);

/* Domain-segmented execution (Sec. 5.2): the same step as chem_advance_ex,
 * issued as consecutive launches over segments of at most segment_cells
 * cells (the paper called its kernel on segments of the grid to cap the
 * memory of per-cell Jacobians).  Results are those of one launch, bit for
 * bit; only the launch granularity changes.  segment_cells <= 0 means one
 * segment. */
int chem_advance_segmented(chem_handle_t h, const chem_advance_args *a, int64_t segment_cells);

/* Same step on HOST buffers (rho_s [N_s*ld], e, optional T_out/status):
 * copies to library-owned device buffers, advances, copies back and
 * synchronizes.  Pinned host memory makes the copies faster. */
int chem_advance_host(chem_handle_t h, int64_t n_cells, int64_t ld, double *rho_s, double *e,
                      double dt, double *T_out, int32_t *status);

/* No counterpart in the paper: an allocation-free chem_advance_host for
 * callers that must not allocate device memory while running (a host flow
 * solver inside a framework that owns the device through its own memory
 * pool, or a real-time loop that forbids cudaMalloc/cudaFree after start-up).
 * Same arguments as chem_advance_host, and the same results for the same
 * launch shape, but the device staging of
 * rho_s, e, T_out, status and the kernel's work counter lives in one fixed
 * 16 MiB file-scope device array (chem_static_scratch_bytes reports the
 * size) that every GPU loading the library keeps until exit; nothing is
 * allocated per call.  A request needing more than the array -- about
 * 16 MiB / (8 N_s + 20) cells -- returns CHEM_E_UNSUPPORTED with the cell
 * limit in chem_last_error_message; split it.  The first call on a device
 * looks up the array's device address (once per device, the handle's device
 * must be current).  All calls share the array and it keeps the last call's
 * contents; calls are serialised per device inside one process, and calls
 * that overlapped on the GPU would race.  Synchronous. */
/* (It never autotunes -- the tuner's sample buffers are allocations: it
 * launches the lane width the handle holds for its precision.  With
 * chem_options.autotune set, call chem_autotune once beforehand to get the
 * tuned shape.) */
int chem_advance_host_static(chem_handle_t h, int64_t n_cells, int64_t ld, double *rho_s,
                             double *e, double dt, double *T_out, int32_t *status);

/* Size in bytes of chem_advance_host_static's static device array. */
int chem_static_scratch_bytes(int64_t *bytes);

/* Initial states from temperature T [n], pressure P [n] (Pa) and mass
 * fractions Y [N_s*ld] (all device): rho = P / (R T sum_s Y_s/M_s) (Dalton's
 * law, Eq. 5), rho_s = rho Y_s, e from Eq. 3.  Asynchronous on `stream`. */
int chem_state_from_tpy(chem_handle_t h, int64_t n_cells, int64_t ld, const double *T,
                        const double *P, const double *Y, double *rho_s, double *e,
                        void *stream);

/* Temperature of given states (the recovery every step starts with), on
 * device buffers; T_guess may be NULL.  Asynchronous. */
int chem_temperature(chem_handle_t h, int64_t n_cells, int64_t ld, const double *rho_s,
                     const double *e, const double *T_guess, double *T_out, void *stream);

/* Autotuner: times every launch shape the shared memory allows -- lanes per
 * cell (cells per warp = 32/lanes) and warps per block -- on a strided
 * sample of the given cells (device buffers, same layout as
 * chem_advance_ex; the cells themselves are not modified: the sample is
 * copied), keeps the fastest for `precision` on this handle and returns it.
 * The sample starts at eight waves of the shape that holds the most cells
 * (at least 16,384 cells) and grows, up to all of the cells, until one step
 * of it in the default shape takes 100 ms: where work per cell varies
 * widely, a short sample would time its hardest cells' latency instead of
 * the throughput.
 * Synchronous.  With chem_options.autotune = 1 the first chem_advance_ex of
 * each precision runs it on its own cells first. */
int chem_autotune(chem_handle_t h, int32_t precision, int64_t n_cells, int64_t ld,
                  const double *rho_s, const double *e, double dt, const double *T_in,
                  void *stream, int32_t *lanes_out, int32_t *wpb_out);

/* A captured CUDA graph of one chemistry step (work-counter reset + the
 * persistent step kernel) with fixed arguments, for time loops that step the
 * same device buffers again and again: the work stealing happens inside the
 * kernel, the graph removes the per-step launch work on the host.  The graph
 * owns its work counter.  chem_graph_launch is asynchronous on `stream`;
 * launches of one graph must not overlap on the device. */
typedef struct chem_graph_s *chem_graph_t;
int chem_graph_create(chem_handle_t h, const chem_advance_args *a, chem_graph_t *out);
int chem_graph_launch(chem_graph_t g, void *stream);
int chem_graph_destroy(chem_graph_t g);

/* Formation energies e_f,s = e_s(298.15 K) per unit mass (J/kg) the handle
 * uses (Eq. 3 leaves them out of e; U = e + sum_s rho_s e_f,s is what a step
 * conserves).  e_f is a host array of N_s doubles. */
int chem_formation_energies(chem_handle_t h, double *e_f);

/* Lanes per cell the handle uses for `precision` (after autotuning, if on). */
int chem_get_lanes_per_cell(chem_handle_t h, int32_t precision, int32_t *lanes);

/* Kernel launches this handle has issued since creation (all entry points). */
int chem_launch_count(chem_handle_t h, int64_t *count);

/* ---- serving: continuous batching of requests from many simulations ----
 * A server owns a scheduler thread, a device pool of hbm_budget_bytes and,
 * per (handle, precision) its requests use, a lane: a ring of request
 * descriptors in host memory mapped into the device's address space and
 * persistent instances of the step kernel that claim the ring's cells.
 * chem_submit queues a request (its own mechanism handle, cell count, dt and
 * state); the scheduler admits the head of the FIFO queue when fewer than
 * max_inflight requests are admitted and unfinished and its bytes
 * (n_cells * (8 N_s + 20) + 1024) fit in the remaining budget, and publishes
 * its cells to its lane in chunks of at most 1024, the request with the
 * fewest cells left first (one waiting 50 ms without a chunk goes first),
 * keeping about a quarter of the lane's slots worth of cells published ahead
 * of the kernels.  The free slots of a warp of a running kernel claim
 * consecutive published cells together, so a request admitted while others
 * run is stepped inside the same grid, cells of several requests in flight
 * together on every SM (continuous batching on the device).  Lanes of
 * different mechanisms share the GPU: each lane with work gets an equal share
 * of its full grid.  A server holds at most 16 lanes: a request that would
 * need a 17th finishes FAILED with error CHEM_E_UNSUPPORTED.  Device-resident states (host = 0) are stepped in
 * place and count against the budget while in flight; host states (host = 1)
 * are copied through the pool and back.  A request is computed exactly as by
 * chem_advance_ex with the same handle, whatever else is in flight.
 * Requests larger than the whole budget are refused (CHEM_E_OVER_BUDGET).
 * Handles must outlive their requests; the server keeps a lane per handle
 * used until it is destroyed. */
#define CHEM_REQ_QUEUED    0
#define CHEM_REQ_RUNNING   1
#define CHEM_REQ_DONE      2
#define CHEM_REQ_FAILED    3
#define CHEM_REQ_CANCELLED 4

typedef struct chem_server_s *chem_server_t;

typedef struct chem_server_options {
    int64_t hbm_budget_bytes;   /* device pool and in-flight budget; 0 = a quarter of free memory */
    int32_t max_inflight;       /* requests admitted and unfinished at once, 1..1023; default 64 */
    int32_t queue_capacity;     /* queued requests before chem_submit refuses; default 100000 */
} chem_server_options;

typedef struct chem_request {
    chem_handle_t mech;         /* mechanism and options of this request */
    int64_t  n_cells;
    int64_t  ld;                /* 0 = n_cells */
    double  *rho_s;             /* state, device (host = 0) or host (host = 1), in/out */
    double  *e;
    int32_t  host;
    int32_t  precision;         /* -1 = the handle's */
    double   dt;
    double  *T_out;             /* optional, same memory kind as the state */
    int32_t *status;            /* optional, same memory kind as the state */
    void    *ready_event;       /* optional cudaEvent_t: the request's stream waits for it
                                   before touching device buffers (e.g. recorded after the
                                   writes that produced the state); the event must stay
                                   valid until the request has started */
} chem_request;

typedef struct chem_result {
    int32_t state;              /* CHEM_REQ_* */
    int32_t error;              /* CHEM_E_* when FAILED */
    double  t_submit, t_start, t_done;   /* seconds on the server's monotonic clock */
    uint64_t dev_first_ns;      /* device clock (globaltimer, ns) when the first of the request's
                                   cells was claimed by a slot of a server kernel, */
    uint64_t dev_last_ns;       /* and when its last cell finished (DONE requests; else 0) */
} chem_result;

typedef struct chem_server_stats_t {
    int64_t queued;             /* submitted, not yet admitted */
    int64_t running;            /* admitted, not finished */
    int64_t completed, failed;
    int64_t bytes_in_use, budget_bytes;
    int64_t launches;           /* server kernel instances launched so far */
    int64_t kernel_instances;   /* server kernel instances on the device now */
    int64_t queue_errors;       /* nonzero if a kernel failed to find a claimed cell's request */
} chem_server_stats_t;

int chem_server_default_options(chem_server_options *o);
int chem_server_create(const chem_server_options *o, chem_server_t *out);
/* Cancels queued requests, waits for running ones, frees the server. */
int chem_server_destroy(chem_server_t s);
int chem_submit(chem_server_t s, const chem_request *r, uint64_t *ticket);
/* Non-blocking state of a request. */
int chem_poll(chem_server_t s, uint64_t ticket, chem_result *out);
/* Waits until the request finishes or timeout_us passes (< 0: no limit);
 * CHEM_E_TIMEOUT with the current state in *out when it runs out. */
int chem_wait(chem_server_t s, uint64_t ticket, int64_t timeout_us, chem_result *out);
/* Cancels a request that is still queued (its state is never touched). */
int chem_cancel(chem_server_t s, uint64_t ticket);
/* Forgets a finished request's record. */
int chem_release(chem_server_t s, uint64_t ticket);
int chem_server_stats(chem_server_t s, chem_server_stats_t *out);

/* ---- batched dense solves: the kinetics-only experiment of Sec. 5.2 ----
 * Solves n_sys independent systems A_k x_k = b_k of size n (1..CHEM_LU_MAX_N)
 * in place by Gaussian elimination with row partial pivoting in FP64: the
 * pivot of column j is the first row i >= j of largest |a_ij| (a NaN
 * diagonal stays the pivot; a NaN below it is never taken).  On return A
 * holds L (unit, below the diagonal) and U, b holds x, pivots[k*n + j]
 * (optional) the row swapped into row j, info[k] (optional) 0 or 1 + the
 * first column with a zero or non-finite pivot (elimination continues past
 * it; that system's A and x are then meaningless).  Arithmetic, layout and
 * kernel by method:
 *   CHEM_LU_GLOBAL      A[(i*n + j)*n_sys + k], b[i*n_sys + k] (interleaved);
 *                       the matrices stay in HBM (the paper's global-memory
 *                       approach): a thread per system when the systems
 *                       fill the GPU, else a block of warps per 32 systems
 *                       sharing each step's rows.  Every step explicitly
 *                       rounded in the scalar order (multiplier a_ij / a_jj,
 *                       update a_ik - l a_jk without contraction): factors,
 *                       pivots and x equal a scalar elimination with
 *                       row-by-row substitutions bit for bit.
 *   CHEM_LU_GLOBAL_FMA  same layout and kernels, contracted arithmetic:
 *                       multipliers a_ij times one reciprocal of the pivot,
 *                       updates and substitutions as fused multiply-adds;
 *                       equal to the scalar elimination to rounding.
 *   CHEM_LU_ONCHIP      A[(k*n + i)*n + j], b[k*n + i] (contiguous); one warp
 *                       per system, the matrix in shared memory
 *                       (CHEM_E_UNSUPPORTED when n*(n+1) doubles do not
 *                       fit); factors and pivots bit for bit as
 *                       CHEM_LU_GLOBAL, x to rounding (the back
 *                       substitution runs by columns across the warp).
 * Device pointers; asynchronous on `stream`; CHEM_E_INVALID_ARG for an
 * unknown method, n out of range, n_sys < 0 or a null A or b. */
#define CHEM_LU_GLOBAL     0
#define CHEM_LU_ONCHIP     1
#define CHEM_LU_GLOBAL_FMA 2
#define CHEM_LU_MAX_N      256
int chem_batched_solve(int32_t method, int32_t n, int64_t n_sys, double *A, double *b,
                       int32_t *pivots, int32_t *info, void *stream);

/* Diagnostics: evaluates the step kernel's own exp (table-driven, after
 * Tang) and reciprocal (rcp.approx + two Newton steps) at n device points x,
 * next to CUDA's exp and IEEE division, for tests of their error.
 * Synchronous. */
int chem_selftest_math(int64_t n, const double *x, double *y_exp, double *y_exp_ref,
                       double *y_rcp, double *y_rcp_ref, void *stream);

/* Diagnostics: the step kernel's logarithm of the temperature (table-driven,
 * after Tang, ACM TOMS 16(4), 1990) at n device points x (finite, >= 2: its
 * domain; the kernels take it of T in [200, 6000] K), next to CUDA's log.
 * Synchronous. */
int chem_selftest_log(int64_t n, const double *x, double *y_log, double *y_log_ref, void *stream);

/* Diagnostics for the equilibrium constants' exponent arithmetic (Eq. 24 as
 * the kernels form it): at n device points, exp(x[i]) split into a mantissa
 * y_mant[i] in [0.99, 2.01] and a power of two y_pow[i] (|x| >= 2^22 and
 * infinities saturate the power at +-2^24 with mantissa 1; NaN gives a NaN
 * mantissa), and y_scaled[i] = v[i] 2^k[i] on the exponent bits (zero,
 * subnormal, infinite and NaN v unchanged; results below the normal range
 * are signed zeros, above it infinities).  Synchronous. */
int chem_selftest_scaled_exp(int64_t n, const double *x, double *y_mant, int32_t *y_pow,
                             const double *v, const int32_t *k, double *y_scaled, void *stream);

/* Human-readable text for a CHEM_E_* code (static storage). */
const char *chem_strerror(int code);

/* Detail of the last error raised on the calling thread (static per thread). */
const char *chem_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H */
