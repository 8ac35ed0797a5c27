/*
 * pdlp.h -- C ABI of the GB300 (sm_103a) implementation of PDLP, the restarted
 * primal-dual hybrid gradient method for linear programming of
 * "PDLP: A Practical First-Order Method for Large-Scale Linear Programming".
 *
 * Problem (Sec. 2, Eq. (1)):
 *     minimize c'x   subject to   lc <= A x <= uc,   lv <= x <= uv,
 * with A in R^{m x n} given in CSR form, bounds in R u {-inf, +inf} (IEEE
 * +-INFINITY marks a missing bound).  The dual multipliers y (one per row) follow
 * the sign convention of Eq. (1): y_i >= 0 on a row with only a finite lower bound,
 * y_i <= 0 with only a finite upper bound, y_i = 0 on a free row.
 *
 * Conventions for every entry point:
 *   - All arrays are owned by the caller; the library neither frees nor retains
 *     them after the call returns.  The library allocates its own device work
 *     memory (cudaMalloc) for the duration of a call and frees it before returning.
 *   - params->inputs_on_device selects where the input AND output arrays live:
 *     0 = host memory (pageable or pinned), 1 = device memory of the current CUDA
 *     device.  Device arrays must not be written by other work while the call runs.
 *   - params->cuda_stream (a cudaStream_t, may be NULL) is the stream all device work
 *     is ordered on; the call blocks until its results are complete.
 *   - Return value: 0 on success (for pdlp_solve: status OPTIMAL), a positive status
 *     for a finished solve that did not reach the tolerance, a negative code for an
 *     error, in which case outputs are not written and pdlp_last_error() describes
 *     the failure.  No C++ exception crosses this interface.
 *   - Every entry point is thread-compatible: concurrent calls need distinct
 *     streams and output buffers; the only global state is the thread-local error
 *     string.
 */
#ifndef PDLP_H_
#define PDLP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status and error codes ------------------------------------------------ */
#define PDLP_OPTIMAL 0            /* termination criterion met                    */
#define PDLP_ITERATION_LIMIT 1    /* params->max_iters accepted iterations done   */
#define PDLP_TIME_LIMIT 2         /* params->time_limit_s exceeded                */
#define PDLP_PRIMAL_INFEASIBLE 3  /* App. C certificate found: y returns it        */
#define PDLP_DUAL_INFEASIBLE 4    /* App. C certificate found: x returns the ray    */
#define PDLP_NUMERICAL_ERROR 5    /* non-finite step or step-retry cap reached    */
#define PDLP_INVALID_ARGUMENT (-1)
#define PDLP_OUT_OF_MEMORY (-2)
#define PDLP_CUDA_ERROR (-3)

/* precision of the bulk data (matrix values, iterates, SpMV accumulation) */
#define PDLP_FP64 0
#define PDLP_FP32_BULK 1

/* Constraint matrix in CSR form (Sec. 5 "Multithreading": A x and A'y are the two
 * sparse products of every iteration; this library builds the transpose itself).
 *   row_ptr[m+1]: row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz.
 *   col_idx[nnz]: strictly increasing within a row, 0 <= col < n.
 *   val[nnz]:     finite.                                                        */
typedef struct {
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} pdlp_csr;

/* Algorithm parameters.  pdlp_params_default() fills the paper's defaults. */
typedef struct {
  double eps_rel_kkt;      /* termination_mode 0: stop when the relative KKT error
                              (max of relative primal residual, relative dual
                              residual, relative gap; all on the unscaled LP) is
                              <= this.  Default 1e-8.                               */
  int termination_mode;    /* 0: relative KKT; 1: Sec. 7 / Eq. (9): l_inf primal and
                              dual residual <= eps_abs_feas and the relative gap of
                              Eq. (8) <= eps_rel_gap; 2: the same on the paper's
                              rescaled instances (Sec. 6: right-hand sides and costs
                              scaled to magnitude 1), read on the LP as given (Eq.
                              (10)): row i's violation <= eps_abs_feas q_i with q_i the
                              largest magnitude of its finite nonzero bounds (1 if
                              none), column j's dual residual <= eps_abs_feas |c_j|
                              (eps_abs_feas if c_j = 0).  Polishing phases use the
                              primal / dual half of the criteria in force.          */
  double eps_abs_feas;     /* default 1e-8                                          */
  double eps_rel_gap;      /* default 1e-2                                          */
  int64_t max_iters;       /* accepted PDHG iterations; default 1e9                  */
  double time_limit_s;     /* wall-clock limit of the solve; default +inf            */
  int ruiz_iters;          /* Sec. 3 "Diagonal Preconditioning": default 10          */
  double pc_alpha;         /* Pock-Chambolle alpha in (0,2); <= 0 disables; default 1 */
  int check_period;        /* restart/termination evaluation period (Sec. 3); 64    */
  double beta_suff, beta_nec, beta_art; /* restart criteria (i)-(iii): 0.1, 0.9, 0.5 */
  double theta;            /* primal weight smoothing (Algorithm 3): 0.5             */
  double eps_zero;         /* Algorithm 3's tolerance: 1e-10                         */
  int max_step_retries;    /* cap of Algorithm 2's retry loop: 60                    */
  int precision;           /* PDLP_FP64 (default) or PDLP_FP32_BULK                  */
  int inputs_on_device;    /* 0 host arrays (default), 1 device arrays              */
  void* cuda_stream;       /* cudaStream_t or NULL                                  */
  int64_t trace_iters;     /* > 0: record the first trace_iters accepted iterations  */
  double* trace_out;       /* host array [trace_iters * (PDLP_TRACE_HEADER + n + m)] */
  int profile;             /* 1: time the hot kernels with CUDA events (stats)       */
  int verbose;             /* 1: one line per check to stderr                        */
  int feasibility_polishing; /* 1: Algorithm 4 (Sec. 5).  Normal PDLP pauses after
                              k = 100, 200, 400, ... iterations when the relative gap
                              (Eq. (8)) of its average iterate is < eps_rel_gap; PDLP
                              then runs on the primal feasibility problem (objective
                              0) from (x^k, 0) and, if that reaches the primal half
                              of the termination criteria, on the dual feasibility
                              problem (finite bounds set to 0) from (0, y^k), each
                              for at most k/8 iterations with normal PDLP's current
                              primal weight and step; the pair is returned when it
                              meets the termination criteria, else normal PDLP
                              resumes.  Default 0.                                  */
  int64_t polish_log_cap;  /* rows available in polish_log                          */
  double* polish_log;      /* host [polish_log_cap * PDLP_POLISH_LOG_COLS] or NULL:
                              one row per pause (see PDLP_POLISH_LOG_COLS)          */
  int detect_infeasibility; /* 1 (default): at every check of normal PDLP, after the
                              termination test, test three candidate directions --
                              the difference of the last two iterates, the current
                              iterate, the average since the last restart -- as
                              certificates of App. C on the unscaled LP: y projected
                              onto Y with r = proj_R(-A'y): primal infeasible if
                              lc'y+ - uc'y- + lv'r+ - uv'r- > 0 and ||A'y + r||_inf
                              <= eps_infeas times it (status 3, y = the certificate,
                              x = current); x projected onto the recession cone of
                              the box with s = proj_Sbar(-Ax): dual infeasible if
                              c'x < 0 and ||Ax + s||_inf <= eps_infeas |c'x| (status
                              4, x = the ray, not clipped to the bounds, y = current).
                              Costs four sparse products per check.                */
  double eps_infeas;       /* App. C's threshold: 1e-9                              */
  int reduced_costs;       /* reduced costs r of the dual residual and objective in
                              every optimality measure: 0 (default) r = proj_R(c -
                              A'y) (Sec. 2); 1 App. A's choice, r_i = (c - A'y)_i
                              when it is positive and x_i - lv_i <= |x_i|, or
                              negative and uv_i - x_i <= |x_i|, else 0 (robust to
                              huge bounds; changes the measures, not the iterates) */
  double fixed_step;       /* > 0: every step attempt uses eta = fixed_step and is
                              accepted (plain PDHG of Eq. (3) with constant steps, the
                              Chambolle-Pock iteration Algorithm 2 adapts); 0
                              (default): Algorithm 2.  Must be finite and >= 0.   */
  double fixed_omega;      /* > 0: the primal weight is fixed_omega throughout (no
                              InitializePrimalWeight, no Algorithm 3 update at
                              restarts); 0 (default): Sec. 3's rules.  Finite, >= 0. */
} pdlp_params;

/* Row of params->polish_log for one pause of Algorithm 4:
 *   [0] k (normal iterations done), [1] relative gap (Eq. (8)) of the average
 *   iterate, [2] primal-phase iterations, [3] 1 if the primal phase reached primal
 *   feasibility, [4] dual-phase iterations, [5] 1 if the dual phase reached dual
 *   feasibility, [6] 1 if the pair was returned.                                   */
#define PDLP_POLISH_LOG_COLS 7

/* Trace record of one accepted iteration k (scaled space, i.e. of the
 * preconditioned LP): PDLP_TRACE_HEADER doubles, then x[n], then y[m].
 * header: [0] k, [1] accepted eta, [2] omega used, [3] eta_hat after,
 *         [4] attempts in this iteration, [5] restart kind (0 none, 1 (i),
 *         2 (ii), 3 (iii)), [6] mu(current), [7] mu(average) (NaN when not
 *         evaluated at this iteration).                                           */
#define PDLP_TRACE_HEADER 8

typedef struct {
  int status;
  int64_t iterations;      /* accepted PDHG iterations                             */
  int64_t attempts;        /* step attempts (accepted + rejected)                  */
  int64_t rejected_steps;
  int64_t restarts[3];     /* restarts by criterion (i), (ii), (iii)               */
  double kkt_passes;       /* (number of A x products + number of A'y products)/2  */
  double rel_kkt, rel_primal, rel_dual, rel_gap;
  double primal_res_l2, dual_res_l2, primal_res_inf, dual_res_inf;
  double pobj, dobj, paper_gap;
  double omega, eta_hat;
  double seconds_setup, seconds_solve, seconds_total;
  /* profile == 1: device time of the two fused SpMV kernels and their launches */
  double ms_spmv_a, ms_spmv_at, ms_primal, ms_checks;
  int64_t launches_spmv_a, launches_spmv_at;
  int64_t kernel_launches; /* kernels of this library launched by the call         */
  double bytes_spmv_a, bytes_spmv_at; /* algorithmic bytes per launch              */
  int64_t gap_evals;       /* normalized duality gap evaluations                   */
  int64_t gap_fallbacks;   /* ... that needed the FP64 bracket scan                */
  int64_t gap_failures;    /* ... left unresolved (mu treated as NaN: no restart by
                              criteria (i)/(ii) at that check; pdlp_last_error()
                              describes the last one)                              */
  int64_t polish_pauses;   /* Algorithm 4: pauses of normal PDLP                     */
  int64_t polish_primal_iters, polish_dual_iters; /* iterations of all phases      */
  int64_t polish_accepted_k; /* k of the pause whose pair was returned, else 0     */
  int64_t device_bytes;    /* peak device memory the call held (stream-ordered
                              allocations; setup temporaries -- the staged input, the
                              transpose, the preconditioner's and renumbering scratch --
                              are freed once the layouts exist) */
  /* wall-clock milliseconds of the periodic checks (device work and the host
     synchronisations they need): normalized duality gaps, KKT measures, infeasibility
     tests, and the number of evaluation points (checks, (iii) iterations, restarts) */
  double ms_gap, ms_kkt, ms_infeas;
  int64_t evaluations;
  /* l_inf residuals of the returned point with row i divided by q_i and column j by
     w_j of Sec. 7's Eq. (10) (see termination_mode 2) */
  double primal_res_rel_inf, dual_res_rel_inf;
  /* pdlp_solve_batch_persistent: device time of the whole persistent launch (CUDA
     events; the same for every LP of the call), and the SM that solved this LP */
  double batch_launch_s;
  int64_t batch_sm;
} pdlp_stats;

/* Fills *p with the defaults listed above. */
void pdlp_params_default(pdlp_params* p);

/* Solves the LP with PDLP (Algorithm 1 after the preconditioning of Sec. 3, the
 * adaptive step of Algorithm 2, the restart scheme of Sec. 3 and the primal weight
 * update of Algorithm 3).
 *   m >= 0 rows, n >= 1 columns; A->nnz >= 0.
 *   c[n], lc[m], uc[m], lv[n], uv[n]: lc <= uc, lv <= uv, lv < +inf, uv > -inf,
 *       no NaN.  c finite.
 *   x_out[n], y_out[m]: the returned point (unscaled).  Written for status >= 0.
 *   stats: may be NULL.
 * Errors: PDLP_INVALID_ARGUMENT for malformed input (the message names the first
 * offending index), PDLP_OUT_OF_MEMORY, PDLP_CUDA_ERROR. */
int pdlp_solve(int64_t m, int64_t n, const pdlp_csr* A, const double* c, const double* lc,
               const double* uc, const double* lv, const double* uv, const pdlp_params* p,
               double* x_out, double* y_out, pdlp_stats* stats);

/* The diagonal preconditioning alone (Sec. 3 "Diagonal Preconditioning":
 * p->ruiz_iters Ruiz passes, then Pock-Chambolle with p->pc_alpha), on the GPU.
 * Writes d1_out[m], d2_out[n] (A~ = D1 A D2) and, if scaled_val_out is not NULL,
 * the values of A~ in the order of A->val.  Same memory conventions as pdlp_solve. */
int pdlp_precondition(int64_t m, int64_t n, const pdlp_csr* A, const pdlp_params* p,
                      double* d1_out, double* d2_out, double* scaled_val_out);

/* The normalized duality gap mu(z, z_ref) = rho_r(z) with r = ||z - z_ref||_omega
 * (Sec. 3 "Adaptive restarts") of the point z = (x, y) for the LP exactly as given
 * (no preconditioning), computed by the same GPU kernels the solver uses.
 * x, x_ref: [n]; y, y_ref: [m]; x must lie in [lv, uv] and y in the sign set Y.
 * Writes *mu_out (host).  Same memory conventions as pdlp_solve for the arrays. */
int pdlp_normalized_gap(int64_t m, int64_t n, const pdlp_csr* A, const double* c,
                        const double* lc, const double* uc, const double* lv,
                        const double* uv, const double* x, const double* y,
                        const double* x_ref, const double* y_ref, double omega,
                        const pdlp_params* p, double* mu_out);

/* Optimality measures of a point (x, y) for the LP as given: residuals, objectives
 * and gaps with the reduced costs r = proj_R(c - A'y) (Sec. 2), as used by the
 * termination test.  out[11] (host) receives: rel_kkt, rel_primal, rel_dual,
 * rel_gap, primal_res_l2, dual_res_l2, primal_res_inf, dual_res_inf, pobj, dobj,
 * paper_gap (Eq. (8)). */
int pdlp_kkt(int64_t m, int64_t n, const pdlp_csr* A, const double* c, const double* lc,
             const double* uc, const double* lv, const double* uv, const double* x,
             const double* y, const pdlp_params* p, double* out);

/* The measures of pdlp_kkt for a point whose products A x and A'y the caller already
 * holds, computed WITHOUT ALLOCATING ANY MEMORY.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device memory
 * mid-run -- for instance an application whose memory manager owns the whole device
 * (a framework pool or a preallocated arena) or a loop with a fixed latency budget
 * where a cudaMalloc/cudaFree could block -- but still want the optimality
 * measures of an iterate they computed themselves.
 *   All arrays are DEVICE arrays of the current device: c, lv, uv, x, aty [n];
 *   lc, uc, y, ax [m] (ax = A x, aty = A'y of the LP as given).  out[11] is host
 *   memory and receives the values in pdlp_kkt's order.  cuda_stream may be NULL.
 *   m in [0, 2^31-1], n in [1, 2^31-1]; other sizes return PDLP_INVALID_ARGUMENT.
 * Scratch: the per-CTA partial sums (at most 1024 CTAs), the arrival counter and the
 * result live in one fixed file-scope device array of about 74 KB, which every GPU
 * that loads the library keeps until the process exits; its size does not depend on
 * m or n.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and caches it per device index; make that first call before
 * any stream capture.  The cached address belongs to the context that was current at
 * that first call, normally the device's primary context (the runtime API's); callers
 * that switch to other contexts of the same device must not use this entry point.  Every call clears the counter and overwrites the rest.  All calls share
 * the one array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and give wrong results, so serialize them.  The call blocks until
 * its result is in out.  Returns 0, PDLP_INVALID_ARGUMENT or PDLP_CUDA_ERROR. */
int pdlp_kkt_products_noalloc(int64_t m, int64_t n, const double* c, const double* lc,
                              const double* uc, const double* lv, const double* uv,
                              const double* x, const double* y, const double* ax,
                              const double* aty, void* cuda_stream, double* out);

/* One LP of a batch: the arguments of pdlp_solve, outputs included. */
typedef struct {
  int64_t m, n;
  pdlp_csr A;
  const double *c, *lc, *uc, *lv, *uv;
  double* x_out; /* [n] */
  double* y_out; /* [m] */
} pdlp_problem;

/* Solves `count` independent LPs of any sizes (a batch, e.g. many small LPs that one
 * solve alone cannot fill the GPU with): each LP runs the whole method of pdlp_solve --
 * its own step sizes (Algorithm 2), primal weight (Algorithm 3), restarts and
 * termination -- with the parameters *p for every LP.  `concurrency` LPs (<= 0: 16) are
 * in flight at once, each on its own CUDA stream driven by its own host thread, on the
 * calling thread's current device; device memory is allocated stream-ordered, so the
 * solves do not synchronise one another.  params->inputs_on_device selects host or
 * device arrays for every problem; params->cuda_stream, trace and polish-log outputs
 * are ignored.  status_out[count] receives each LP's pdlp_solve return value and
 * stats_out[count] (may be NULL) its statistics.  Returns 0 when every LP was attempted
 * (see status_out; pdlp_last_error() then describes the first LP that returned a
 * negative code), PDLP_INVALID_ARGUMENT for bad arguments of the call itself. */
int pdlp_solve_batch(int64_t count, const pdlp_problem* problems, const pdlp_params* p,
                     int concurrency, int* status_out, pdlp_stats* stats_out);

/* The batch of pdlp_solve_batch solved by ONE persistent kernel launch: each CTA takes
 * LPs from a device queue, largest first, and runs the whole method on its LP alone --
 * Algorithm 1 with the adaptive steps of Algorithm 2, the restart scheme of Sec. 3,
 * Algorithm 3's primal weight and App. C's infeasibility tests, each LP with its own
 * step sizes, primal weight, restarts and termination (the same rules as pdlp_solve,
 * with its own reduction order, so iterates agree with pdlp_solve's to rounding, not
 * bit for bit; one run is deterministic for a fixed `tune`).  The setup of Sec. 3
 * (preconditioning, layouts) runs per LP on 16 worker streams first.  The vectors the
 * two sparse products gather are held in shared memory when an LP's fit (x' and y',
 * else the one that fits, x' first).
 *   tune: 0 = autotune -- time three check periods of iterations of a sample of the
 *   batch (spread over its sizes) under every launch configuration and solve with the
 *   fastest; 1..6 = that
 *   configuration (threads per CTA / CTAs per SM / shared memory per CTA / staging):
 *   1 = 1024/1/200 KB/on, 2 = 1024/1/200 KB/off, 3 = 768/1/200 KB/on, 4 = 512/1/200 KB/on,
 *   5 = 512/2/100 KB/on, 6 = 512/2/100 KB/off.  tune_out (may be NULL) receives the
 *   configuration used.
 *   params: as pdlp_solve_batch; feasibility_polishing must be 0; trace, polish log,
 *   profile and verbose are ignored.  precision PDLP_FP32_BULK keeps FP64 for the KKT
 *   measures, the normalized gaps, the restart decisions and the primal weight.
 *   status_out[count], stats_out[count] (may be NULL) as pdlp_solve_batch; in stats,
 *   seconds_solve is the LP's device time inside the launch, seconds_setup its setup,
 *   seconds_total the whole call; ms_primal, ms_spmv_a, ms_spmv_at and ms_checks split
 *   seconds_solve by phase (the primal step; A x' with the dual step and Algorithm 2;
 *   A'y' with the running sums; evaluation points, start and output), and ms_gap,
 *   ms_kkt, ms_infeas the evaluation points' normalized gaps, KKT measures and
 *   infeasibility tests, in proportion to the SM clock cycles the CTA spent in each.
 * Returns 0 when every LP was attempted (see status_out), or a negative code for bad
 * arguments of the call itself. */
int pdlp_solve_batch_persistent(int64_t count, const pdlp_problem* problems, const pdlp_params* p,
                                int tune, int* status_out, pdlp_stats* stats_out, int* tune_out);

/* Unrolled PDHG and its adjoint (a differentiable layer; Eq. (3), Sec. 2): K steps of
 * Eq. (3) on the LP as given -- no preconditioning, restarts or adaptive steps: the
 * constant steps are tau = eta/omega, sigma = eta*omega (eta < 1/||A||_2 for the
 * convergence theory) -- from (proj_X(0), 0), with the dual step
 * y' = yh - proj_[-sigma uc, -sigma lc](yh), yh = y - sigma (2 A x' - A x).  Writes
 * x_K (x_out[n]) and y_K (y_out[m]).  With gx[n] and gy[m] non-NULL it also computes the
 * gradients of L = gx'x_K + gy'y_K with respect to c, lc, uc, lv, uv into the non-NULL
 * grad_* arrays (the vector-Jacobian product of the unrolled map; at a clamp boundary
 * the derivative of the inside branch is taken; infinite bounds get 0), by a reverse
 * pass that recomputes the iterates from checkpoints stored every checkpoint_every
 * steps (<= 0: 50): memory 2(m+n)(K/checkpoint_every + checkpoint_every + 2) values,
 * time about 3x the forward pass.  params->precision: PDLP_FP64 runs everything in
 * FP64; PDLP_FP32_BULK runs the forward iteration (matrix values, iterates, products,
 * checkpoints) in FP32 with steps rounded to FP32, and the reverse pass in FP64 (FP64
 * matrix and adjoints) with each clamp branch taken as the FP32 forward took it: the
 * gradient of the exact map along the FP32 trajectory.  inputs_on_device (host or
 * device arrays, outputs alike) and cuda_stream are used too; the rest is ignored.
 * Returns 0 or a negative error code. */
int pdlp_unrolled_pdhg(int64_t m, int64_t n, const pdlp_csr* A, const double* c,
                       const double* lc, const double* uc, const double* lv, const double* uv,
                       int64_t K, double eta, double omega, int64_t checkpoint_every,
                       const double* gx, const double* gy, const pdlp_params* p, double* x_out,
                       double* y_out, double* grad_c, double* grad_lc, double* grad_uc,
                       double* grad_lv, double* grad_uv);

/* One LP of a batch of unrolled-PDHG calls: the arguments of pdlp_unrolled_pdhg. */
typedef struct {
  int64_t m, n;
  pdlp_csr A;
  const double *c, *lc, *uc, *lv, *uv;
  int64_t K;
  double eta, omega;
  int64_t checkpoint_every;
  const double *gx, *gy;                      /* NULL: forward only          */
  double *x_out, *y_out;                      /* [n], [m]                    */
  double *grad_c, *grad_lc, *grad_uc, *grad_lv, *grad_uv; /* each may be NULL */
} pdlp_unrolled_problem;

/* pdlp_unrolled_pdhg for `count` LPs, `concurrency` (<= 0: 16) at a time on per-worker
 * streams and host threads of the calling thread's device (as pdlp_solve_batch).
 * status_out[count] receives each call's return value.  Returns 0 when every LP was
 * attempted (pdlp_last_error() then describes the first failed one), or
 * PDLP_INVALID_ARGUMENT. */
int pdlp_unrolled_pdhg_batch(int64_t count, const pdlp_unrolled_problem* problems,
                             const pdlp_params* p, int concurrency, int* status_out);

/* The batch of pdlp_unrolled_pdhg_batch run by ONE persistent kernel launch: each CTA
 * takes an LP from a device queue (the longest first) and runs its K steps of Eq. (3),
 * the checkpoints and, with an upstream gradient, the reverse pass, on its own -- the
 * computation of pdlp_unrolled_pdhg for that LP (each row's sum in the same entry order;
 * rows longer than 4096 entries are summed in another order).  An LP's forward state and
 * its two gathered FP64 adjoints live in the CTA's shared memory, so each LP must have
 * 2 (m + n) forward values (FP64, or FP32 for PDLP_FP32_BULK) plus 8 (m + n) bytes within
 * 200 KB (about m + n <= 8500 in FP64, 12800 with an FP32 forward); a larger LP fails
 * alone with PDLP_INVALID_ARGUMENT.  params: precision, inputs_on_device and
 * cuda_stream as pdlp_unrolled_pdhg; verbose = 1 prints one line to stderr with the host
 * time of the call's phases (the setup, also by step summed over the LPs; the launch with
 * the copies; the release); the rest is ignored.  status_out[count] receives
 * each LP's return value.  Returns 0 when every LP was attempted (pdlp_last_error()
 * then describes the first failed one), or PDLP_INVALID_ARGUMENT. */
int pdlp_unrolled_pdhg_batch_persistent(int64_t count, const pdlp_unrolled_problem* problems,
                                        const pdlp_params* p, int* status_out);

/* Message for the last nonzero return of a call made by this thread. */
const char* pdlp_last_error(void);

/* Measurement, not part of the solve: the random-gather ceiling of this GPU for the
 * access pattern of the two sparse products, which Sec. 5 ("Multithreading") finds
 * memory bound.  It times y = M t for a synthetic SELL-32 matrix M (32-row slices of
 * row_len entries each, floor(nnz / (32 row_len)) slices) whose entries gather one
 * element of a vector t of table_len elements: at uniform random indices (degree_s <=
 * 0), or (degree_s > 1, != 2) at the columns of a matrix whose table_len columns have
 * degrees from the truncated power law P(d) ~ d^-degree_s on [dmin, dmax], numbered by
 * decreasing degree as the solver numbers them.  method: 0 = one global load per entry
 * (the design of the solver's kernels), 1 = TMA tile::gather4 of 32-byte rows into
 * shared memory, 2 = half the warps each way; elem_bytes 8 (4 for method 0 only);
 * methods 1 and 2 need row_len 8 or 24.  The data are generated on the current device
 * (cudaMalloc'd for the call, freed before return); the best of reps timed launches
 * (after one warm-up) is reported.
 *   out[0] microseconds per launch, out[1] gathered entries per second, out[2] largest
 *   |y - y_LSU| of methods 1 and 2 against method 0 (0 for method 0), out[3] entries.
 * Returns 0, PDLP_INVALID_ARGUMENT, PDLP_OUT_OF_MEMORY or PDLP_CUDA_ERROR (also when a
 * bounded wait for a TMA copy gave up). */
int pdlp_gather_bench(int method, int elem_bytes, int64_t table_len, int row_len, int64_t nnz,
                      double degree_s, double dmin, double dmax, int reps, double* out);

#ifdef __cplusplus
}
#endif
#endif /* PDLP_H_ */
