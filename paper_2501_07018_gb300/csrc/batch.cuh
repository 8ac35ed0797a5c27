// Launch interface of the persistent batch kernel (batch_impl.cuh, instantiated by
// batch_f32.cu and batch_f64.cu): many LPs solved by one
// launch, one CTA per LP at a time.
#pragma once

#include "gap.cuh"
#include "pdhg.cuh"

namespace pdlp {

// Element type of the running sums of Algorithm 1: FP64 for both precisions.  In FP32
// the sum of thousands of steps of a restart period loses the digits the average
// iterate needs: on the uneven 64-LP batch at relative KKT 1e-6, FP32 sums took 5.3x the
// iterations of FP64 (one LP hit 400,000), FP64 sums the same count as FP64 throughout.
template <class T>
struct BatchSum {
  using type = double;
};

// One preconditioned, renumbered LP of a batch and its device work buffers (all
// device pointers, owned by the host driver).
template <class T>
struct BatchLP {
  using S = typename BatchSum<T>::type;
  Mat<T> A, AT;
  int64_t m, n;
  const T *c, *lc, *uc, *lv, *uv;  // preconditioned objective and bounds
  OrigVecs o;                      // unscaled FP64 vectors and the scalings D1, D2
  const int32_t *perm_r, *perm_c;  // renumbered -> caller's numbering
  double c_norm, b_norm;           // ||c||, ||Combine(lc, uc)|| of the unscaled LP
  double eta0, omega0;             // eta_hat = 1/||A~||_inf, InitializePrimalWeight
  T *X[2], *Y[2], *AX[2], *ATY[2];
  S *Sx, *Sy;                      // running sums of eta * x and eta * y (Algorithm 1)
  const uint16_t* a_col16;         // SELL column indices of A and A' in 16 bits when the
  const uint16_t* at_col16;        // matrix has <= 65536 columns (else null)
  T *X0, *Y0;                      // z^{n,0}
  T *Xa, *Ya, *AXa, *ATYa;         // the average since the last restart
  T *yd, *atyd, *xb, *axb;         // infeasibility candidates [m], [n], [3n], [3m]
  float4* gp_row;                  // FP32 bracket-scan parameters of the normalized
  float* gp_x;                     // gap: [m] per row, [3n] per column
  double *x_out, *y_out;           // device outputs in the caller's numbering
};

// The algorithm parameters every LP of the batch uses (from pdlp_params).
struct BatchParams {
  double eps_rel_kkt, eps_abs_feas, eps_rel_gap;
  int termination_mode, reduced_costs, check_period, max_retries, detect_infeasibility;
  int64_t max_iters;
  double time_limit_s, beta_suff, beta_nec, beta_art, theta, eps_zero, fixed_step, fixed_omega,
      eps_infeas;
  const double* step_tab;  // Algorithm 2's factors by accepted count (fill_step_table)
  int64_t step_len;
};

// Result of one LP, written by the CTA that solved it.
struct BatchResult {
  int32_t status;
  int32_t staged;  // gathered vectors held in shared memory: 1 x', 2 y'
  int64_t k, attempts, rejected, restarts[3], evaluations, gap_evals, gap_fallbacks,
      gap_failures;
  double rel_kkt, rel_primal, rel_dual, rel_gap, pres2, dres2, pres_inf, dres_inf, pobj, dobj,
      paper_gap, pres_rel_inf, dres_rel_inf;
  double omega, eta_hat;
  double seconds;  // device time of the LP's solve (global timer)
  int64_t sm;      // SM that solved it
  int64_t cycles[8];  // SM clock cycles by phase: primal step, A x' with the dual step and
                      // Algorithm 2, A'y' with the sums, evaluation points (other work),
                      // start and output, normalized gaps, KKT measures, infeasibility tests
};

// Launch configurations 1..batch_config_count() (threads per CTA, CTAs per SM, shared
// memory, staging; the table is in batch_impl.cuh and in include/pdlp.h).
int batch_config_count();
// CTAs of configuration `config` resident at once on this device.
template <class T>
int batch_resident_ctas(int config);
// Solves the LPs lps[order[0..count)] (device arrays) with `ctas` CTAs of configuration
// `config`; queue[0] must be 0.
template <class T>
void launch_batch(const BatchLP<T>* lps, const int32_t* order, int count, const BatchParams& prm,
                  BatchResult* res, unsigned int* queue, int config, int ctas, cudaStream_t s);

}  // namespace pdlp
