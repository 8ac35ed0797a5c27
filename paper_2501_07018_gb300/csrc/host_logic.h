// Decisions of the restart scheme (Sec. 3, "Adaptive restarts") and of the primal
// weight update (Algorithm 3), in plain C++ so that they compile and can be tested
// without a GPU.  The single-LP solver calls these on the host; the persistent batch
// kernel calls the same functions on the device (nvcc marks them __host__ __device__).
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define PDLP_HD __host__ __device__
#else
#define PDLP_HD
#endif

namespace pdlp {

// The first j >= 1 for which restart criterion (iii), t + j >= beta_art (k + j), holds
// after j more accepted iterations from (k accepted in total, t since the last restart);
// a quarter of INT64_MAX ("never") when beta_art >= 1 or is NaN, and also when that j
// exceeds 2^52 (no run gets that far; beyond it the doubles of the test below no
// longer resolve single iterations).  The host synchronises with the device at that
// iteration at the latest.
PDLP_HD inline int64_t steps_to_artificial(int64_t k, int64_t t, double beta_art) {
  const int64_t never = INT64_MAX / 4;
  if (!(beta_art < 1.0)) return never;
  int64_t j = 1;
  const double need = (beta_art * (double)k - (double)t) / (1.0 - beta_art);
  if (!(need < 4503599627370496.0)) return never;  // 2^52, NaN included
  if (need > 1.0) j = (int64_t)ceil(need);
  // the estimate may be off by rounding: settle on the first j that satisfies the test
  while (j > 1 && (double)(t + j - 1) >= beta_art * (double)(k + j - 1)) --j;
  while (!((double)(t + j) >= beta_art * (double)(k + j))) ++j;
  return j;
}

// Restart kind at an evaluation point: 0 none, 1 sufficient decay (i), 2 necessary decay
// with no progress (ii), 3 artificial (iii).  (i) and (ii) are tested only at the
// periodic checks and once mu(z^{n,0}, z^{n-1,0}) exists; (i) before (ii); (iii) only
// when neither holds.  mu_c_prev is the candidate gap of the previous check in the same
// outer loop (+inf if none).
PDLP_HD inline int restart_kind(bool is_check, bool is_art, bool have_mu_ref, double mu_c,
                        double mu_ref, double mu_c_prev, double beta_suff, double beta_nec) {
  int kind = 0;
  if (is_check && have_mu_ref) {
    if (mu_c <= beta_suff * mu_ref)
      kind = 1;
    else if (mu_c <= beta_nec * mu_ref && mu_c > mu_c_prev)
      kind = 2;
  }
  if (kind == 0 && is_art) kind = 3;
  return kind;
}

// Algorithm 3: omega <- exp(theta log(dy / dx) + (1 - theta) log(omega)) when both
// distances moved by the restart lie in (eps_zero, 1 / eps_zero); else omega unchanged.
PDLP_HD inline double primal_weight(double omega, double dx, double dy, double theta, double eps_zero) {
  if (eps_zero < dx && dx < 1.0 / eps_zero && eps_zero < dy && dy < 1.0 / eps_zero)
    return exp(theta * log(dy / dx) + (1.0 - theta) * log(omega));
  return omega;
}

}  // namespace pdlp
