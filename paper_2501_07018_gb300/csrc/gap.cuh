// Launch interface of the periodic-check kernels (gap.cu): KKT measures, the
// normalized duality gap, and the restart helpers.
#pragma once

#include <string>

#include "problem.cuh"

namespace pdlp {

// A point of the preconditioned LP together with its two matrix products.
template <class T>
struct PointRef {
  const T* x;
  const T* y;
  const T* ax;
  const T* aty;
};

// Scaled problem vectors (device).
template <class T>
struct ScaledVecs {
  const T* c;
  const T* lc;
  const T* uc;
  const T* lv;
  const T* uv;
  int64_t m, n;
};

// Unscaled problem vectors and the diagonal scalings (device, FP64).
struct OrigVecs {
  const double* c;
  const double* lc;
  const double* uc;
  const double* lv;
  const double* uv;
  const double* d1;
  const double* d2;
  const double* inv_d1;
  const double* inv_d2;
};

// KKT sums of a point (unscaled LP); see kkt_finish in solver.cu for their use.
struct KktSums {
  double pres2, dres2, pres_max, dres_max, pobj, dobj_rows, dobj_cols;
  double pres_rel_max, dres_rel_max;  // l_inf residuals scaled as in Sec. 7's Eq. (10)
};

// Scratch of the KKT reduction (partials, counter, result), sized for grid_ctas(4).
constexpr int kKktPartials = 9;  // 5 sums and 4 maxima per CTA
struct KktScratch {
  double* part;  // [kKktPartials * grid]
  unsigned int* counter;
  KktSums* out;
  int grid;
  int rc_mode = 0;  // reduced costs: 0 proj_R(c - A'y) (Sec. 2), 1 App. A's bound proximity
};
template <class T>
void launch_kkt(const PointRef<T>& z, const OrigVecs& o, int64_t m, int64_t n,
                const KktScratch& ks, cudaStream_t s);

// Normalized duality gap mu(z, z_ref) (Sec. 3 "Adaptive restarts") of a point of the
// preconditioned LP; see gap.cu for the method.
struct GapCtx;  // device-side context (opaque to the host)
struct GapScratch {
  GapCtx* ctx;
  double* part;  // [kGapPartials * grid]
  unsigned int* counter;
  int64_t* cand;  // [kGapCandCap] candidate breakpoints
  void* params;   // gap_param_bytes(m, n): FP32 scan parameters written by pass 0
  int grid;
};
size_t gap_param_bytes(int64_t m, int64_t n);
constexpr int kGapQ = 32;
constexpr int kGapCandCap = 2048;
constexpr int kGapPartials = kGapQ + 8;
size_t gap_ctx_bytes();

// Evaluation counters: `fallbacks` counts evaluations that needed the FP64 bracket
// scan, `failures` those that could not be resolved (the result is then NaN and
// `last_failure` describes the bracket).
struct GapStats {
  int64_t evals = 0, fallbacks = 0, failures = 0;
  std::string last_failure;
};
template <class T>
double normalized_gap(const PointRef<T>& z, const T* x_ref, const T* y_ref, double omega,
                      const ScaledVecs<T>& p, const GapScratch& gs, cudaStream_t s,
                      int* launches, GapStats* stats);

// Helpers of the restart step and of the check: x_avg = S x / W etc. (clamped into the
// box for x), copies, and sums of squared differences.
template <class T>
void launch_average(const T* Sx, const T* Sy, const T* SAx, const T* SATy, double inv_w,
                    const T* lv, const T* uv, T* x, T* y, T* ax, T* aty, int64_t m, int64_t n,
                    cudaStream_t s);
template <class T>
void launch_dist2(const T* x, const T* x0, const T* y, const T* y0, int64_t m, int64_t n,
                  double* part, unsigned int* counter, double* out2, int grid, cudaStream_t s);

}  // namespace pdlp
