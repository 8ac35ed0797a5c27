// Interface of the unrolled-PDHG forward and adjoint passes (adjoint.cu).
#pragma once

#include "pdhg.cuh"
#include "problem.cuh"

namespace pdlp {

// The LP (identity scaling, renumbered SELL layout) and the fixed step sizes.
struct UnrolledLp {
  int64_t m, n;
  Mat<double> A, AT;
  const double *c, *lc, *uc, *lv, *uv;  // renumbered
  const int32_t *perm_r, *perm_c;       // new -> caller's numbering
};
struct UnrolledProblem {
  const UnrolledLp* P;
  double tau, sigma;
  int grid_a, grid_at;
};

// The forward iteration in precision T (double, or float for an FP32 forward): the
// matrix and vectors in T, and the step sizes rounded to T.
template <class T>
struct UnrolledFwd {
  Mat<T> A, AT;
  const T *c, *lc, *uc, *lv, *uv;  // renumbered
  T tau, sigma;
  int grid_a, grid_at;
};

// Output gradients in the caller's numbering (each may be null).
struct UnrolledGrads {
  double *c, *lc, *uc, *lv, *uv;
};

// K steps of F from (proj_X(0), 0), checkpoints every `every` steps; x_out/y_out
// receive x_K, y_K (FP64); with grads, the reverse pass contracts the derivative with
// (gx, gy) (device arrays in the caller's numbering) in FP64 with U's FP64 matrix and
// steps, the clamp branches taken from the recomputed T iterates.  Returns the number
// of kernel launches.
template <class T>
int64_t unrolled_pdhg_run(DeviceArena& arena, const UnrolledProblem& U, const UnrolledFwd<T>& F,
                          int64_t K, int64_t every, const double* gx, const double* gy,
                          double* x_out, double* y_out, UnrolledGrads* grads, cudaStream_t st);

}  // namespace pdlp
