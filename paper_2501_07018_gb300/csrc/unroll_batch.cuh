// Launch interface of the persistent unrolled-PDHG batch (unroll_batch.cu): many
// differentiable LP layers -- K fixed-step iterations of Eq. (3) and their adjoint --
// run by one launch, one CTA per LP at a time.
#pragma once

#include "problem.cuh"

namespace pdlp {

// One LP of the batch (device pointers, owned by the host driver).  Vectors are in the
// renumbered order of the SELL layouts; T is the forward precision.
template <class T>
struct UnrollLP {
  int64_t m, n, K, C;     // sizes, steps, checkpoint spacing
  double tau, sigma;      // the steps of the reverse pass (FP64)
  T tau_t, sigma_t;       // the forward steps rounded to T
  Mat<T> A, AT;           // forward layouts
  Mat<double> A64, AT64;  // FP64 layouts of the reverse pass (the same numbering)
  const T *c, *lc, *uc, *lv, *uv;
  const int32_t *perm_r, *perm_c;  // renumbered -> caller's numbering
  T* cp;                  // checkpoints: (K / C + 1) states of 2 (m + n) values
  T* seg;                 // one segment's recomputed states: (C + 1) states
  const double *gx, *gy;  // upstream gradient (renumbered; gx null: forward only)
  double *bx, *by;        // adjoints of x and y
  double *g[5];           // gradients wrt c, lc, uc, lv, uv (renumbered)
  double *x_out, *y_out;  // device outputs in the caller's numbering
  double *gout[5];        // device gradient outputs in the caller's numbering (or null)
};

// Shared memory one CTA needs for an LP with m rows and n columns (forward state in T,
// the two gathered adjoints in FP64), and the largest it may use.
size_t unroll_smem_need(int64_t m, int64_t n, size_t t_bytes);
size_t unroll_smem_max();
template <class T>
int unroll_resident_ctas();
// Runs lps[order[0..count)] (device arrays); queue[0] must be 0.
template <class T>
void launch_unroll_batch(const UnrollLP<T>* lps, const int32_t* order, int count,
                         unsigned int* queue, int ctas, cudaStream_t s);

}  // namespace pdlp
