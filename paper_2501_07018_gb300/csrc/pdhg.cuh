// Launch interface of the PDHG iteration kernels (pdhg.cu).
#pragma once

#include "problem.cuh"

namespace pdlp {

// The iterate buffers of one solve.  X[b], Y[b], AX[b], ATY[b] for b in {0,1} hold two
// consecutive iterates; DevState::cur selects the accepted one (z^{n,t}), the other is
// written by a step attempt and becomes current when the attempt is accepted.
template <class T>
struct IterBuffers {
  T* X[2];
  T* Y[2];
  T* AX[2];
  T* ATY[2];
  T* Sx;   // running sums of eta * x, eta * y, eta * A x, eta * A'y since the restart
  T* Sy;
  T* SAx;
  T* SATy;
  const T* c;  // preconditioned objective and bounds
  const T* lc;
  const T* uc;
  const T* lv;
  const T* uv;
  int64_t m, n;
};

enum SpmvEpilogue { kEpiPlain = 0, kEpiDual = 1, kEpiAverage = 2 };

// Algorithm 2's factors 1 - (k+2)^-0.3 and 1 + (k+2)^-0.6 for accepted counts k in
// [0, len): f[2k], f[2k+1].  Precomputed (same device pow) so that the accept
// decision at the end of the A-side SpMV does not evaluate pow on a single lane.
struct StepTable {
  const double* f;
  int64_t len;
};
void fill_step_table(double* f, int64_t len, cudaStream_t s);

template <class T>
int spmv_grid(const Mat<T>& M, int epi);
int primal_grid(int64_t n);

// Eq. (3a) for the attempt of the current eta: X[cur^1] = proj_X(X[cur] - tau (c - ATY[cur]))
// and per-CTA partial sums of ||x' - x||^2 into part[grid].
template <class T>
void launch_primal(const IterBuffers<T>& b, DevState* st, double* part, int grid, cudaStream_t s);

// A x' with the dual step of Eq. (3b) fused into the row epilogue, the partial sums
// ||y'-y||^2 and (y'-y)'(Ax'-Ax), and, in the last CTA, Algorithm 2's accept/reject
// decision on the device (part_dual needs 2*grid doubles).
template <class T>
void launch_spmv_dual(const Mat<T>& A, const IterBuffers<T>& b, DevState* st,
                      const double* part_primal, int grid_primal, double* part_dual,
                      unsigned int* counter, StepTable tab, int grid, cudaStream_t s);

// A'y' with the running-average update (Algorithm 1) fused; a no-op when the last
// attempt was rejected.
template <class T>
void launch_spmv_avg(const Mat<T>& AT, const IterBuffers<T>& b, DevState* st, int grid,
                     cudaStream_t s);

// dst = M src
template <class T>
void launch_spmv_plain(const Mat<T>& M, const T* src, T* dst, int grid, cudaStream_t s);

}  // namespace pdlp
