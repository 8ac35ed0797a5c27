// Launch interface of the infeasibility-certificate measures (infeas.cu).
#pragma once

#include "gap.cuh"
#include "pdhg.cuh"

namespace pdlp {

// The three candidate directions of one check, as scaled and renumbered vectors:
// difference (x - x_prev, y - y_prev), current (x, y) with its A'y product, average
// (xa, ya) with its A'y product.  lc..uv are the scaled bounds (only their finiteness
// is used).
template <class T>
struct InfeasInputs {
  const T *x, *y, *aty;
  const T *x_prev, *y_prev;
  const T *xa, *ya, *atya;
  const T *lc, *uc, *lv, *uv;
};

// Work vectors: yd = proj_Y(y - y_prev) [m] and atyd = A~'yd [n]; xb = the three x
// candidates projected onto X-bar [3n] and axb = their A~ products [3m]; reduction
// partials [15 * grid], counter (0 between launches) and the results [18]: 15 measures,
// then c'x-bar of the three x candidates from the projection pass.
template <class T>
struct InfeasScratch {
  T* yd;
  T* atyd;
  T* xb;
  T* axb;
  double* part;
  unsigned int* counter;
  double* out;
  int grid;
};

// App. C's numbers per candidate c (0 difference, 1 current, 2 average):
// primal test: y_obj = lc'y+ - uc'y- + lv'r+ - uv'r-, y_res = ||A'y + r||_inf;
// dual test:   cx = c'x-bar, x_res = ||A x-bar + s||_inf.
struct InfeasMeasures {
  double y_obj[3], y_res[3], cx[3], x_res[3];
};

template <class T>
InfeasMeasures infeasibility_measures(const InfeasInputs<T>& in, const InfeasScratch<T>& sc,
                                      const OrigVecs& o, const Mat<T>& A, const Mat<T>& AT,
                                      int grid_a, int grid_at, int64_t m, int64_t n,
                                      cudaStream_t s, int* launches);

}  // namespace pdlp
