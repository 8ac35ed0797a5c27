// Infeasibility detection (Sec. 3 "Infeasibility detection", App. C): the measures of
// the primal-infeasibility and dual-infeasibility certificate tests for three candidate
// directions per check -- the difference of the last two iterates, the current
// iterate, the average since the last restart -- on the unscaled LP.
//
// A candidate's y is projected onto Y and paired with the reduced costs
// r = proj_R(-A'y) that make ||A'y + r||_inf smallest; its x is projected onto the
// recession cone X-bar of the variable box and paired with the slack s = proj_Sbar(-Ax).
// Iterates and averages lie in Y already, so only the difference needs a product of its
// own on the A' side; every x candidate needs one on the A side (the projection onto
// X-bar zeroes the doubly bounded variables).
#include <algorithm>

#include "infeas.cuh"

namespace pdlp {
namespace {

__device__ __forceinline__ int64_t gi() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gs() { return (int64_t)gridDim.x * blockDim.x; }

// sign sets by which bounds are finite (the scaled bounds have the same pattern)
__device__ __forceinline__ double proj_y(double v, bool lf, bool uf) {
  if (lf && uf) return v;
  if (lf) return fmax(v, 0.0);
  if (uf) return fmin(v, 0.0);
  return 0.0;
}
__device__ __forceinline__ double proj_xbar(double v, bool lf, bool uf) {
  if (lf && uf) return 0.0;
  if (lf) return fmax(v, 0.0);
  if (uf) return fmin(v, 0.0);
  return v;
}
__device__ __forceinline__ double proj_r(double v, bool lf, bool uf) {
  if (lf && uf) return v;
  if (lf) return fmax(v, 0.0);
  if (uf) return fmin(v, 0.0);
  return 0.0;
}
__device__ __forceinline__ double proj_sbar(double v, bool lf, bool uf) {
  if (lf && uf) return 0.0;
  if (uf) return fmax(v, 0.0);  // only an upper bound: R^+
  if (lf) return fmin(v, 0.0);  // only a lower bound: R^-
  return v;
}

// The projected candidates and, per candidate, c'x-bar (unscaled): the dual test needs
// c'x-bar < 0, so the A-side products are formed only for candidates that pass it.
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_infeas_prep(InfeasInputs<T> in, InfeasScratch<T> sc, OrigVecs o, int64_t m, int64_t n) {
  __shared__ double red[3 * kWarps];
  __shared__ double mred[1 * kWarps];  // exact sizes: block_reduce_partials<3, 1>
  for (int64_t i = gi(); i < m; i += gs()) {
    const bool lf = isfinite(in.lc[i]), uf = isfinite(in.uc[i]);
    sc.yd[i] = (T)proj_y((double)in.y[i] - (double)in.y_prev[i], lf, uf);
  }
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t j = gi(); j < n; j += gs()) {
    const bool lf = isfinite(in.lv[j]), uf = isfinite(in.uv[j]);
    const T a = (T)proj_xbar((double)in.x[j] - (double)in.x_prev[j], lf, uf);
    const T b = (T)proj_xbar((double)in.x[j], lf, uf);
    const T c = (T)proj_xbar((double)in.xa[j], lf, uf);
    sc.xb[j] = a;
    sc.xb[n + j] = b;
    sc.xb[2 * n + j] = c;
    const double w = o.c[j] * o.d2[j];
    v[0] += w * (double)a;
    v[1] += w * (double)b;
    v[2] += w * (double)c;
  }
  block_sum<3>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) sc.part[k * G + blockIdx.x] = v[k];
    sc.part[3 * G + blockIdx.x] = 0.0;  // (no maximum is taken here)
  }
  if (!last_block_arrival(sc.counter)) return;
  double tot[3], unused[1];
  block_reduce_partials<3, 1>(sc.part, G, tot, unused, red, mred);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) sc.out[15 + k] = tot[k];
}

// 9 sums (y-objective rows, y-objective columns, c'x-bar per candidate) and 6 maxima
// (||A'y + r||_inf, ||A x + s||_inf per candidate); per-CTA partials, fixed-order total
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_infeas_reduce(InfeasInputs<T> in, InfeasScratch<T> sc, OrigVecs o, int64_t m, int64_t n,
                    unsigned xmask) {
  __shared__ double red[9 * kWarps];
  __shared__ double mred[6 * kWarps];
  const T* yc[3] = {sc.yd, in.y, in.ya};
  const T* atyc[3] = {sc.atyd, in.aty, in.atya};
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double mx[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = gi(); i < m; i += gs()) {
    const double l = o.lc[i], u = o.uc[i];
    const bool lf = isfinite(l), uf = isfinite(u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double y = (double)yc[c][i] * o.d1[i];
      if (y > 0.0)
        v[c] += l * y;
      else if (y < 0.0)
        v[c] += u * y;
      if (xmask & (1u << c)) {  // A x-bar formed for this candidate
        const double p = (double)sc.axb[c * m + i] * o.inv_d1[i];
        mx[3 + c] = fmax(mx[3 + c], fabs(p + proj_sbar(-p, lf, uf)));
      }
    }
  }
  for (int64_t j = gi(); j < n; j += gs()) {
    const double l = o.lv[j], u = o.uv[j];
    const bool lf = isfinite(l), uf = isfinite(u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double q = (double)atyc[c][j] * o.inv_d2[j];
      const double r = proj_r(-q, lf, uf);
      mx[c] = fmax(mx[c], fabs(q + r));
      if (r > 0.0)
        v[3 + c] += l * r;
      else if (r < 0.0)
        v[3 + c] += u * r;
      v[6 + c] += o.c[j] * ((double)sc.xb[c * n + j] * o.d2[j]);
    }
  }
  block_sum<9>(v, red);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double w = warp_max(mx[k]);
    if (lane == 0) mred[k * kWarps + warp] = w;
  }
  __syncthreads();
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 9; ++k) sc.part[k * G + blockIdx.x] = v[k];
    for (int k = 0; k < 6; ++k) {
      double a = 0.0;
      for (int w = 0; w < kWarps; ++w) a = fmax(a, mred[k * kWarps + w]);
      sc.part[(9 + k) * G + blockIdx.x] = a;
    }
  }
  if (!last_block_arrival(sc.counter)) return;
  double tot[9], mxt[6];
  block_reduce_partials<9, 6>(sc.part, G, tot, mxt, red, mred);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 9; ++k) sc.out[k] = tot[k];
    for (int k = 0; k < 6; ++k) sc.out[9 + k] = mxt[k];
  }
}

}  // namespace

template <class T>
InfeasMeasures infeasibility_measures(const InfeasInputs<T>& in, const InfeasScratch<T>& sc,
                                      const OrigVecs& o, const Mat<T>& A, const Mat<T>& AT,
                                      int grid_a, int grid_at, int64_t m, int64_t n,
                                      cudaStream_t s, int* launches) {
  const int64_t need = (std::max(m, n) + kThreads - 1) / kThreads;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
  k_infeas_prep<T><<<std::min(g, sc.grid), kThreads, 0, s>>>(in, sc, o, m, n);
  PDLP_LAUNCH_CHECK();
  launch_spmv_plain<T>(AT, sc.yd, sc.atyd, grid_at, s);
  double cx0[3];
  PDLP_CUDA_CHECK(cudaMemcpyAsync(cx0, sc.out + 15, sizeof(cx0), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  unsigned xmask = 0;
  int nl = 2;
  for (int c = 0; c < 3; ++c) {
    if (!(cx0[c] < 0.0)) continue;
    launch_spmv_plain<T>(A, sc.xb + c * n, sc.axb + c * m, grid_a, s);
    xmask |= 1u << c;
    ++nl;
  }
  k_infeas_reduce<T><<<sc.grid, kThreads, 0, s>>>(in, sc, o, m, n, xmask);
  PDLP_LAUNCH_CHECK();
  if (launches) *launches += nl + 1;
  double h[15];
  PDLP_CUDA_CHECK(cudaMemcpyAsync(h, sc.out, sizeof(h), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  InfeasMeasures r;
  for (int c = 0; c < 3; ++c) {
    r.y_obj[c] = h[c] + h[3 + c];
    r.cx[c] = h[6 + c];
    r.y_res[c] = h[9 + c];
    // a candidate without its product cannot pass the dual test (c'x-bar >= 0)
    r.x_res[c] = (xmask >> c) & 1u ? h[12 + c] : INFINITY;
  }
  return r;
}

template InfeasMeasures infeasibility_measures<double>(const InfeasInputs<double>&,
                                                       const InfeasScratch<double>&,
                                                       const OrigVecs&, const Mat<double>&,
                                                       const Mat<double>&, int, int, int64_t,
                                                       int64_t, cudaStream_t, int*);
template InfeasMeasures infeasibility_measures<float>(const InfeasInputs<float>&,
                                                      const InfeasScratch<float>&,
                                                      const OrigVecs&, const Mat<float>&,
                                                      const Mat<float>&, int, int, int64_t,
                                                      int64_t, cudaStream_t, int*);

}  // namespace pdlp
