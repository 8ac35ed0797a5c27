// The PDHG iteration on the GPU (Sec. 2 Eq. (3), Algorithm 2, the running average of
// Algorithm 1), as three kernels per step attempt:
//   k_primal          x' = proj_X(x - tau (c - A'y))                       Eq. (3a)
//   k_spmv<kEpiDual>  A x', then per row y' = yhat - proj_[-s uc,-s lc](yhat),
//                     yhat = y - sigma (2 A x' - A x)                       Eq. (3b)
//                     + the step-size sums and, in the last CTA, the accept test
//   k_spmv<kEpiAverage>  A'y' and the running sums of eta * (x, y, Ax, A'y)
// Both sparse products share one tiled engine: a CTA stages a tile of rows (column
// indices and values, kChunk entries at most) in shared memory, then groups of G
// lanes reduce one row each; rows longer than kLongRow are split into chunks.
#include <algorithm>

#include "pdhg.cuh"

namespace pdlp {

__device__ __forceinline__ int64_t gtid2() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride2() { return (int64_t)gridDim.x * blockDim.x; }

template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  return fmin(fmax(v, lo), hi);
}
template <>
__device__ __forceinline__ float clampv<float>(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}

// ---------------------------------------------------------------------------
// Eq. (3a)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads) k_primal(IterBuffers<T> b, DevState* st, double* part) {
  __shared__ double red[kWarps];
  const int cur = st->cur;
  const bool err = st->error != 0;
  const double eta = st->eta, omega = st->omega;
  double acc[1] = {0.0};
  if (!err) {
    const T tau = (T)(eta / omega);
    const T* __restrict__ x = b.X[cur];
    const T* __restrict__ aty = b.ATY[cur];
    T* __restrict__ xn = b.X[cur ^ 1];
    for (int64_t j = gtid2(); j < b.n; j += gstride2()) {
      const T xo = x[j];
      const T v = clampv<T>(xo - tau * (b.c[j] - aty[j]), b.lv[j], b.uv[j]);
      xn[j] = v;
      const double d = (double)v - (double)xo;
      acc[0] += d * d;
    }
  }
  block_sum<1>(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
}

// ---------------------------------------------------------------------------
// tiled SpMV engine with fused row epilogues
// ---------------------------------------------------------------------------
template <class T>
struct SpmvArgs {
  Mat<T> M;
  const T* src;  // gathered vector
  T* dst;        // plain product output
  IterBuffers<T> b;
  DevState* st;
  const double* part_primal;
  int grid_primal;
  double* part_dual;
  unsigned int* counter;
};

// Per-launch scalars and pointers every CTA reads once (kept in registers).
template <class T>
struct EpiCtx {
  int cur;
  T sigma;    // kEpiDual
  T eta_acc;  // kEpiAverage
  const T* src;
  T* out0;        // plain: dst; dual: A x'; average: A'y'
  T* out1;        // dual: y'
  const T* in0;   // dual: A x; average: x'
  const T* in1;   // dual: y
  const T* lo;    // dual: lc
  const T* hi;    // dual: uc
  T* acc0;        // average: S x
  T* acc1;        // average: S A'y
};

// Row epilogue.  Returns the two step-size contributions for kEpiDual.
template <class T, int EPI>
__device__ __forceinline__ void row_epilogue(const EpiCtx<T>& e, int64_t row, T v, double& c0,
                                             double& c1) {
  if (EPI == kEpiPlain) {
    e.out0[row] = v;
  } else if (EPI == kEpiDual) {
    const T axo = e.in0[row];
    const T yo = e.in1[row];
    const T q = (T)2 * v - axo;
    const T yh = yo - e.sigma * q;
    const T yn = yh - clampv<T>(yh, -e.sigma * e.hi[row], -e.sigma * e.lo[row]);
    e.out0[row] = v;
    e.out1[row] = yn;
    const double dy = (double)yn - (double)yo;
    const double dax = (double)v - (double)axo;
    c0 += dy * dy;
    c1 += dy * dax;
  } else {
    e.out0[row] = v;
    e.acc0[row] += e.eta_acc * e.in0[row];
    e.acc1[row] += e.eta_acc * v;
  }
}

template <class T>
__device__ __forceinline__ T group_sum(T v, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T, int EPI, int G>
__device__ __forceinline__ void tile_rows(const EpiCtx<T>& e, int64_t r0,
                                          int nre, const int32_t* s_off, const int32_t* s_col,
                                          const T* s_val, double& c0, double& c1) {
  const int lane_g = threadIdx.x % G;
  const int gid = threadIdx.x / G;
  constexpr int ngroups = kThreads / G;
  const T* __restrict__ src = e.src;
  for (int base = 0; base < nre; base += ngroups) {
    const int rr = base + gid;
    T acc = (T)0;
    if (rr < nre) {
      const int pb = s_off[rr], pe = s_off[rr + 1];
      for (int p = pb + lane_g; p < pe; p += G) acc += s_val[p] * src[s_col[p]];
    }
    if (G > 1) acc = group_sum<T>(acc, G);
    if (rr < nre && lane_g == 0) row_epilogue<T, EPI>(e, r0 + rr, acc, c0, c1);
  }
}

template <class T, int EPI>
__global__ void __launch_bounds__(kThreads) k_spmv(SpmvArgs<T> a) {
  __shared__ int32_t s_off[kTileDiag + 1];
  __shared__ int32_t s_col[kChunk];
  __shared__ T s_val[kChunk];
  __shared__ double red[2 * kWarps];
  __shared__ int s_nre;

  EpiCtx<T> e;
  e.sigma = (T)0;
  e.eta_acc = (T)0;
  e.out1 = nullptr;
  e.in0 = e.in1 = e.lo = e.hi = nullptr;
  e.acc0 = e.acc1 = nullptr;
  if (EPI == kEpiPlain) {
    e.cur = 0;
    e.src = a.src;
    e.out0 = a.dst;
  } else {
    const int cur = a.st->cur;
    e.cur = cur;
    const bool err = a.st->error != 0;
    if (EPI == kEpiDual) {
      if (err) return;  // every CTA returns: the arrival counter stays consistent
      e.sigma = (T)(a.st->eta * a.st->omega);
      e.src = a.b.X[cur ^ 1];
      e.out0 = a.b.AX[cur ^ 1];
      e.out1 = a.b.Y[cur ^ 1];
      e.in0 = a.b.AX[cur];
      e.in1 = a.b.Y[cur];
      e.lo = a.b.lc;
      e.hi = a.b.uc;
    } else {
      if (err || a.st->accepted == 0) return;
      e.eta_acc = (T)a.st->eta_acc;
      e.src = a.b.Y[cur];
      e.out0 = a.b.ATY[cur];
      e.in0 = a.b.X[cur];
      e.acc0 = a.b.Sx;
      e.acc1 = a.b.SATy;
      // the m-side of the running sums (Algorithm 1): Sy += eta y', SAx += eta A x'
      const T* __restrict__ y = a.b.Y[cur];
      const T* __restrict__ ax = a.b.AX[cur];
      T* __restrict__ sy = a.b.Sy;
      T* __restrict__ sax = a.b.SAx;
      const T w = e.eta_acc;
      for (int64_t i = gtid2(); i < a.b.m; i += gstride2()) {
        sy[i] += w * y[i];
        sax[i] += w * ax[i];
      }
    }
  }

  const Mat<T>& M = a.M;
  double c0 = 0.0, c1 = 0.0;
  const int64_t items = (int64_t)M.ntiles + M.nchunks;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    if (it < M.ntiles) {
      const int64_t r0 = M.tile_row[it], r1 = M.tile_row[it + 1];
      const int nr = (int)(r1 - r0);
      if (nr == 0) continue;
      const int64_t nzb = M.row_ptr[r0];
      for (int i = threadIdx.x; i <= nr; i += kThreads) s_off[i] = (int32_t)(M.row_ptr[r0 + i] - nzb);
      __syncthreads();
      if (threadIdx.x == 0) s_nre = (s_off[nr] - s_off[nr - 1] > kLongRow) ? nr - 1 : nr;
      __syncthreads();
      const int nre = s_nre;
      const int nz = s_off[nre];
      for (int p = threadIdx.x; p < nz; p += kThreads) {
        s_col[p] = M.col[nzb + p];
        s_val[p] = M.val[nzb + p];
      }
      __syncthreads();
      const int avg = nre > 0 ? (nz + nre - 1) / nre : 1;
      if (avg <= 2)
        tile_rows<T, EPI, 1>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      else if (avg <= 4)
        tile_rows<T, EPI, 2>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      else if (avg <= 8)
        tile_rows<T, EPI, 4>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      else if (avg <= 16)
        tile_rows<T, EPI, 8>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      else if (avg <= 48)
        tile_rows<T, EPI, 16>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      else
        tile_rows<T, EPI, 32>(e, r0, nre, s_off, s_col, s_val, c0, c1);
      __syncthreads();
    } else {
      // one chunk of a long row
      const int64_t ci = it - M.ntiles;
      const int lr = M.chunk_owner[ci];
      const int64_t row = M.long_rows[lr];
      const int64_t first = M.chunk_ptr[lr];
      const int64_t nch = M.chunk_ptr[lr + 1] - first;
      const int64_t rb = M.row_ptr[row], re = M.row_ptr[row + 1];
      const int64_t pb = rb + (ci - first) * kChunk;
      const int64_t pe = min(pb + (int64_t)kChunk, re);
      T acc = (T)0;
      for (int64_t p = pb + threadIdx.x; p < pe; p += kThreads) acc += M.val[p] * e.src[M.col[p]];
      double v[1] = {(double)acc};
      block_sum<1>(v, red);
      if (threadIdx.x == 0) {
        M.long_part[ci] = v[0];
        __threadfence();
        const unsigned prev = atomicAdd(&M.long_cnt[lr], 1u);
        if (prev == (unsigned)(nch - 1)) {
          __threadfence();
          double sum = 0.0;
          for (int64_t q = 0; q < nch; ++q) sum += ((volatile double*)M.long_part)[first + q];
          M.long_cnt[lr] = 0u;
          double d0 = 0.0, d1 = 0.0;
          row_epilogue<T, EPI>(e, row, (T)sum, d0, d1);
          if (EPI == kEpiDual) {
            M.long_contrib[2 * lr] = d0;
            M.long_contrib[2 * lr + 1] = d1;
          }
        }
      }
    }
  }

  if (EPI != kEpiDual) return;

  // step-size sums: per CTA, then the last CTA reduces in fixed order and decides
  double v[2] = {c0, c1};
  block_sum<2>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    a.part_dual[blockIdx.x] = v[0];
    a.part_dual[G + blockIdx.x] = v[1];
  }
  if (!last_block_arrival(a.counter)) return;
  const double dx2 = block_sum_array(a.part_primal, a.grid_primal, red);
  const double dy2_t = block_sum_array(a.part_dual, G, red);
  const double in_t = block_sum_array(a.part_dual + G, G, red);
  double lc0[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < M.nlong; i += kThreads) {
    lc0[0] += ((volatile double*)M.long_contrib)[2 * i];
    lc0[1] += ((volatile double*)M.long_contrib)[2 * i + 1];
  }
  block_sum<2>(lc0, red);
  if (threadIdx.x != 0) return;
  const double dy2 = dy2_t + lc0[0];
  const double inter = in_t + lc0[1];
  DevState* s = a.st;
  const double omega = s->omega, eta = s->eta;
  // Algorithm 2 with the interaction taken in magnitude (Eq. (5) for K = -A)
  const double num = omega * dx2 + dy2 / omega;
  const double den = 2.0 * fabs(inter);
  const double eta_bar = den > 0.0 ? num / den : INFINITY;
  const double kf = (double)(s->k + 2);
  const double red_f = 1.0 - pow(kf, -0.3);
  const double grow_f = 1.0 + pow(kf, -0.6);
  const double eta_new = fmin(red_f * eta_bar, grow_f * eta);
  s->attempts += 1;
  s->last_dx2 = dx2;
  s->last_dy2 = dy2;
  s->last_inter = inter;
  s->last_eta_bar = eta_bar;
  if (!(isfinite(eta_new) && isfinite(num))) {
    s->error = 1;
    s->accepted = 0;
  } else if (eta <= eta_bar) {
    s->eta_acc = eta;
    s->eta_hat = eta_new;
    s->eta = eta_new;
    s->cur ^= 1;
    s->k += 1;
    s->t += 1;
    s->W += eta;
    s->accepted = 1;
    s->retries = 0;
  } else {
    s->eta = eta_new;
    s->accepted = 0;
    s->retries += 1;
    s->rejected += 1;
    if (s->retries >= s->max_retries) s->error = 2;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class T, int EPI>
static int spmv_grid_impl(const Mat<T>& M) {
  static int occ = 0;
  if (occ == 0) {
    PDLP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv<T, EPI>, kThreads, 0));
    if (occ < 1) occ = 1;
  }
  const int64_t items = M.work_items();
  const int64_t cap = (int64_t)num_sms() * occ;
  return (int)std::max<int64_t>(1, std::min(items, cap));
}

template <class T>
int spmv_grid(const Mat<T>& M, int epi) {
  if (epi == kEpiDual) return spmv_grid_impl<T, kEpiDual>(M);
  if (epi == kEpiAverage) return spmv_grid_impl<T, kEpiAverage>(M);
  return spmv_grid_impl<T, kEpiPlain>(M);
}

int primal_grid(int64_t n) {
  const int64_t need = (n + kThreads * 4 - 1) / (kThreads * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 4));
}

template <class T>
void launch_primal(const IterBuffers<T>& b, DevState* st, double* part, int grid, cudaStream_t s) {
  k_primal<T><<<grid, kThreads, 0, s>>>(b, st, part);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_dual(const Mat<T>& A, const IterBuffers<T>& b, DevState* st,
                      const double* part_primal, int grid_primal, double* part_dual,
                      unsigned int* counter, int grid, cudaStream_t s) {
  SpmvArgs<T> a{};
  a.M = A;
  a.b = b;
  a.st = st;
  a.part_primal = part_primal;
  a.grid_primal = grid_primal;
  a.part_dual = part_dual;
  a.counter = counter;
  k_spmv<T, kEpiDual><<<grid, kThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_avg(const Mat<T>& AT, const IterBuffers<T>& b, DevState* st, int grid,
                     cudaStream_t s) {
  SpmvArgs<T> a{};
  a.M = AT;
  a.b = b;
  a.st = st;
  k_spmv<T, kEpiAverage><<<grid, kThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

template <class T>
void launch_spmv_plain(const Mat<T>& M, const T* src, T* dst, int grid, cudaStream_t s) {
  SpmvArgs<T> a{};
  a.M = M;
  a.src = src;
  a.dst = dst;
  k_spmv<T, kEpiPlain><<<grid, kThreads, 0, s>>>(a);
  PDLP_LAUNCH_CHECK();
}

#define PDLP_INST(T)                                                                        \
  template int spmv_grid<T>(const Mat<T>&, int);                                            \
  template void launch_primal<T>(const IterBuffers<T>&, DevState*, double*, int, cudaStream_t); \
  template void launch_spmv_dual<T>(const Mat<T>&, const IterBuffers<T>&, DevState*,        \
                                    const double*, int, double*, unsigned int*, int,        \
                                    cudaStream_t);                                          \
  template void launch_spmv_avg<T>(const Mat<T>&, const IterBuffers<T>&, DevState*, int,    \
                                   cudaStream_t);                                           \
  template void launch_spmv_plain<T>(const Mat<T>&, const T*, T*, int, cudaStream_t);
PDLP_INST(double)
PDLP_INST(float)

}  // namespace pdlp
