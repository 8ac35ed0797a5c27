// Unrolled PDHG and its adjoint: K steps of Eq. (3) with fixed step sizes on the LP as
// given (identity scaling, the renumbered SELL layout of problem.cuh), and the
// reverse-mode derivative of (x_K, y_K) contracted with an upstream gradient (gx, gy)
// with respect to c, lc, uc, lv, uv.
//
// One forward step:  x' = clamp(x - tau (c - A'y), lv, uv);  Ax' = A x';
//                    yh = y - sigma (2 Ax' - Ax);  y' = yh - clamp(yh, -sigma uc, -sigma lc);
//                    A'y' = A' y'.
// One reverse step (adjoints bx, by of x', y'):
//   rows:     byh = by where yh is outside [-sigma uc, -sigma lc] (else 0);
//             g_uc += sigma by where yh < -sigma uc;  g_lc += sigma by where yh > -sigma lc
//   q = A' byh
//   columns:  bxn = bx - 2 sigma q  (the total adjoint of x');  u = x - tau (c - A'y);
//             bu = bxn strictly inside [lv, uv] (else 0); g_lv += bxn where u < lv;
//             g_uv += bxn where u > uv;  g_c -= tau bu;  bx <- sigma q + bu
//   r = A bu
//   rows:     by <- byh + tau r
// The iterates a reverse step needs are recomputed segment by segment from checkpoints
// stored every `checkpoint_every` steps of the forward pass.
#include <algorithm>
#include <vector>

#include "../../include/pdlp.h"
#include "adjoint.cuh"
#include "graph.cuh"

namespace pdlp {
namespace {

__device__ __forceinline__ int64_t gi() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gs() { return (int64_t)gridDim.x * blockDim.x; }

unsigned vgrid(int64_t len) {
  const int64_t need = (len + kThreads - 1) / kThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
}

// Forward kernels in the forward precision T (double, or float for FP32 forward).
template <class T>
__global__ void k_ad_start(const T* lv, const T* uv, T* x, T* y, T* aty, int64_t m, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    x[j] = fmin(fmax((T)0, lv[j]), uv[j]);
    aty[j] = (T)0;
  }
  for (int64_t i = gi(); i < m; i += gs()) y[i] = (T)0;
}

template <class T>
__global__ void k_ad_primal(const T* x, const T* aty, const T* c, const T* lv, const T* uv, T tau,
                            T* xn, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs())
    xn[j] = fmin(fmax(x[j] - tau * (c[j] - aty[j]), lv[j]), uv[j]);
}

template <class T>
__global__ void k_ad_dual(const T* y, const T* ax, const T* axn, const T* lc, const T* uc, T sigma,
                          T* yn, int64_t m) {
  for (int64_t i = gi(); i < m; i += gs()) {
    const T yh = y[i] - sigma * ((T)2 * axn[i] - ax[i]);
    yn[i] = yh - fmin(fmax(yh, -sigma * uc[i]), -sigma * lc[i]);
  }
}

// Reverse kernels: the clamp branches are re-evaluated on the recomputed iterates in the
// forward precision T, with the forward's own (T) step sizes and vectors, so that they
// are the branches the forward took; the adjoints accumulate in FP64 with the FP64 steps.
template <class T>
__global__ void k_ad_back_rows(const T* y, const T* ax, const T* axn, const T* lc, const T* uc,
                               T sigma_t, double sigma, const double* by, double* byh,
                               double* g_lc, double* g_uc, int64_t m) {
  for (int64_t i = gi(); i < m; i += gs()) {
    const T yh = y[i] - sigma_t * ((T)2 * axn[i] - ax[i]);
    const bool below = yh < -sigma_t * uc[i], above = yh > -sigma_t * lc[i];
    const double b = by[i];
    byh[i] = (below || above) ? b : 0.0;
    if (below) g_uc[i] += sigma * b;
    if (above) g_lc[i] += sigma * b;
  }
}

template <class T>
__global__ void k_ad_back_cols(const T* x, const T* aty, const T* c, const T* lv, const T* uv,
                               T tau_t, double tau, double sigma, const double* q, double* bx,
                               double* bu, double* g_c, double* g_lv, double* g_uv, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    const double bxn = bx[j] - 2.0 * sigma * q[j];
    const T u = x[j] - tau_t * (c[j] - aty[j]);
    const bool lo = u < lv[j], hi = u > uv[j];
    const double b = (lo || hi) ? 0.0 : bxn;
    if (lo) g_lv[j] += bxn;
    if (hi) g_uv[j] += bxn;
    g_c[j] -= tau * b;
    bu[j] = b;
    bx[j] = sigma * q[j] + b;
  }
}

__global__ void k_ad_back_y(const double* byh, const double* r, double tau, double* by, int64_t m) {
  for (int64_t i = gi(); i < m; i += gs()) by[i] = byh[i] + tau * r[i];
}

// x_0 = clamp(0, lv, uv) (branch in the forward precision); gradients of infinite
// bounds are 0
template <class T>
__global__ void k_ad_finish(const double* bx, const T* lc, const T* uc, const T* lv, const T* uv,
                            double* g_lc, double* g_uc, double* g_lv, double* g_uv, int64_t m,
                            int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    if ((T)0 < lv[j]) g_lv[j] += bx[j];
    if ((T)0 > uv[j]) g_uv[j] += bx[j];
    if (!isfinite(lv[j])) g_lv[j] = 0.0;
    if (!isfinite(uv[j])) g_uv[j] = 0.0;
  }
  for (int64_t i = gi(); i < m; i += gs()) {
    if (!isfinite(lc[i])) g_lc[i] = 0.0;
    if (!isfinite(uc[i])) g_uc[i] = 0.0;
  }
}

template <class T>
__global__ void k_scatter(const T* in, const int32_t* perm, double* out, int64_t len) {
  for (int64_t i = gi(); i < len; i += gs()) out[perm[i]] = (double)in[i];
}

}  // namespace

// state k of a trajectory: x, y, Ax, A'y at offsets 0, n, n+m, n+2m of a block of 2(n+m)
template <class T>
struct State {
  T *x, *y, *ax, *aty;
};
template <class T>
static State<T> state_at(T* base, int64_t k, int64_t m, int64_t n) {
  T* b = base + (size_t)k * 2 * (size_t)(m + n);
  return State<T>{b, b + n, b + n + m, b + n + 2 * m};
}

template <class T>
static void unrolled_forward_step(const UnrolledFwd<T>& F, int64_t m, int64_t n,
                                  const State<T>& s, const State<T>& t, cudaStream_t st) {
  k_ad_primal<T><<<vgrid(n), kThreads, 0, st>>>(s.x, s.aty, F.c, F.lv, F.uv, F.tau, t.x, n);
  PDLP_LAUNCH_CHECK();
  launch_spmv_plain<T>(F.A, t.x, t.ax, F.grid_a, st);
  if (m) {
    k_ad_dual<T><<<vgrid(m), kThreads, 0, st>>>(s.y, s.ax, t.ax, F.lc, F.uc, F.sigma, t.y, m);
    PDLP_LAUNCH_CHECK();
  }
  launch_spmv_plain<T>(F.AT, t.y, t.aty, F.grid_at, st);
}

template <class T>
int64_t unrolled_pdhg_run(DeviceArena& arena, const UnrolledProblem& U, const UnrolledFwd<T>& F,
                          int64_t K, int64_t every, const double* gx, const double* gy,
                          double* x_out, double* y_out, UnrolledGrads* grads, cudaStream_t st) {
  const int64_t m = U.P->m, n = U.P->n;
  const int64_t C = std::max<int64_t>(1, every);
  const int64_t ncp = K / C + 1;  // checkpoints at k = 0, C, 2C, ...
  const int64_t full = K / C;     // segments of C steps that end at a checkpoint
  const size_t state_bytes = sizeof(T) * 2 * (size_t)(m + n);
  T* cp = arena.alloc<T>(ncp * 2 * (m + n));
  T* seg = arena.alloc<T>((C + 1) * 2 * (m + n));
  int64_t launches = 0;
  auto copy_state = [&](const State<T>& dst, const State<T>& src) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dst.x, src.x, state_bytes, cudaMemcpyDeviceToDevice, st));
  };
  // forward: the running state alternates between seg slots 0 and 1, every full segment
  // starting in slot 0 (one captured sequence of C steps, replayed), its last state
  // copied to the checkpoint
  const State<T> s0 = state_at(cp, 0, m, n);
  k_ad_start<T><<<vgrid(std::max(m, n)), kThreads, 0, st>>>(F.lv, F.uv, s0.x, s0.y, s0.aty, m, n);
  PDLP_LAUNCH_CHECK();
  launch_spmv_plain<T>(F.A, s0.x, s0.ax, F.grid_a, st);
  launches += 2;
  copy_state(state_at(seg, 0, m, n), s0);
  auto forward_steps = [&](int64_t count) {
    for (int64_t i = 0; i < count; ++i)
      unrolled_forward_step<T>(F, m, n, state_at(seg, i % 2, m, n), state_at(seg, (i + 1) % 2, m, n),
                               st);
  };
  {
    Replay fwd;
    const bool graph = full >= 2 && fwd.capture(st, [&] { forward_steps(C); });
    for (int64_t sg = 0; sg < full; ++sg) {
      if (graph)
        fwd.launch(st);
      else
        forward_steps(C);
      launches += 4 * C;
      const State<T> end = state_at(seg, C % 2, m, n);
      copy_state(state_at(cp, sg + 1, m, n), end);
      if (C % 2) copy_state(state_at(seg, 0, m, n), end);
    }
  }
  const int64_t rest = K - full * C;
  forward_steps(rest);
  launches += 4 * rest;
  const State<T> cur = state_at(seg, rest % 2, m, n);
  // outputs x_K, y_K in the caller's numbering
  k_scatter<T><<<vgrid(n), kThreads, 0, st>>>(cur.x, U.P->perm_c, x_out, n);
  if (m) k_scatter<T><<<vgrid(m), kThreads, 0, st>>>(cur.y, U.P->perm_r, y_out, m);
  PDLP_LAUNCH_CHECK();
  launches += 2;
  if (!grads) return launches;

  // reverse pass: FP64 adjoints and the FP64 matrix
  double* bx = arena.alloc<double>(n);
  double* bu = arena.alloc<double>(n);
  double* q = arena.alloc<double>(n);
  double* by = arena.alloc<double>(m);
  double* byh = arena.alloc<double>(m);
  double* r = arena.alloc<double>(m);
  double* g[5];  // c, lc, uc, lv, uv (renumbered)
  const int64_t len[5] = {n, m, m, n, n};
  for (int k = 0; k < 5; ++k) {
    g[k] = arena.alloc<double>(len[k]);
    PDLP_CUDA_CHECK(cudaMemsetAsync(g[k], 0, sizeof(double) * std::max<int64_t>(1, len[k]), st));
  }
  gather_f64(gx, U.P->perm_c, bx, n, st);
  if (m) gather_f64(gy, U.P->perm_r, by, m, st);
  launches += 2;
  // one segment from its checkpoint (already in seg slot 0): recompute its states into
  // seg[0 .. steps], then the reverse steps from the last to the first
  auto segment_back = [&](int64_t steps) {
    for (int64_t i = 0; i < steps; ++i)
      unrolled_forward_step<T>(F, m, n, state_at(seg, i, m, n), state_at(seg, i + 1, m, n), st);
    for (int64_t i = steps - 1; i >= 0; --i) {
      const State<T> s = state_at(seg, i, m, n), t = state_at(seg, i + 1, m, n);
      if (m) {
        k_ad_back_rows<T><<<vgrid(m), kThreads, 0, st>>>(s.y, s.ax, t.ax, F.lc, F.uc, F.sigma,
                                                         U.sigma, by, byh, g[1], g[2], m);
        PDLP_LAUNCH_CHECK();
      }
      launch_spmv_plain<double>(U.P->AT, byh, q, U.grid_at, st);
      k_ad_back_cols<T><<<vgrid(n), kThreads, 0, st>>>(s.x, s.aty, F.c, F.lv, F.uv, F.tau, U.tau,
                                                       U.sigma, q, bx, bu, g[0], g[3], g[4], n);
      PDLP_LAUNCH_CHECK();
      launch_spmv_plain<double>(U.P->A, bu, r, U.grid_a, st);
      if (m) {
        k_ad_back_y<<<vgrid(m), kThreads, 0, st>>>(byh, r, U.tau, by, m);
        PDLP_LAUNCH_CHECK();
      }
    }
  };
  {
    Replay bwd;
    const bool graph = full >= 2 && bwd.capture(st, [&] { segment_back(C); });
    for (int64_t sgi = (K - 1) / C; K > 0 && sgi >= 0; --sgi) {
      const int64_t k0 = sgi * C, steps = std::min(K, k0 + C) - k0;
      copy_state(state_at(seg, 0, m, n), state_at(cp, sgi, m, n));
      if (graph && steps == C)
        bwd.launch(st);
      else
        segment_back(steps);
      launches += 9 * steps;
    }
  }
  k_ad_finish<T><<<vgrid(std::max(m, n)), kThreads, 0, st>>>(bx, F.lc, F.uc, F.lv, F.uv, g[1], g[2],
                                                             g[3], g[4], m, n);
  PDLP_LAUNCH_CHECK();
  double* outs[5] = {grads->c, grads->lc, grads->uc, grads->lv, grads->uv};
  const int32_t* perms[5] = {U.P->perm_c, U.P->perm_r, U.P->perm_r, U.P->perm_c, U.P->perm_c};
  for (int k = 0; k < 5; ++k) {
    if (!outs[k] || len[k] == 0) continue;
    k_scatter<double><<<vgrid(len[k]), kThreads, 0, st>>>(g[k], perms[k], outs[k], len[k]);
    PDLP_LAUNCH_CHECK();
    launches++;
  }
  return launches + 1;
}

template int64_t unrolled_pdhg_run<double>(DeviceArena&, const UnrolledProblem&,
                                           const UnrolledFwd<double>&, int64_t, int64_t,
                                           const double*, const double*, double*, double*,
                                           UnrolledGrads*, cudaStream_t);
template int64_t unrolled_pdhg_run<float>(DeviceArena&, const UnrolledProblem&,
                                          const UnrolledFwd<float>&, int64_t, int64_t,
                                          const double*, const double*, double*, double*,
                                          UnrolledGrads*, cudaStream_t);

}  // namespace pdlp
