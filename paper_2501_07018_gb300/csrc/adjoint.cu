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

__global__ void k_ad_start(const double* lv, const double* uv, double* x, double* y,
                           double* aty, int64_t m, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    x[j] = fmin(fmax(0.0, lv[j]), uv[j]);
    aty[j] = 0.0;
  }
  for (int64_t i = gi(); i < m; i += gs()) y[i] = 0.0;
}

__global__ void k_ad_primal(const double* x, const double* aty, const double* c, const double* lv,
                            const double* uv, double tau, double* xn, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs())
    xn[j] = fmin(fmax(x[j] - tau * (c[j] - aty[j]), lv[j]), uv[j]);
}

__global__ void k_ad_dual(const double* y, const double* ax, const double* axn, const double* lc,
                          const double* uc, double sigma, double* yn, int64_t m) {
  for (int64_t i = gi(); i < m; i += gs()) {
    const double yh = y[i] - sigma * (2.0 * axn[i] - ax[i]);
    yn[i] = yh - fmin(fmax(yh, -sigma * uc[i]), -sigma * lc[i]);
  }
}

__global__ void k_ad_back_rows(const double* y, const double* ax, const double* axn,
                               const double* lc, const double* uc, double sigma, const double* by,
                               double* byh, double* g_lc, double* g_uc, int64_t m) {
  for (int64_t i = gi(); i < m; i += gs()) {
    const double yh = y[i] - sigma * (2.0 * axn[i] - ax[i]);
    const bool below = yh < -sigma * uc[i], above = yh > -sigma * lc[i];
    const double b = by[i];
    byh[i] = (below || above) ? b : 0.0;
    if (below) g_uc[i] += sigma * b;
    if (above) g_lc[i] += sigma * b;
  }
}

__global__ void k_ad_back_cols(const double* x, const double* aty, const double* c,
                               const double* lv, const double* uv, double tau, double sigma,
                               const double* q, double* bx, double* bu, double* g_c,
                               double* g_lv, double* g_uv, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    const double bxn = bx[j] - 2.0 * sigma * q[j];
    const double u = x[j] - tau * (c[j] - aty[j]);
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

// x_0 = clamp(0, lv, uv); gradients of infinite bounds are 0
__global__ void k_ad_finish(const double* bx, const double* lc, const double* uc,
                            const double* lv, const double* uv, double* g_lc, double* g_uc,
                            double* g_lv, double* g_uv, int64_t m, int64_t n) {
  for (int64_t j = gi(); j < n; j += gs()) {
    if (0.0 < lv[j]) g_lv[j] += bx[j];
    if (0.0 > uv[j]) g_uv[j] += bx[j];
    if (!isfinite(lv[j])) g_lv[j] = 0.0;
    if (!isfinite(uv[j])) g_uv[j] = 0.0;
  }
  for (int64_t i = gi(); i < m; i += gs()) {
    if (!isfinite(lc[i])) g_lc[i] = 0.0;
    if (!isfinite(uc[i])) g_uc[i] = 0.0;
  }
}

__global__ void k_scatter(const double* in, const int32_t* perm, double* out, int64_t len) {
  for (int64_t i = gi(); i < len; i += gs()) out[perm[i]] = in[i];
}

}  // namespace

// state k of a trajectory: x, y, Ax, A'y at offsets 0, n, n+m, n+2m of a block of 2(n+m)
struct State {
  double *x, *y, *ax, *aty;
};
static State state_at(double* base, int64_t k, int64_t m, int64_t n) {
  double* b = base + (size_t)k * 2 * (size_t)(m + n);
  return State{b, b + n, b + n + m, b + n + 2 * m};
}

void unrolled_forward_step(const UnrolledProblem& U, const State& s, const State& t,
                           cudaStream_t st) {
  const int64_t m = U.P->m, n = U.P->n;
  k_ad_primal<<<vgrid(n), kThreads, 0, st>>>(s.x, s.aty, U.P->c, U.P->lv, U.P->uv, U.tau, t.x, n);
  PDLP_LAUNCH_CHECK();
  launch_spmv_plain<double>(U.P->A, t.x, t.ax, U.grid_a, st);
  if (m) {
    k_ad_dual<<<vgrid(m), kThreads, 0, st>>>(s.y, s.ax, t.ax, U.P->lc, U.P->uc, U.sigma, t.y, m);
    PDLP_LAUNCH_CHECK();
  }
  launch_spmv_plain<double>(U.P->AT, t.y, t.aty, U.grid_at, st);
}

int64_t unrolled_pdhg_run(DeviceArena& arena, const UnrolledProblem& U, int64_t K,
                          int64_t every, const double* gx, const double* gy, double* x_out,
                          double* y_out, UnrolledGrads* grads, cudaStream_t st) {
  const int64_t m = U.P->m, n = U.P->n;
  const int64_t C = std::max<int64_t>(1, every);
  const int64_t ncp = K / C + 1;  // checkpoints at k = 0, C, 2C, ...
  const int64_t full = K / C;     // segments of C steps that end at a checkpoint
  const size_t state_bytes = sizeof(double) * 2 * (size_t)(m + n);
  double* cp = arena.alloc<double>(ncp * 2 * (m + n));
  double* seg = arena.alloc<double>((C + 1) * 2 * (m + n));
  int64_t launches = 0;
  auto copy_state = [&](const State& dst, const State& src) {
    PDLP_CUDA_CHECK(cudaMemcpyAsync(dst.x, src.x, state_bytes, cudaMemcpyDeviceToDevice, st));
  };
  // forward: the running state alternates between seg slots 0 and 1, every full segment
  // starting in slot 0 (one captured sequence of C steps, replayed), its last state
  // copied to the checkpoint
  const State s0 = state_at(cp, 0, m, n);
  k_ad_start<<<vgrid(std::max(m, n)), kThreads, 0, st>>>(U.P->lv, U.P->uv, s0.x, s0.y, s0.aty, m, n);
  PDLP_LAUNCH_CHECK();
  launch_spmv_plain<double>(U.P->A, s0.x, s0.ax, U.grid_a, st);
  launches += 2;
  copy_state(state_at(seg, 0, m, n), s0);
  auto forward_steps = [&](int64_t count) {
    for (int64_t i = 0; i < count; ++i)
      unrolled_forward_step(U, state_at(seg, i % 2, m, n), state_at(seg, (i + 1) % 2, m, n), st);
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
      const State end = state_at(seg, C % 2, m, n);
      copy_state(state_at(cp, sg + 1, m, n), end);
      if (C % 2) copy_state(state_at(seg, 0, m, n), end);
    }
  }
  const int64_t rest = K - full * C;
  forward_steps(rest);
  launches += 4 * rest;
  const State cur = state_at(seg, rest % 2, m, n);
  // outputs x_K, y_K in the caller's numbering
  k_scatter<<<vgrid(n), kThreads, 0, st>>>(cur.x, U.P->perm_c, x_out, n);
  if (m) k_scatter<<<vgrid(m), kThreads, 0, st>>>(cur.y, U.P->perm_r, y_out, m);
  PDLP_LAUNCH_CHECK();
  launches += 2;
  if (!grads) return launches;

  // reverse pass
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
      unrolled_forward_step(U, state_at(seg, i, m, n), state_at(seg, i + 1, m, n), st);
    for (int64_t i = steps - 1; i >= 0; --i) {
      const State s = state_at(seg, i, m, n), t = state_at(seg, i + 1, m, n);
      if (m) {
        k_ad_back_rows<<<vgrid(m), kThreads, 0, st>>>(s.y, s.ax, t.ax, U.P->lc, U.P->uc, U.sigma,
                                                      by, byh, g[1], g[2], m);
        PDLP_LAUNCH_CHECK();
      }
      launch_spmv_plain<double>(U.P->AT, byh, q, U.grid_at, st);
      k_ad_back_cols<<<vgrid(n), kThreads, 0, st>>>(s.x, s.aty, U.P->c, U.P->lv, U.P->uv, U.tau,
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
  k_ad_finish<<<vgrid(std::max(m, n)), kThreads, 0, st>>>(bx, U.P->lc, U.P->uc, U.P->lv, U.P->uv,
                                                          g[1], g[2], g[3], g[4], m, n);
  PDLP_LAUNCH_CHECK();
  double* outs[5] = {grads->c, grads->lc, grads->uc, grads->lv, grads->uv};
  const int32_t* perms[5] = {U.P->perm_c, U.P->perm_r, U.P->perm_r, U.P->perm_c, U.P->perm_c};
  for (int k = 0; k < 5; ++k) {
    if (!outs[k] || len[k] == 0) continue;
    k_scatter<<<vgrid(len[k]), kThreads, 0, st>>>(g[k], perms[k], outs[k], len[k]);
    PDLP_LAUNCH_CHECK();
    launches++;
  }
  return launches + 1;
}

}  // namespace pdlp
