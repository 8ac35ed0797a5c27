// Periodic-check kernels: optimality measures (termination test) and the
// normalized duality gap of Sec. 3 ("Adaptive restarts"), plus restart helpers.
//
// Normalized duality gap.  For z = (x, y) and radius r,
//   r * rho_r(z) = max { L(x,yh) - L(xh,y) : zh in X x Y, ||zh - z||_omega <= r }.
// The objective is separable: -g_j (xh_j - x_j) with g = c - A'y for every column, and
// h_i(yh_i) - h_i(y_i) with h_i(s) = (lc_i - (Ax)_i) s for s > 0, (uc_i - (Ax)_i) s for
// s < 0 for every row.  With a multiplier on the ball, parametrised by s = 1/lambda,
// every coordinate of the maximiser follows a path with at most three linear pieces
// (moving, parked at a bound or at 0, moving again), and along the path
//     ||zh(s) - z||_omega^2 = alpha(s) s^2 + gamma(s),   F(s) = beta(s) s + phi(s)
// with alpha, gamma, beta, phi piecewise constant: they change only at the
// coordinates' breakpoints.  The kernels find the piece where the squared distance
// crosses r^2 and solve alpha s^2 + gamma = r^2 there exactly:
//   pass 0    (FP64) r, the slope at s = 0+, the fully saturated limit
//   passes 1-4 (FP32) squared distance at kGapQ points: a geometric scan from the
//             lower bound r / slope, then three linear refinements of the bracket
//   exact     (FP64) coefficients at the bracket's left end, squared distance at its
//             right end (verifies the bracket), and the breakpoints inside it
//   finish    (one CTA) sorts those breakpoints and walks the pieces to the root.
// If the FP32 scan mislocates the bracket or leaves too many breakpoints in it, the
// host repeats the scan in FP64.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "gap.cuh"
#include "gap_paths.cuh"

namespace pdlp {

__device__ __forceinline__ int64_t gi() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gs() { return (int64_t)gridDim.x * blockDim.x; }

// ---------------------------------------------------------------------------
// KKT sums of a point of the preconditioned LP, evaluated on the unscaled LP:
// x = D2 x~, y = D1 y~, A x = D1^-1 (A~ x~), A'y = D2^-1 (A~' y~).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kThreads)
    k_kkt(PointRef<T> z, OrigVecs o, int64_t m, int64_t n, KktScratch ks, int rc_mode) {
  __shared__ double red[5 * kWarps];
  double v[5] = {0, 0, 0, 0, 0};  // pres2, dres2, pobj, dobj_rows, dobj_cols
  double mx[4] = {0, 0, 0, 0};     // l_inf residuals, then scaled by Eq. (10)'s q_i, w_j
  for (int64_t i = gi(); i < m; i += gs()) {
    const double ax = (double)z.ax[i] * o.inv_d1[i];
    const double y = (double)z.y[i] * o.d1[i];
    const double lc = o.lc[i], uc = o.uc[i];
    const double pr = ax - fmin(fmax(ax, lc), uc);
    v[0] += pr * pr;
    mx[0] = fmax(mx[0], fabs(pr));
    // q_i (Sec. 7, Eq. (10a)): the finite nonzero bounds' largest magnitude, else 1
    const bool lq = isfinite(lc) && lc != 0.0, uq = isfinite(uc) && uc != 0.0;
    const double q = lq ? (uq ? fmax(fabs(lc), fabs(uc)) : fabs(lc)) : (uq ? fabs(uc) : 1.0);
    mx[2] = fmax(mx[2], fabs(pr) / q);
    if (y > 0.0)
      v[3] += o.lc[i] * y;
    else if (y < 0.0)
      v[3] += o.uc[i] * y;
  }
  for (int64_t j = gi(); j < n; j += gs()) {
    const double x = (double)z.x[j] * o.d2[j];
    const double aty = (double)z.aty[j] * o.inv_d2[j];
    const double g = o.c[j] - aty;
    double r;
    if (rc_mode == 1) {
      // App. A: the reduced cost is kept only next to the bound it prices (relative to |x|)
      const bool near_lo = x - o.lv[j] <= fabs(x), near_hi = o.uv[j] - x <= fabs(x);
      r = (g > 0.0 && near_lo) ? g : ((g < 0.0 && near_hi) ? g : 0.0);
    } else {
      const bool lf = isfinite(o.lv[j]), uf = isfinite(o.uv[j]);
      r = g;
      if (lf && !uf) r = fmax(g, 0.0);
      if (!lf && uf) r = fmin(g, 0.0);
      if (!lf && !uf) r = 0.0;
    }
    const double dr = g - r;
    v[1] += dr * dr;
    mx[1] = fmax(mx[1], fabs(dr));
    mx[3] = fmax(mx[3], fabs(dr) / (o.c[j] != 0.0 ? fabs(o.c[j]) : 1.0));  // w_j, Eq. (10b)
    v[2] += o.c[j] * x;
    if (r > 0.0)
      v[4] += o.lv[j] * r;
    else if (r < 0.0)
      v[4] += o.uv[j] * r;
  }
  block_sum<5>(v, red);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double mred[4 * kWarps];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double t = warp_max(mx[k]);
    if (lane == 0) mred[k * kWarps + warp] = t;
  }
  __syncthreads();
  const int G = gridDim.x;
  static_assert(kKktPartials == 5 + 4, "KKT partial arrays");
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) ks.part[k * G + blockIdx.x] = v[k];
    for (int k = 0; k < 4; ++k) {
      double a = 0;
      for (int w = 0; w < kWarps; ++w) a = fmax(a, mred[k * kWarps + w]);
      ks.part[(5 + k) * G + blockIdx.x] = a;
    }
  }
  if (!last_block_arrival(ks.counter)) return;
  double tot[5], mxt[4];
  block_reduce_partials<5, 4>(ks.part, G, tot, mxt, red, mred);
  if (threadIdx.x == 0) {
    KktSums r;
    r.pres2 = tot[0];
    r.dres2 = tot[1];
    r.pobj = tot[2];
    r.dobj_rows = tot[3];
    r.dobj_cols = tot[4];
    r.pres_max = mxt[0];
    r.dres_max = mxt[1];
    r.pres_rel_max = mxt[2];
    r.dres_rel_max = mxt[3];
    *ks.out = r;
  }
}

template <class T>
void launch_kkt(const PointRef<T>& z, const OrigVecs& o, int64_t m, int64_t n,
                const KktScratch& ks, cudaStream_t s) {
  k_kkt<T><<<ks.grid, kThreads, 0, s>>>(z, o, m, n, ks, ks.rc_mode);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// restart helpers
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_average(const T* Sx, const T* Sy, const T* SAx, const T* SATy, double inv_w,
                          const T* lv, const T* uv, T* x, T* y, T* ax, T* aty, int64_t m,
                          int64_t n) {
  const T w = (T)inv_w;
  for (int64_t j = gi(); j < n; j += gs()) {
    const T v = Sx[j] * w;
    x[j] = v < lv[j] ? lv[j] : (v > uv[j] ? uv[j] : v);
    aty[j] = SATy[j] * w;
  }
  for (int64_t i = gi(); i < m; i += gs()) {
    y[i] = Sy[i] * w;
    ax[i] = SAx[i] * w;
  }
}

template <class T>
void launch_average(const T* Sx, const T* Sy, const T* SAx, const T* SATy, double inv_w,
                    const T* lv, const T* uv, T* x, T* y, T* ax, T* aty, int64_t m, int64_t n,
                    cudaStream_t s) {
  const int64_t need = (std::max(m, n) + kThreads - 1) / kThreads;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms() * 8));
  k_average<T><<<g, kThreads, 0, s>>>(Sx, Sy, SAx, SATy, inv_w, lv, uv, x, y, ax, aty, m, n);
  PDLP_LAUNCH_CHECK();
}

template <class T>
__global__ void __launch_bounds__(kThreads)
    k_dist2(const T* x, const T* x0, const T* y, const T* y0, int64_t m, int64_t n, double* part,
            unsigned int* counter, double* out2) {
  __shared__ double red[2 * kWarps];
  double v[2] = {0, 0};
  for (int64_t j = gi(); j < n; j += gs()) {
    const double d = (double)x[j] - (double)x0[j];
    v[0] += d * d;
  }
  for (int64_t i = gi(); i < m; i += gs()) {
    const double d = (double)y[i] - (double)y0[i];
    v[1] += d * d;
  }
  block_sum<2>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[G + blockIdx.x] = v[1];
  }
  if (!last_block_arrival(counter)) return;
  const double a = block_sum_array(part, G, red);
  const double b = block_sum_array(part + G, G, red);
  if (threadIdx.x == 0) {
    out2[0] = a;
    out2[1] = b;
  }
}

template <class T>
void launch_dist2(const T* x, const T* x0, const T* y, const T* y0, int64_t m, int64_t n,
                  double* part, unsigned int* counter, double* out2, int grid, cudaStream_t s) {
  k_dist2<T><<<grid, kThreads, 0, s>>>(x, x0, y, y0, m, n, part, counter, out2);
  PDLP_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// normalized duality gap
// ---------------------------------------------------------------------------
enum { kGapActive = 0, kGapDone = 1, kGapFailed = 2, kGapNeedMore = 3 };
enum { kPlanGeo = 0, kPlanLin = 1 };

struct GapCtx {
  int state;
  int plan;
  int ncand;
  int unb;
  double omega, r2, r;
  double slope2, dinf2, finf;
  double s_base;       // geometric plan: points s_base * 2^q
  double s_lb;         // lower bound r / slope
  double s_lo, s_hi;   // current bracket (linear plan)
  double alpha, gamma, beta, phi, d2lo, d2hi;
  double mu;
};

size_t gap_ctx_bytes() { return sizeof(GapCtx); }
size_t gap_param_bytes(int64_t m, int64_t n) {
  return sizeof(float4) * (size_t)m + 3 * sizeof(float) * (size_t)n + 256;
}

// FP32 parameters of the bracket scan, written by pass 0: per column
// (|g|, omega room, omega room^2) with |g| = 0 for a column that does not move; per
// row (omega |k1|, omega |k2|, |y|, y^2 / omega) with omega |k1| = 0 for a fixed row,
// |y| = +inf for a row that moves away forever and omega |k2| = 0 without a third piece.
struct ScanParams {
  float4* row;   // [m]
  float* xg;     // [n]
  float* xorm;   // [n]
  float* xsat;   // [n]
};

template <class T>
struct GapArgs {
  PointRef<T> z;
  const T* x_ref;
  const T* y_ref;
  ScaledVecs<T> p;
  GapCtx* ctx;
  double* part;
  unsigned int* counter;
  int64_t* cand;
  ScanParams sp;
};

// pass 0: r^2, slope^2 at 0+, saturated limits, unbounded count; FP32 scan parameters
template <class T>
__global__ void __launch_bounds__(kThreads) k_gap_pass0(GapArgs<T> a, double omega) {
  __shared__ double red6[6 * kWarps];
  // v: sum dx^2, sum dy^2 (r^2 = omega sum dx^2 + sum dy^2 / omega), dinf2, finf; the
  // slope at 0+ only positions the bracket and is accumulated in FP32
  double v[5] = {0, 0, 0, 0, 0};
  float slope = 0.0f;
  unsigned int unb = 0;
  const double om = omega, iom = 1.0 / omega;
  const float iomf = (float)iom, omf = (float)om;
  for (int64_t j = gi(); j < a.p.n; j += gs()) {
    const double x = a.z.x[j];
    const double dx = x - (double)a.x_ref[j];
    v[0] = fma(dx, dx, v[0]);
    const XPath q = x_path(x, a.p.c[j], a.z.aty[j], a.p.lv[j], a.p.uv[j]);
    const double orm = om * q.room;
    const float gaf = q.moves ? (float)q.ga : 0.0f, ormf = (float)orm, roomf = (float)q.room;
    a.sp.xg[j] = gaf;
    a.sp.xorm[j] = ormf;
    a.sp.xsat[j] = ormf * roomf;
    if (!q.moves) continue;
    if (q.room > 0.0) slope = fmaf(gaf * gaf, iomf, slope);  // every column that moves at 0+
    if (isinf(q.room)) {
      ++unb;
      continue;
    }
    v[2] = fma(orm, q.room, v[2]);
    v[3] = fma(q.ga, q.room, v[3]);
  }
  for (int64_t i = gi(); i < a.p.m; i += gs()) {
    const double y = a.z.y[i];
    const double dy = y - (double)a.y_ref[i];
    v[1] = fma(dy, dy, v[1]);
    const YPath q = y_path(y, a.p.lc[i], a.p.uc[i], a.z.ax[i]);
    const float yf = (float)q.y;
    const float y2f = yf * yf * iomf;
    const float w1 = omf * fabsf((float)q.k1);
    float4 prm;
    prm.x = q.kind == 0 ? 0.0f : w1;
    prm.y = q.kind == 3 ? omf * fabsf((float)q.k2) : 0.0f;
    prm.z = q.kind == 1 ? INFINITY : fabsf(yf);
    prm.w = y2f;
    a.sp.row[i] = prm;
    if (q.kind == 0) continue;
    slope = fmaf(w1, fabsf((float)q.k1), slope);
    if (q.kind == 1 || q.kind == 3) {
      ++unb;
      continue;
    }
    v[2] = fma(q.y * q.y, iom, v[2]);
    v[3] = fma(-q.k1, q.y, v[3]);
  }
  double w6[6] = {v[0], v[1], v[2], v[3], (double)unb, (double)slope};
  block_sum<6>(w6, red6);
  const int G = gridDim.x;
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) a.part[k * G + blockIdx.x] = w6[k];
  if (!last_block_arrival(a.counter)) return;
  double t[6];
  for (int k = 0; k < 6; ++k) t[k] = block_sum_array(a.part + k * G, G, red6);
  if (threadIdx.x != 0) return;
  GapCtx* c = a.ctx;
  c->omega = om;
  c->r2 = om * t[0] + t[1] / om;
  c->r = sqrt(c->r2);
  c->slope2 = t[5];
  c->dinf2 = t[2];
  c->finf = t[3];
  c->unb = (int)t[4];
  c->ncand = 0;
  c->plan = kPlanGeo;
  if (c->r2 == 0.0) {
    c->mu = 0.0;
    c->state = kGapDone;
  } else if (c->unb == 0 && c->dinf2 <= c->r2 * (1.0 + 1e-12)) {
    // every coordinate parks inside the ball (up to rounding): the maximiser is the
    // fully saturated point
    c->mu = c->finf / c->r;
    c->state = kGapDone;
  } else if (!(c->slope2 > 0.0)) {
    c->mu = 0.0;
    c->state = kGapDone;
  } else {
    // r / slope is a lower bound of the crossing; the slope is summed in FP32, so
    // back off by a margin far above its rounding error
    c->s_lb = (1.0 - 1e-4) * c->r / sqrt(c->slope2);
    c->s_base = c->s_lb;
    c->state = kGapActive;
  }
}

// New bracket from the squared distances d2 at the scan points (thread 0 of the last
// CTA of a scan)
__device__ void gap_update_bracket(GapCtx* c, const double* d2, const double* s_pts, int plan,
                                   int widen) {
  int first = -1;
  for (int q = 0; q < kGapQ; ++q)
    if (d2[q] >= c->r2) {
      first = q;
      break;
    }
  if (plan == kPlanGeo) {
    // points s_base * 2^(q - kGapQ/2); a crossing off either end moves the window
    // (the window spans 2^(kGapQ-1); moving it by that much makes windows abut)
    if (first < 0) {
      c->s_base = ldexp(c->s_base, kGapQ - 1);
      c->state = kGapNeedMore;
      return;
    }
    if (first == 0) {
      c->s_base = ldexp(c->s_base, -(kGapQ - 1));
      c->state = kGapNeedMore;
      return;
    }
    c->s_lo = s_pts[first - 1];
    c->s_hi = s_pts[first];
    c->plan = kPlanLin;
  } else {
    int lo_i = (first < 0 ? kGapQ : first) - 1;  // bracket [p_lo_i, p_lo_i+1], p_-1 = s_lo
    int hi_i = lo_i + 1;
    if (widen) {
      lo_i -= 1;
      hi_i += 1;
    }
    const double nlo = lo_i < 0 ? c->s_lo : s_pts[lo_i];
    const double nhi = hi_i >= kGapQ ? c->s_hi : s_pts[hi_i];
    c->s_lo = nlo;
    c->s_hi = nhi;
  }
}

// squared distance at kGapQ points, accumulated in Acc, from the pass-0 parameters
template <class T, class Acc>
__global__ void __launch_bounds__(kThreads) k_gap_scan(GapArgs<T> a, int plan, int widen) {
  __shared__ double red[kGapQ * kWarps];
  __shared__ double s_pts[kGapQ];
  GapCtx* c = a.ctx;
  if (c->state != kGapActive || c->plan != plan) return;
  const double om = c->omega;
  if (threadIdx.x < kGapQ) {
    const int q = threadIdx.x;
    s_pts[q] = (plan == kPlanGeo) ? ldexp(c->s_base, q - kGapQ / 2)
                                  : c->s_lo + (c->s_hi - c->s_lo) * (double)(q + 1) / (double)(kGapQ + 1);
  }
  __syncthreads();
  Acc pts[kGapQ];
#pragma unroll
  for (int q = 0; q < kGapQ; ++q) pts[q] = (Acc)s_pts[q];
  Acc acc[kGapQ];
#pragma unroll
  for (int q = 0; q < kGapQ; ++q) acc[q] = (Acc)0;
  const Acc iomA = (Acc)(1.0 / om);
  for (int64_t j = gi(); j < a.p.n; j += gs()) {
    const Acc ga = (Acc)a.sp.xg[j];
    if (ga == (Acc)0) continue;
    const Acc orm = (Acc)a.sp.xorm[j];
    const Acc sat = (Acc)a.sp.xsat[j];
#pragma unroll
    for (int q = 0; q < kGapQ; ++q) {
      const Acc t = pts[q] * ga;
      acc[q] += (t < orm) ? t * t * iomA : sat;
    }
  }
  for (int64_t i = gi(); i < a.p.m; i += gs()) {
    const float4 prm = a.sp.row[i];
    if (prm.x == 0.0f) continue;
    const Acc w1 = (Acc)prm.x, w2 = (Acc)prm.y, ay = (Acc)prm.z, y2 = (Acc)prm.w;
#pragma unroll
    for (int q = 0; q < kGapQ; ++q) {
      const Acc t1 = pts[q] * w1;
      Acc v;
      if (t1 < ay) {
        v = t1 * t1 * iomA;
      } else {
        const Acc t2 = pts[q] * w2;
        v = (w2 > (Acc)0 && t2 >= ay) ? t2 * t2 * iomA : y2;
      }
      acc[q] += v;
    }
  }
  // warp stage in Acc (a double shuffle tree per value would load the FP64 pipe more
  // than the scan itself), then one FP64 sum over the warps per value
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kGapQ; ++q) {
    Acc t = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    acc[q] = t;
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < kGapQ; ++q) red[q * kWarps + warp] = (double)acc[q];
  __syncthreads();
  const int G = gridDim.x;
  if (threadIdx.x < kGapQ) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += red[threadIdx.x * kWarps + w];
    a.part[threadIdx.x * G + blockIdx.x] = t;
  }
  if (!last_block_arrival(a.counter)) return;
  __shared__ double d2[kGapQ];
  {
    const double t = group_sum_arrays<kGapQ>(a.part, G);
    constexpr int GS = kThreads / kGapQ;
    if (threadIdx.x % GS == 0) d2[threadIdx.x / GS] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  gap_update_bracket(c, d2, s_pts, plan, widen);
}

// FP64 version of the scan for the fallback path: parameters recomputed in FP64
// from the vectors, so the bracket it returns is reliable where FP32 is not
template <class T>
__global__ void __launch_bounds__(kThreads) k_gap_scan64(GapArgs<T> a, int plan, int widen) {
  __shared__ double red[kGapQ * kWarps];
  __shared__ double s_pts[kGapQ];
  GapCtx* c = a.ctx;
  if (c->state != kGapActive || c->plan != plan) return;
  const double om = c->omega, iom = 1.0 / om;
  if (threadIdx.x < kGapQ) {
    const int q = threadIdx.x;
    s_pts[q] = (plan == kPlanGeo) ? ldexp(c->s_base, q - kGapQ / 2)
                                  : c->s_lo + (c->s_hi - c->s_lo) * (double)(q + 1) / (double)(kGapQ + 1);
  }
  __syncthreads();
  double acc[kGapQ];
#pragma unroll
  for (int q = 0; q < kGapQ; ++q) acc[q] = 0.0;
  for (int64_t j = gi(); j < a.p.n; j += gs()) {
    const XPath p = x_path(a.z.x[j], a.p.c[j], a.z.aty[j], a.p.lv[j], a.p.uv[j]);
    if (!p.moves) continue;
    const double orm = om * p.room, sat = orm * p.room;
#pragma unroll
    for (int q = 0; q < kGapQ; ++q) {
      const double t = s_pts[q] * p.ga;
      acc[q] += (t < orm) ? t * t * iom : sat;
    }
  }
  for (int64_t i = gi(); i < a.p.m; i += gs()) {
    const YPath p = y_path(a.z.y[i], a.p.lc[i], a.p.uc[i], a.z.ax[i]);
    if (p.kind == 0) continue;
    const double w1 = om * fabs(p.k1), w2 = om * fabs(p.k2), ay = fabs(p.y);
    const double y2 = p.y * p.y * iom;
#pragma unroll
    for (int q = 0; q < kGapQ; ++q) {
      const double t1 = s_pts[q] * w1;
      double v;
      if (p.kind == 1 || t1 < ay) {
        v = t1 * t1 * iom;
      } else {
        const double t2 = s_pts[q] * w2;
        v = (p.kind == 3 && t2 >= ay) ? t2 * t2 * iom : y2;
      }
      acc[q] += v;
    }
  }
  block_sum<kGapQ>(acc, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0)
    for (int q = 0; q < kGapQ; ++q) a.part[q * G + blockIdx.x] = acc[q];
  if (!last_block_arrival(a.counter)) return;
  __shared__ double d2[kGapQ];
  {
    const double t = group_sum_arrays<kGapQ>(a.part, G);
    constexpr int GS = kThreads / kGapQ;
    if (threadIdx.x % GS == 0) d2[threadIdx.x / GS] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  gap_update_bracket(c, d2, s_pts, plan, widen);
}

// exact FP64 coefficients at s_lo and the breakpoints in (s_lo, s_hi]; the squared
// distance at s_hi is verified by the finish kernel from these
template <class T>
__global__ void __launch_bounds__(kThreads) k_gap_exact(GapArgs<T> a) {
  __shared__ double red[4 * kWarps];
  GapCtx* c = a.ctx;
  if (c->state != kGapActive) return;
  const double om = c->omega, iom = 1.0 / om, slo = c->s_lo, shi = c->s_hi;
  double v[4] = {0, 0, 0, 0};  // alpha, gamma, beta, phi at s_lo
  for (int64_t j = gi(); j < a.p.n; j += gs()) {
    const XPath q = x_path(a.z.x[j], a.p.c[j], a.z.aty[j], a.p.lv[j], a.p.uv[j]);
    if (!q.moves) continue;
    x_coef(q, slo, om, iom, v);
    const double orm = om * q.room;
    if (slo * q.ga < orm && orm <= shi * q.ga) {
      const int k = atomicAdd(&c->ncand, 1);
      if (k < kGapCandCap) a.cand[k] = j * 4 + 0;
    }
  }
  for (int64_t i = gi(); i < a.p.m; i += gs()) {
    const YPath q = y_path(a.z.y[i], a.p.lc[i], a.p.uc[i], a.z.ax[i]);
    if (q.kind == 0) continue;
    y_coef(q, slo, om, iom, v);
    if (q.kind == 1) continue;
    const double ay = fabs(q.y);
    const double w1 = om * fabs(q.k1);
    if (slo * w1 < ay && ay <= shi * w1) {
      const int k = atomicAdd(&c->ncand, 1);
      if (k < kGapCandCap) a.cand[k] = i * 4 + 1;
    }
    if (q.kind == 3) {
      const double w2 = om * fabs(q.k2);
      if (slo * w2 < ay && ay <= shi * w2) {
        const int k = atomicAdd(&c->ncand, 1);
        if (k < kGapCandCap) a.cand[k] = i * 4 + 2;
      }
    }
  }
  block_sum<4>(v, red);
  const int G = gridDim.x;
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) a.part[k * G + blockIdx.x] = v[k];
  if (!last_block_arrival(a.counter)) return;
  double t[4];
  for (int k = 0; k < 4; ++k) t[k] = block_sum_array(a.part + k * G, G, red);
  if (threadIdx.x != 0) return;
  c->alpha = t[0];
  c->gamma = t[1];
  c->beta = t[2];
  c->phi = t[3];
  c->d2lo = t[0] * slo * slo + t[1];
  const int nc = ((volatile int*)&c->ncand)[0];
  // the crossing must not lie left of the bracket (up to rounding)
  if (!(c->d2lo < c->r2 * (1.0 + 1e-12)) || nc > kGapCandCap) c->state = kGapFailed;
}

// breakpoint value and coefficient change of one candidate
template <class T>
__device__ void cand_info(const GapArgs<T>& a, double om, int64_t code, double* bp, double* d4) {
  const int64_t idx = code >> 2;
  const int which = (int)(code & 3);
  if (which == 0)
    x_cand(x_path(a.z.x[idx], a.p.c[idx], a.z.aty[idx], a.p.lv[idx], a.p.uv[idx]), om, bp, d4);
  else
    y_cand(y_path(a.z.y[idx], a.p.lc[idx], a.p.uc[idx], a.z.ax[idx]), which, om, bp, d4);
}

constexpr int kFinPer = kGapCandCap / kThreads;

// one CTA: sort the breakpoints, prefix-sum their coefficient changes, find the piece
// where alpha s^2 + gamma reaches r^2 and solve there
template <class T>
__global__ void __launch_bounds__(kThreads) k_gap_finish(GapArgs<T> a) {
  __shared__ double s_key[kGapCandCap];
  __shared__ long long s_code[kGapCandCap];
  __shared__ double s_wsum[4][kWarps];
  __shared__ int s_first;
  GapCtx* c = a.ctx;
  if (c->state != kGapActive) return;
  const double om = c->omega;
  const int nc = c->ncand;
  const int tid = threadIdx.x;
  for (int i = tid; i < kGapCandCap; i += kThreads) {
    if (i < nc) {
      double d4[4];
      double bp;
      cand_info(a, om, a.cand[i], &bp, d4);
      s_key[i] = bp;
      s_code[i] = a.cand[i];
    } else {
      s_key[i] = INFINITY;
      s_code[i] = LLONG_MAX;
    }
  }
  __syncthreads();
  // bitonic sort by (key, code) over the smallest power of two holding the candidates
  int P = 2;
  while (P < nc) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += kThreads) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const double ki = s_key[i], kl = s_key[l];
          const long long ci = s_code[i], cl = s_code[l];
          const bool gt = (ki > kl) || (ki == kl && ci > cl);
          if (gt == up) {
            s_key[i] = kl;
            s_key[l] = ki;
            s_code[i] = cl;
            s_code[l] = ci;
          }
        }
      }
      __syncthreads();
    }
  }
  // exclusive prefix of the coefficient changes in sorted order; thread t owns the
  // consecutive items [t*kFinPer, (t+1)*kFinPer)
  double dl[kFinPer][4];
  double run[4] = {0, 0, 0, 0};
  for (int q = 0; q < kFinPer; ++q) {
    const int i = tid * kFinPer + q;
    double d4[4] = {0, 0, 0, 0};
    if (i < nc) {
      double bp;
      cand_info(a, om, s_code[i], &bp, d4);
    }
    for (int k = 0; k < 4; ++k) {
      dl[q][k] = run[k];
      run[k] += d4[k];
    }
  }
  const int lane = tid & 31, warp = tid >> 5;
  double off[4];
  for (int k = 0; k < 4; ++k) {
    double inc = run[k];
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_wsum[k][warp] = inc;
    off[k] = inc - run[k];
  }
  if (tid == 0) s_first = INT_MAX;
  __syncthreads();
  for (int k = 0; k < 4; ++k)
    for (int w = 0; w < warp; ++w) off[k] += s_wsum[k][w];
  const double al0 = c->alpha, ga0 = c->gamma, r2 = c->r2;
  for (int q = 0; q < kFinPer; ++q) {
    const int i = tid * kFinPer + q;
    if (i >= nc) break;
    const double al = al0 + (off[0] + dl[q][0]);
    const double gm = ga0 + (off[1] + dl[q][1]);
    const double b = s_key[i];
    if (al * b * b + gm >= r2) {
      atomicMin(&s_first, i);
      break;
    }
  }
  __syncthreads();
  const int first = s_first;
  // coefficients of the crossing piece: exclusive prefix at `first` (or the total)
  const int owner = (first == INT_MAX) ? -1 : first / kFinPer;
  __shared__ double s_coef[4];
  __shared__ double s_tot[4];
  if (tid == kThreads - 1)
    for (int k = 0; k < 4; ++k) s_tot[k] = off[k] + run[k];
  if (tid == owner)
    for (int k = 0; k < 4; ++k) s_coef[k] = off[k] + dl[first - owner * kFinPer][k];
  __syncthreads();
  if (tid != 0) return;
  {
    // verify the right end of the bracket: alpha(s_hi) s_hi^2 + gamma(s_hi) >= r^2
    const double a_hi = c->alpha + s_tot[0], g_hi = c->gamma + s_tot[1];
    c->d2hi = a_hi * c->s_hi * c->s_hi + g_hi;
    if (first == INT_MAX && !(c->d2hi >= r2 * (1.0 - 1e-12))) {
      c->state = kGapFailed;
      return;
    }
  }
  double cf[4];
  double lo_b, hi_b;
  if (first == INT_MAX) {
    for (int k = 0; k < 4; ++k) cf[k] = s_tot[k];
    lo_b = nc > 0 ? s_key[nc - 1] : c->s_lo;
    hi_b = c->s_hi;
  } else {
    for (int k = 0; k < 4; ++k) cf[k] = s_coef[k];
    lo_b = first == 0 ? c->s_lo : s_key[first - 1];
    hi_b = s_key[first];
  }
  const double al = c->alpha + cf[0], gm = c->gamma + cf[1];
  const double be = c->beta + cf[2], ph = c->phi + cf[3];
  double s_star = lo_b;
  if (al > 0.0) s_star = sqrt(fmax(r2 - gm, 0.0) / al);
  s_star = fmin(fmax(s_star, lo_b), hi_b);
  c->mu = (be * s_star + ph) / c->r;
  c->state = kGapDone;
}

// reset_base: restart the geometric window at the lower-bound estimate
__global__ void k_gap_set(GapCtx* c, int state, int plan, int reset_base) {
  c->state = state;
  c->plan = plan;
  if (reset_base) c->s_base = c->s_lb;
  c->ncand = 0;
}
__global__ void k_gap_clear_cand(GapCtx* c) { c->ncand = 0; }

// bracket narrowed to rounding width: F at its left end from the exact coefficients
__global__ void k_gap_degenerate(GapCtx* c) {
  c->mu = (c->beta * c->s_lo + c->phi) / c->r;
  c->state = kGapDone;
}

template <class T>
double normalized_gap(const PointRef<T>& z, const T* x_ref, const T* y_ref, double omega,
                      const ScaledVecs<T>& p, const GapScratch& gsc, cudaStream_t s,
                      int* launches, GapStats* stats) {
  if (stats) stats->evals++;
  GapArgs<T> a;
  a.z = z;
  a.x_ref = x_ref;
  a.y_ref = y_ref;
  a.p = p;
  a.ctx = gsc.ctx;
  a.part = gsc.part;
  a.counter = gsc.counter;
  a.cand = gsc.cand;
  {
    char* base = static_cast<char*>(gsc.params);
    a.sp.row = reinterpret_cast<float4*>(base);
    base += sizeof(float4) * (size_t)p.m;
    a.sp.xg = reinterpret_cast<float*>(base);
    a.sp.xorm = a.sp.xg + p.n;
    a.sp.xsat = a.sp.xorm + p.n;
  }
  const int G = gsc.grid;
  int nl = 0;
  k_gap_pass0<T><<<G, kThreads, 0, s>>>(a, omega);
  k_gap_scan<T, float><<<G, kThreads, 0, s>>>(a, kPlanGeo, 0);
  k_gap_scan<T, float><<<G, kThreads, 0, s>>>(a, kPlanLin, 0);
  k_gap_scan<T, float><<<G, kThreads, 0, s>>>(a, kPlanLin, 0);
  k_gap_scan<T, float><<<G, kThreads, 0, s>>>(a, kPlanLin, 1);
  k_gap_exact<T><<<G, kThreads, 0, s>>>(a);
  k_gap_finish<T><<<1, kThreads, 0, s>>>(a);
  nl += 7;
  PDLP_LAUNCH_CHECK();
  GapCtx h;
  PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, gsc.ctx, sizeof(GapCtx), cudaMemcpyDeviceToHost, s));
  PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
  if (h.state != kGapDone) {
    // FP64 scan: a geometric window around the slope estimate (moved until it holds
    // the crossing), then linear refinement until the exact pass accepts the bracket
    if (stats) stats->fallbacks++;
    for (int rep = 0; rep < 64; ++rep) {
      k_gap_set<<<1, 1, 0, s>>>(gsc.ctx, kGapActive, kPlanGeo, rep == 0 ? 1 : 0);
      k_gap_scan64<T><<<G, kThreads, 0, s>>>(a, kPlanGeo, 0);
      nl += 2;
      PDLP_LAUNCH_CHECK();
      PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, gsc.ctx, sizeof(GapCtx), cudaMemcpyDeviceToHost, s));
      PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
      if (h.state != kGapNeedMore) break;
    }
    for (int rep = 0; rep < 80 && h.state == kGapActive; ++rep) {
      k_gap_clear_cand<<<1, 1, 0, s>>>(gsc.ctx);
      k_gap_exact<T><<<G, kThreads, 0, s>>>(a);
      k_gap_finish<T><<<1, kThreads, 0, s>>>(a);
      nl += 3;
      PDLP_LAUNCH_CHECK();
      PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, gsc.ctx, sizeof(GapCtx), cudaMemcpyDeviceToHost, s));
      PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
      if (h.state == kGapDone) break;
      if (h.s_hi - h.s_lo <= 1e-15 * h.s_hi) {
        k_gap_degenerate<<<1, 1, 0, s>>>(gsc.ctx);
        nl += 1;
        PDLP_LAUNCH_CHECK();
        PDLP_CUDA_CHECK(cudaMemcpyAsync(&h, gsc.ctx, sizeof(GapCtx), cudaMemcpyDeviceToHost, s));
        PDLP_CUDA_CHECK(cudaStreamSynchronize(s));
        break;
      }
      k_gap_set<<<1, 1, 0, s>>>(gsc.ctx, kGapActive, kPlanLin, 0);
      k_gap_scan64<T><<<G, kThreads, 0, s>>>(a, kPlanLin, 1);
      nl += 2;
      PDLP_LAUNCH_CHECK();
      h.state = kGapActive;  // the next pass re-reads the device state
    }
    if (h.state != kGapDone) {
      char buf[320];
      std::snprintf(buf, sizeof(buf),
                    "normalized duality gap not resolved: state %d r2 %.17g s_lo %.17g s_hi %.17g "
                    "d2lo %.17g d2hi %.17g ncand %d unb %d dinf2 %.17g",
                    h.state, h.r2, h.s_lo, h.s_hi, h.d2lo, h.d2hi, h.ncand, h.unb, h.dinf2);
      if (stats) {
        stats->failures++;
        stats->last_failure = buf;
      }
      if (launches) *launches += nl;
      return NAN;
    }
  }
  if (launches) *launches += nl;
  return h.mu;
}

#define PDLP_GAP_INST(T)                                                                       \
  template void launch_kkt<T>(const PointRef<T>&, const OrigVecs&, int64_t, int64_t,            \
                              const KktScratch&, cudaStream_t);                                 \
  template double normalized_gap<T>(const PointRef<T>&, const T*, const T*, double,             \
                                    const ScaledVecs<T>&, const GapScratch&, cudaStream_t,      \
                                    int*, GapStats*);                                           \
  template void launch_average<T>(const T*, const T*, const T*, const T*, double, const T*,     \
                                  const T*, T*, T*, T*, T*, int64_t, int64_t, cudaStream_t);    \
  template void launch_dist2<T>(const T*, const T*, const T*, const T*, int64_t, int64_t,       \
                                double*, unsigned int*, double*, int, cudaStream_t);
PDLP_GAP_INST(double)
PDLP_GAP_INST(float)

}  // namespace pdlp
