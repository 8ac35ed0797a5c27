// Persistent batched PDLP (templates; batch_f32.cu and batch_f64.cu instantiate them):
// one launch solves many LPs of uneven sizes.
//
// Every CTA takes LPs from a device queue (largest first) and runs the whole method on
// its LP alone, separated into phases by CTA barriers:
//   Eq. (3a)                  x' = proj_X(x - tau (c - A'y))       (threads over columns)
//   A x' + Eq. (3b)           y' = yh - proj_[-s uc, -s lc](yh)   (warps over SELL slices)
//   Algorithm 2               accept / reject on eta_bar          (thread 0)
//   A'y' + Algorithm 1 sums   running sums of eta * (x, y, Ax, A'y)
//   periodic checks (Sec. 3)  KKT measures of the restart candidate, the normalized
//                             duality gaps of the current and the average iterate,
//                             restart criteria (i)-(iii), Algorithm 3's primal weight,
//                             App. C's infeasibility tests
// so that an LP never needs a grid-wide synchronisation and each LP keeps its own step
// sizes, primal weight, restarts and termination.  The preconditioning (Sec. 3) and the
// SELL-32 layouts come from the single-LP setup.
//
// GB300 specifics: the two vectors the sparse products gather (x' and y') are staged in
// shared memory when they fit, so the random gathers of an LP hit shared memory (several
// entries per clock per SM) instead of the L1/L2 path (under one per clock); the
// matrices stream through with evict-first loads.  The FP64 pipe is narrow (2 lanes per
// clock per SM), so scalar FP64 logic runs on one thread and is broadcast through
// shared memory, and FP32-bulk reductions shuffle in FP32 before one FP64 sum across
// warps.  Scalars that every thread needs are computed once by thread 0.
#pragma once

#include <math.h>

#include "../../include/pdlp.h"
#include "batch.cuh"
#include "gap_paths.cuh"
#include "host_logic.h"

namespace pdlp {
namespace {

constexpr int kQ = 16;      // points per bracket scan of the normalized gap
constexpr int kCap = 2048;  // breakpoints resolved exactly per gap evaluation
constexpr int kMaxK = 32;   // values per CTA reduction
// Configurations of the persistent launch (the autotuner times them all): threads per
// CTA, CTAs per SM (which sets the registers per thread: 65536 / (threads x CTAs)), the
// dynamic shared memory per CTA and whether x' and y' are staged in it.
struct BatchConfig {
  int threads, per_sm, smem_kb;
  bool stage;
};
constexpr BatchConfig kConfigs[] = {
    {1024, 1, 200, true}, {1024, 1, 200, false}, {768, 1, 200, true},
    {512, 1, 200, true},  {512, 2, 100, true},   {512, 2, 100, false},
};
constexpr int kNumConfigs = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));

// entries per lane in flight in the products: 8 with 128 registers per thread, fewer
// where a thread has 64 or 80
#ifndef PDLP_BATCH_B_SMALL_REGS
#define PDLP_BATCH_B_SMALL_REGS 4
#endif
#ifndef PDLP_BATCH_B_THRESHOLD
#define PDLP_BATCH_B_THRESHOLD 768
#endif

enum { kGActive = 0, kGDone = 1, kGFailed = 2, kGNeedMore = 3 };
enum { kGeo = 0, kLin = 1 };
enum { kEpPlain = 0, kEpDual = 1, kEpAvg = 2 };

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-thread accumulator of the step-size sums: FP64 for the FP64 path, FP32 for FP32
// bulk (combined across warps in FP64).
template <class T>
struct Acc {
  using type = double;
};
template <>
struct Acc<float> {
  using type = float;
};

// Monotone integer key of a non-NaN double (clamps on the integer pipe).
__device__ __forceinline__ long long dkey(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
template <class T>
__device__ __forceinline__ T clampv(T v, T lo, T hi);
template <>
__device__ __forceinline__ double clampv<double>(double v, double lo, double hi) {
  const long long kv = dkey(v);
  return kv < dkey(lo) ? lo : (kv > dkey(hi) ? hi : v);
}
template <>
__device__ __forceinline__ float clampv<float>(float v, float lo, float hi) {
  return fminf(fmaxf(v, lo), hi);
}
__device__ __forceinline__ bool neg_strict(double v) {
  const long long b = __double_as_longlong(v);
  return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool pos_strict(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool neg_strict(float v) { return v < 0.0f; }
__device__ __forceinline__ bool pos_strict(float v) { return v > 0.0f; }

// Optimality measures of a point on the unscaled LP (the termination test).
struct Kkt {
  double rel_kkt, rel_primal, rel_dual, rel_gap, pres2, dres2, pres_inf, dres_inf, pobj, dobj,
      paper_gap, pres_rel_inf, dres_rel_inf;
};

template <class T>
struct Sh {
  double red[kMaxK * 32];  // per-warp partials of a reduction
  double out[kMaxK];       // its totals, read by every thread
  // LP state (written by thread 0 between barriers)
  int64_t k, t, attempts, rejected, restarts[3], evaluations, gap_evals, gap_fallbacks,
      gap_failures;
  double eta, eta_hat, eta_acc, omega, W, mu_ref, mu_c_prev;
  int cur, accepted, retries, err, have_mu_ref;
  int ev;        // evaluation point after the last accepted step: 1 check, 2 (iii), 4 limit
  // thread 0's verdicts broadcast to the CTA, one field each (a field is rewritten only
  // after a barrier that follows every read of its previous value)
  int dec_avg, dec_conv, dec_time;
  T tau, sigma;  // step scalars broadcast to every thread
  typename BatchSum<T>::type wacc, winv;
  unsigned long long t0;
  long long cyc[8];  // SM cycles by phase (thread 0's clock between barriers)
  long long mark;    // thread 0's clock at the last phase boundary
  // normalized-gap evaluation (thread 0 keeps the bracket)
  int g_state, g_plan, ncand, first;
  double g_om, g_r2, g_r, g_slope2, g_dinf2, g_finf, g_sbase, g_slb, g_slo, g_shi;
  double g_alpha, g_gamma, g_beta, g_phi, g_mu;
  double s_pts[kQ];
  double coef[4], tot[4];
  double woff[4][32];
  Kkt kk;
  double im[18];  // infeasibility measures
  int flag;
};

// ---------------------------------------------------------------------------
// CTA reductions (fixed order: lanes, then warps in order; deterministic)
// ---------------------------------------------------------------------------
template <int NT, int K, class A, class T>
__device__ __forceinline__ void cta_sum(A (&v)[K], Sh<T>& sh) {
  constexpr int NW = NT / 32;
  static_assert(K <= kMaxK, "reduction width");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh.red[k * NW + w] = (double)t;
  }
  __syncthreads();
  if (w == 0 && lane < K) {
    double s = 0.0;
    for (int q = 0; q < NW; ++q) s += sh.red[lane * NW + q];
    sh.out[lane] = s;
  }
  __syncthreads();
}

// maxima of non-negative values
template <int NT, int K, class T>
__device__ __forceinline__ void cta_max(double (&v)[K], Sh<T>& sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) sh.red[k * NW + w] = t;
  }
  __syncthreads();
  if (w == 0 && lane < K) {
    double s = 0.0;
    for (int q = 0; q < NW; ++q) s = fmax(s, sh.red[lane * NW + q]);
    sh.out[lane] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// sparse products of one LP by one CTA (warp w takes items w, w + NW, ...: long rows
// in CSR, then SELL-32 slices with one row per lane; entries in stored order)
// ---------------------------------------------------------------------------
template <class T>
struct Epi {
  const T* src;  // gathered vector (shared or global memory)
  T* out0;       // the product (A x', A'y', or the plain product)
  T* out1;       // dual: y'
  T* stage1;     // dual: shared copy of y' (or null)
  const T* in0;  // dual: A x; average: x'
  const T* in1;  // dual: y
  const T* lo;   // dual: lc
  const T* hi;   // dual: uc
  typename BatchSum<T>::type* acc0;  // average: S x
  T sigma;
  typename BatchSum<T>::type wacc;
};

// Epilogue operands of one row, loaded before its product is formed so that their
// latency overlaps the matrix stream.
template <class T>
struct EpiIn {
  T a, b, c, d;
  typename BatchSum<T>::type s0;
};

template <class T, int EPI>
__device__ __forceinline__ EpiIn<T> epi_load(const Epi<T>& e, int64_t row) {
  EpiIn<T> r{};
  if (EPI == kEpDual) {
    r.a = e.in0[row];
    r.b = e.in1[row];
    r.c = __ldg(e.lo + row);
    r.d = __ldg(e.hi + row);
  } else if (EPI == kEpAvg) {
    r.a = e.in0[row];
    r.s0 = e.acc0[row];
  }
  return r;
}

template <class T, int EPI, class A>
__device__ __forceinline__ void epilogue(const Epi<T>& e, const EpiIn<T>& in, int64_t row, T v,
                                         A& c0, A& c1) {
  if (EPI == kEpPlain) {
    e.out0[row] = v;
  } else if (EPI == kEpDual) {
    const T axo = in.a, yo = in.b;
    const T lo = in.c, hi = in.d;
    // Eq. (3b) by Sec. 2's case analysis: y' = yh + sigma uc if negative, yh + sigma lc if
    // positive, else 0, with yh = y - sigma (2 A x' - A x)
    const T yh = yo - e.sigma * ((T)2 * v - axo);
    const T tu = fma(e.sigma, hi, yh);
    const T tl = fma(e.sigma, lo, yh);
    const T yn = neg_strict(tu) ? tu : (pos_strict(tl) ? tl : (T)0);
    e.out0[row] = v;
    e.out1[row] = yn;
    if (e.stage1) e.stage1[row] = yn;
    const A dy = (A)yn - (A)yo;
    const A dax = (A)v - (A)axo;
    c0 = fma(dy, dy, c0);
    c1 = fma(dy, dax, c1);
  } else {
    using S = typename BatchSum<T>::type;
    e.out0[row] = v;
    e.acc0[row] = in.s0 + e.wacc * (S)in.a;
  }
}

// B: entries per lane whose loads and gathers are in flight together (8 where each
// thread has 128 registers, 4 where it has 64 or 80)
template <class T, int NT, int B, int EPI, class IDX>
__device__ __forceinline__ void cta_spmv_idx(const Mat<T>& M, const IDX* __restrict__ scol,
                                             const Epi<T>& e, typename Acc<T>::type& c0,
                                             typename Acc<T>::type& c1) {
  using A = typename Acc<T>::type;
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const T* src = e.src;
  const int64_t R0 = M.R0;
  const int64_t items = R0 + M.nslices;
  for (int64_t it = w; it < items; it += NW) {
    if (it >= R0) {
      const int64_t sl = it - R0;
      const int64_t row = R0 + 32 * sl + lane;
      const bool own = row < M.rows;
      EpiIn<T> ein{};
      if (own) ein = epi_load<T, EPI>(e, row);
      const int L = M.slice_len[sl];
      const IDX* __restrict__ cp = scol + M.slice_ptr[sl] + lane;
      const T* __restrict__ vp = M.sell_val + M.slice_ptr[sl] + lane;
      T acc_e = (T)0, acc_o = (T)0;
      for (int k0 = 0; k0 < L; k0 += B) {
        int cr[B];
        T vr[B], xr[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const bool in = k0 + u < L;
          cr[u] = in ? (int)__ldcs(cp + 32 * (k0 + u)) : 0;
          vr[u] = in ? __ldcs(vp + 32 * (k0 + u)) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) xr[u] = (k0 + u < L) ? src[cr[u]] : (T)0;
#pragma unroll
        for (int u = 0; u < B; ++u) {
          if (k0 + u < L) {
            if (u & 1)
              acc_o = fma(vr[u], xr[u], acc_o);
            else
              acc_e = fma(vr[u], xr[u], acc_e);
          }
        }
      }
      if (own) epilogue<T, EPI, A>(e, ein, row, acc_e + acc_o, c0, c1);
    } else {
      // a long row (CSR): lanes stride over its entries, then a fixed shuffle tree
      const int64_t row = it;
      const int64_t rb = M.row_ptr[row], re = M.row_ptr[row + 1];
      T acc = (T)0;
      for (int64_t p = rb + lane; p < re; p += 32) acc = fma(__ldcs(M.val + p), src[__ldcs(M.col + p)], acc);
      double sum = (double)acc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) epilogue<T, EPI, A>(e, epi_load<T, EPI>(e, row), row, (T)sum, c0, c1);
    }
  }
}

// A product with 16-bit column indices when the LP has them (a quarter less matrix
// traffic), else 32-bit ones.
template <class T, int NT, int B, int EPI>
__device__ __forceinline__ void cta_spmv(const Mat<T>& M, const uint16_t* col16, const Epi<T>& e,
                                         typename Acc<T>::type& c0, typename Acc<T>::type& c1) {
  if (col16)
    cta_spmv_idx<T, NT, B, EPI, uint16_t>(M, col16, e, c0, c1);
  else
    cta_spmv_idx<T, NT, B, EPI, int32_t>(M, M.sell_col, e, c0, c1);
}

// ---------------------------------------------------------------------------
// optimality measures of a point (x~, y~, A~x~, A~'y~) on the unscaled LP
// ---------------------------------------------------------------------------
template <class T>
struct Pt {
  const T* x;
  const T* y;
  const T* ax;
  const T* aty;
};

template <class T, int NT>
__device__ __noinline__ void cta_kkt(const BatchLP<T>& L, const BatchParams& P, const Pt<T>& z, Sh<T>& sh) {
  const OrigVecs& o = L.o;
  double v[5] = {0, 0, 0, 0, 0};  // pres2, dres2, pobj, dobj_rows, dobj_cols
  double mx[4] = {0, 0, 0, 0};     // l_inf residuals; scaled by Eq. (10)'s q_i, w_j
  const bool scaled = P.termination_mode == 2;
  for (int64_t i = threadIdx.x; i < L.m; i += NT) {
    const double ax = (double)z.ax[i] * o.inv_d1[i];
    const double y = (double)z.y[i] * o.d1[i];
    const double lc = o.lc[i], uc = o.uc[i];
    const double pr = ax - fmin(fmax(ax, lc), uc);
    v[0] += pr * pr;
    mx[0] = fmax(mx[0], fabs(pr));
    if (scaled) {
      const bool lq = isfinite(lc) && lc != 0.0, uq = isfinite(uc) && uc != 0.0;
      const double q = lq ? (uq ? fmax(fabs(lc), fabs(uc)) : fabs(lc)) : (uq ? fabs(uc) : 1.0);
      mx[2] = fmax(mx[2], fabs(pr) / q);
    }
    if (y > 0.0)
      v[3] += lc * y;
    else if (y < 0.0)
      v[3] += uc * y;
  }
  for (int64_t j = threadIdx.x; j < L.n; j += NT) {
    const double x = (double)z.x[j] * o.d2[j];
    const double aty = (double)z.aty[j] * o.inv_d2[j];
    const double cj = o.c[j], lv = o.lv[j], uv = o.uv[j];
    const double g = cj - aty;
    double r;
    if (P.reduced_costs == 1) {
      const bool near_lo = x - lv <= fabs(x), near_hi = uv - x <= fabs(x);
      r = (g > 0.0 && near_lo) ? g : ((g < 0.0 && near_hi) ? g : 0.0);
    } else {
      const bool lf = isfinite(lv), uf = isfinite(uv);
      r = g;
      if (lf && !uf) r = fmax(g, 0.0);
      if (!lf && uf) r = fmin(g, 0.0);
      if (!lf && !uf) r = 0.0;
    }
    const double dr = g - r;
    v[1] += dr * dr;
    mx[1] = fmax(mx[1], fabs(dr));
    if (scaled) mx[3] = fmax(mx[3], fabs(dr) / (cj != 0.0 ? fabs(cj) : 1.0));
    v[2] += cj * x;
    if (r > 0.0)
      v[4] += lv * r;
    else if (r < 0.0)
      v[4] += uv * r;
  }
  cta_sum<NT, 5>(v, sh);
  double tot[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) tot[q] = sh.out[q];
  cta_max<NT, 4>(mx, sh);
  if (threadIdx.x == 0) {
    Kkt& r = sh.kk;
    r.pres2 = sqrt(tot[0]);
    r.dres2 = sqrt(tot[1]);
    r.pres_inf = sh.out[0];
    r.dres_inf = sh.out[1];
    r.pres_rel_inf = sh.out[2];
    r.dres_rel_inf = sh.out[3];
    r.pobj = tot[2];
    r.dobj = tot[3] + tot[4];
    r.rel_primal = r.pres2 / (1.0 + L.b_norm);
    r.rel_dual = r.dres2 / (1.0 + L.c_norm);
    r.rel_gap = fabs(r.pobj - r.dobj) / (1.0 + fabs(r.pobj) + fabs(r.dobj));
    r.rel_kkt = fmax(r.rel_primal, fmax(r.rel_dual, r.rel_gap));
    const double den = fabs(r.pobj) + fabs(r.dobj);
    r.paper_gap = den > 0.0 ? fabs(r.pobj - r.dobj) / den : 0.0;
  }
  __syncthreads();
}

// the termination criteria in force (relative KKT, Eq. (9) or Eq. (10))
__device__ __forceinline__ bool converged(const Kkt& r, const BatchParams& p) {
  if (p.termination_mode == 0) return r.rel_kkt <= p.eps_rel_kkt;
  const double pr = p.termination_mode == 2 ? r.pres_rel_inf : r.pres_inf;
  const double du = p.termination_mode == 2 ? r.dres_rel_inf : r.dres_inf;
  return pr <= p.eps_abs_feas && du <= p.eps_abs_feas && r.paper_gap <= p.eps_rel_gap;
}

// ---------------------------------------------------------------------------
// normalized duality gap mu(z, z_ref) (Sec. 3), by the method of gap.cu: an FP64 pass
// for r and the saturated limit, FP32 bracket scans of the squared distance along the
// maximiser's path, an exact FP64 pass at the bracket, and a sort of the breakpoints
// inside it; FP64 scans when the FP32 bracket is rejected
// ---------------------------------------------------------------------------
template <class T, int NT>
__device__ void gap_pass0(const BatchLP<T>& L, const Pt<T>& z, const T* xr, const T* yr,
                          Sh<T>& sh) {
  const double om = sh.g_om, iom = 1.0 / om;
  double v[6] = {0, 0, 0, 0, 0, 0};
  float slope = 0.0f;
  const float iomf = (float)iom, omf = (float)om;
  for (int64_t j = threadIdx.x; j < L.n; j += NT) {
    const double x = z.x[j];
    const double dx = x - (double)xr[j];
    v[0] = fma(dx, dx, v[0]);
    const XPath q = x_path(x, L.c[j], z.aty[j], L.lv[j], L.uv[j]);
    // FP32 scan parameters (|g|, omega room, omega room^2; |g| = 0: does not move),
    // computed in FP64 first so that a small reduced cost keeps its digits
    const double orm = om * q.room;
    const float gaf = q.moves ? (float)q.ga : 0.0f, ormf = (float)orm;
    L.gp_x[j] = gaf;
    L.gp_x[L.n + j] = ormf;
    L.gp_x[2 * L.n + j] = ormf * (float)q.room;
    if (!q.moves) continue;
    if (q.room > 0.0) slope = fmaf(gaf * gaf, iomf, slope);
    if (isinf(q.room)) {
      v[4] += 1.0;
      continue;
    }
    v[2] = fma(om * q.room, q.room, v[2]);
    v[3] = fma(q.ga, q.room, v[3]);
  }
  for (int64_t i = threadIdx.x; i < L.m; i += NT) {
    const double y = z.y[i];
    const double dy = y - (double)yr[i];
    v[1] = fma(dy, dy, v[1]);
    const YPath q = y_path(y, L.lc[i], L.uc[i], z.ax[i]);
    // per row (omega |k1|, omega |k2|, |y|, y^2 / omega): omega |k1| = 0 for a fixed row,
    // |y| = +inf for a row that moves away forever, omega |k2| = 0 without a third piece
    const float yf = (float)q.y;
    const float w1 = omf * fabsf((float)q.k1);
    float4 prm;
    prm.x = q.kind == 0 ? 0.0f : w1;
    prm.y = q.kind == 3 ? omf * fabsf((float)q.k2) : 0.0f;
    prm.z = q.kind == 1 ? INFINITY : fabsf(yf);
    prm.w = yf * yf * iomf;
    L.gp_row[i] = prm;
    if (q.kind == 0) continue;
    slope = fmaf(w1, fabsf((float)q.k1), slope);
    if (q.kind == 1 || q.kind == 3) {
      v[4] += 1.0;
      continue;
    }
    v[2] = fma(q.y * q.y, iom, v[2]);
    v[3] = fma(-q.k1, q.y, v[3]);
  }
  v[5] = (double)slope;
  cta_sum<NT, 6>(v, sh);
  if (threadIdx.x == 0) {
    const double* t = sh.out;
    sh.g_r2 = om * t[0] + t[1] / om;
    sh.g_r = sqrt(sh.g_r2);
    sh.g_slope2 = t[5];
    sh.g_dinf2 = t[2];
    sh.g_finf = t[3];
    const bool unb = t[4] > 0.0;
    if (sh.g_r2 == 0.0) {
      sh.g_mu = 0.0;
      sh.g_state = kGDone;
    } else if (!unb && sh.g_dinf2 <= sh.g_r2 * (1.0 + 1e-12)) {
      sh.g_mu = sh.g_finf / sh.g_r;  // the fully saturated point lies inside the ball
      sh.g_state = kGDone;
    } else if (!(sh.g_slope2 > 0.0)) {
      sh.g_mu = 0.0;
      sh.g_state = kGDone;
    } else {
      // r / slope bounds the crossing from below; the slope is an FP32 sum: back off
      sh.g_slb = (1.0 - 1e-4) * sh.g_r / sqrt(sh.g_slope2);
      sh.g_sbase = sh.g_slb;
      sh.g_plan = kGeo;
      sh.g_state = kGActive;
    }
  }
  __syncthreads();
}

// new bracket from the squared distances at the scan points (thread 0)
template <class T>
__device__ void gap_bracket(Sh<T>& sh, const double* d2, int plan, int widen) {
  int first = -1;
  for (int q = 0; q < kQ; ++q)
    if (d2[q] >= sh.g_r2) {
      first = q;
      break;
    }
  if (plan == kGeo) {
    if (first < 0) {
      sh.g_sbase = ldexp(sh.g_sbase, kQ - 1);
      sh.g_state = kGNeedMore;
      return;
    }
    if (first == 0) {
      sh.g_sbase = ldexp(sh.g_sbase, -(kQ - 1));
      sh.g_state = kGNeedMore;
      return;
    }
    sh.g_slo = sh.s_pts[first - 1];
    sh.g_shi = sh.s_pts[first];
    sh.g_plan = kLin;
  } else {
    int lo_i = (first < 0 ? kQ : first) - 1;
    int hi_i = lo_i + 1;
    if (widen) {
      lo_i -= 1;
      hi_i += 1;
    }
    const double nlo = lo_i < 0 ? sh.g_slo : sh.s_pts[lo_i];
    const double nhi = hi_i >= kQ ? sh.g_shi : sh.s_pts[hi_i];
    sh.g_slo = nlo;
    sh.g_shi = nhi;
  }
}

// the plan's kQ points into shared memory (threads < kQ)
template <class T>
__device__ __forceinline__ void gap_points(Sh<T>& sh, int plan) {
  if (threadIdx.x < kQ) {
    const int q = threadIdx.x;
    sh.s_pts[q] = plan == kGeo ? ldexp(sh.g_sbase, q - kQ / 2)
                               : sh.g_slo + (sh.g_shi - sh.g_slo) * (double)(q + 1) / (double)(kQ + 1);
  }
  __syncthreads();
}

// squared distance at kQ points in FP32, from the parameters pass 0 wrote
template <class T, int NT>
__device__ void gap_scan32(const BatchLP<T>& L, Sh<T>& sh, int plan, int widen) {
  gap_points(sh, plan);
  const float iom = (float)(1.0 / sh.g_om);
  float pts[kQ], acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    pts[q] = (float)sh.s_pts[q];
    acc[q] = 0.0f;
  }
  const int64_t n = L.n;
  for (int64_t j = threadIdx.x; j < n; j += NT) {
    const float ga = L.gp_x[j];
    if (ga == 0.0f) continue;
    const float orm = L.gp_x[n + j], sat = L.gp_x[2 * n + j];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const float t = pts[q] * ga;
      acc[q] += (t < orm) ? t * t * iom : sat;
    }
  }
  for (int64_t i = threadIdx.x; i < L.m; i += NT) {
    const float4 prm = L.gp_row[i];
    if (prm.x == 0.0f) continue;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const float t1 = pts[q] * prm.x;
      float v;
      if (t1 < prm.z) {
        v = t1 * t1 * iom;
      } else {
        const float t2 = pts[q] * prm.y;
        v = (prm.y > 0.0f && t2 >= prm.z) ? t2 * t2 * iom : prm.w;
      }
      acc[q] += v;
    }
  }
  cta_sum<NT, kQ>(acc, sh);
  if (threadIdx.x == 0) gap_bracket(sh, sh.out, plan, widen);
  __syncthreads();
}

// the same in FP64 with the paths recomputed from the vectors (the fallback when the
// FP32 bracket is rejected); the points are read from shared memory
template <class T, int NT>
__device__ void gap_scan64(const BatchLP<T>& L, const Pt<T>& z, Sh<T>& sh, int plan, int widen) {
  gap_points(sh, plan);
  const double om = sh.g_om, iom = 1.0 / om;
  double acc[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
  for (int64_t j = threadIdx.x; j < L.n; j += NT) {
    const XPath p = x_path(z.x[j], L.c[j], z.aty[j], L.lv[j], L.uv[j]);
    if (!p.moves) continue;
    const double orm = om * p.room, sat = orm * p.room;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const double t = sh.s_pts[q] * p.ga;
      acc[q] += (t < orm) ? t * t * iom : sat;
    }
  }
  for (int64_t i = threadIdx.x; i < L.m; i += NT) {
    const YPath p = y_path(z.y[i], L.lc[i], L.uc[i], z.ax[i]);
    if (p.kind == 0) continue;
    const double w1 = om * fabs(p.k1), w2 = om * fabs(p.k2), ay = fabs(p.y);
    const double y2 = p.y * p.y * iom;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const double t1 = sh.s_pts[q] * w1;
      double v;
      if (p.kind == 1 || t1 < ay) {
        v = t1 * t1 * iom;
      } else {
        const double t2 = sh.s_pts[q] * w2;
        v = (p.kind == 3 && t2 >= ay) ? t2 * t2 * iom : y2;
      }
      acc[q] += v;
    }
  }
  cta_sum<NT, kQ>(acc, sh);
  if (threadIdx.x == 0) gap_bracket(sh, sh.out, plan, widen);
  __syncthreads();
}

// exact FP64 coefficients at s_lo and the breakpoints in (s_lo, s_hi] into shared memory
template <class T, int NT>
__device__ void gap_exact(const BatchLP<T>& L, const Pt<T>& z, Sh<T>& sh, double* keys,
                          long long* codes) {
  if (threadIdx.x == 0) sh.ncand = 0;
  __syncthreads();
  const double om = sh.g_om, iom = 1.0 / om, slo = sh.g_slo, shi = sh.g_shi;
  double v[4] = {0, 0, 0, 0};
  double bp, d4[4];
  for (int64_t j = threadIdx.x; j < L.n; j += NT) {
    const XPath q = x_path(z.x[j], L.c[j], z.aty[j], L.lv[j], L.uv[j]);
    if (!q.moves) continue;
    x_coef(q, slo, om, iom, v);
    const double orm = om * q.room;
    if (slo * q.ga < orm && orm <= shi * q.ga) {
      const int k = atomicAdd(&sh.ncand, 1);
      if (k < kCap) {
        x_cand(q, om, &bp, d4);
        keys[k] = bp;
        codes[k] = (long long)j * 4;
      }
    }
  }
  for (int64_t i = threadIdx.x; i < L.m; i += NT) {
    const YPath q = y_path(z.y[i], L.lc[i], L.uc[i], z.ax[i]);
    if (q.kind == 0) continue;
    y_coef(q, slo, om, iom, v);
    if (q.kind == 1) continue;
    const double ay = fabs(q.y);
    const double w1 = om * fabs(q.k1);
    if (slo * w1 < ay && ay <= shi * w1) {
      const int k = atomicAdd(&sh.ncand, 1);
      if (k < kCap) {
        y_cand(q, 1, om, &bp, d4);
        keys[k] = bp;
        codes[k] = (long long)i * 4 + 1;
      }
    }
    if (q.kind == 3) {
      const double w2 = om * fabs(q.k2);
      if (slo * w2 < ay && ay <= shi * w2) {
        const int k = atomicAdd(&sh.ncand, 1);
        if (k < kCap) {
          y_cand(q, 2, om, &bp, d4);
          keys[k] = bp;
          codes[k] = (long long)i * 4 + 2;
        }
      }
    }
  }
  cta_sum<NT, 4>(v, sh);
  if (threadIdx.x == 0) {
    sh.g_alpha = sh.out[0];
    sh.g_gamma = sh.out[1];
    sh.g_beta = sh.out[2];
    sh.g_phi = sh.out[3];
    const double d2lo = sh.g_alpha * slo * slo + sh.g_gamma;
    // the crossing must not lie left of the bracket (up to rounding)
    if (!(d2lo < sh.g_r2 * (1.0 + 1e-12)) || sh.ncand > kCap) sh.g_state = kGFailed;
  }
  __syncthreads();
}

template <class T>
__device__ __forceinline__ void cand_d4(const BatchLP<T>& L, const Pt<T>& z, double om,
                                        long long code, double* d4) {
  const int64_t idx = code >> 2;
  const int which = (int)(code & 3);
  double bp;
  if (which == 0)
    x_cand(x_path(z.x[idx], L.c[idx], z.aty[idx], L.lv[idx], L.uv[idx]), om, &bp, d4);
  else
    y_cand(y_path(z.y[idx], L.lc[idx], L.uc[idx], z.ax[idx]), which, om, &bp, d4);
}

// sort the breakpoints, prefix-sum their coefficient changes, find the piece where
// alpha s^2 + gamma reaches r^2 and solve there
template <class T, int NT>
__device__ void gap_finish(const BatchLP<T>& L, const Pt<T>& z, Sh<T>& sh, double* keys,
                           long long* codes) {
  constexpr int IT = (kCap + NT - 1) / NT;  // items per thread
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nc = sh.ncand;
  int P = 2;
  while (P < nc) P <<= 1;
  for (int i = nc + tid; i < P; i += NT) {
    keys[i] = INFINITY;
    codes[i] = LLONG_MAX;
  }
  if (tid == 0) sh.first = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += NT) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const double ki = keys[i], kl = keys[l];
          const long long ci = codes[i], cl = codes[l];
          const bool gt = (ki > kl) || (ki == kl && ci > cl);
          if (gt == up) {
            keys[i] = kl;
            keys[l] = ki;
            codes[i] = cl;
            codes[l] = ci;
          }
        }
      }
      __syncthreads();
    }
  }
  const double om = sh.g_om;
  const bool active = w * 32 * IT < nc;  // warp-uniform
  double dl[IT][4];
  double run[4] = {0, 0, 0, 0};
  double off[4] = {0, 0, 0, 0};
  if (active) {
    for (int q = 0; q < IT; ++q) {
      const int i = tid * IT + q;
      double d4[4] = {0, 0, 0, 0};
      if (i < nc) cand_d4(L, z, om, codes[i], d4);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        dl[q][k] = run[k];
        run[k] += d4[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double inc = run[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) sh.woff[k][w] = inc;
      off[k] = inc - run[k];
    }
  }
  __syncthreads();
  if (w == 0) {
    // exclusive prefix of the warp totals (warps past the candidates hold 0)
    const int nact = (nc + 32 * IT - 1) / (32 * IT);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double mine = lane < nact ? sh.woff[k][lane] : 0.0;
      double inc = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const double tot = __shfl_sync(0xffffffffu, inc, 31);
      __syncwarp();
      sh.woff[k][lane] = inc - mine;
      if (lane == 0) sh.tot[k] = tot;
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < 4; ++k) off[k] += sh.woff[k][w];
    const double al0 = sh.g_alpha, ga0 = sh.g_gamma, r2 = sh.g_r2;
    for (int q = 0; q < IT; ++q) {
      const int i = tid * IT + q;
      if (i >= nc) break;
      const double al = al0 + (off[0] + dl[q][0]);
      const double gm = ga0 + (off[1] + dl[q][1]);
      const double b = keys[i];
      if (al * b * b + gm >= r2) {
        atomicMin(&sh.first, i);
        break;
      }
    }
  }
  __syncthreads();
  const int first = sh.first;
  if (active && first != INT_MAX && tid == first / IT) {
    const int q = first - tid * IT;
#pragma unroll
    for (int k = 0; k < 4; ++k) sh.coef[k] = off[k] + dl[q][k];
  }
  __syncthreads();
  if (tid == 0) {
    const double r2 = sh.g_r2;
    // verify the right end of the bracket
    const double a_hi = sh.g_alpha + sh.tot[0], g_hi = sh.g_gamma + sh.tot[1];
    const double d2hi = a_hi * sh.g_shi * sh.g_shi + g_hi;
    if (first == INT_MAX && !(d2hi >= r2 * (1.0 - 1e-12))) {
      sh.g_state = kGFailed;
    } else {
      double cf[4], lo_b, hi_b;
      if (first == INT_MAX) {
        for (int k = 0; k < 4; ++k) cf[k] = sh.tot[k];
        lo_b = nc > 0 ? keys[nc - 1] : sh.g_slo;
        hi_b = sh.g_shi;
      } else {
        for (int k = 0; k < 4; ++k) cf[k] = sh.coef[k];
        lo_b = first == 0 ? sh.g_slo : keys[first - 1];
        hi_b = keys[first];
      }
      const double al = sh.g_alpha + cf[0], gm = sh.g_gamma + cf[1];
      const double be = sh.g_beta + cf[2], ph = sh.g_phi + cf[3];
      double s_star = lo_b;
      if (al > 0.0) s_star = sqrt(fmax(r2 - gm, 0.0) / al);
      s_star = fmin(fmax(s_star, lo_b), hi_b);
      sh.g_mu = (be * s_star + ph) / sh.g_r;
      sh.g_state = kGDone;
    }
  }
  __syncthreads();
}

template <class T, int NT>
__device__ __noinline__ double cta_gap(const BatchLP<T>& L, const Pt<T>& z, const T* xr, const T* yr,
                          double omega, Sh<T>& sh, unsigned char* dsm) {
  double* keys = reinterpret_cast<double*>(dsm);
  long long* codes = reinterpret_cast<long long*>(dsm + sizeof(double) * kCap);
  if (threadIdx.x == 0) {
    sh.g_om = omega;
    sh.gap_evals++;
  }
  __syncthreads();
  gap_pass0<T, NT>(L, z, xr, yr, sh);
  if (sh.g_state == kGDone) return sh.g_mu;
  // FP32 bracket: a geometric window moved until it holds the crossing, then three
  // linear refinements
  for (int rep = 0; rep < 8; ++rep) {
    gap_scan32<T, NT>(L, sh, kGeo, 0);
    if (sh.g_state != kGNeedMore) break;
    __syncthreads();
    if (threadIdx.x == 0) sh.g_state = kGActive;
    __syncthreads();
  }
  if (sh.g_state == kGActive) {
    gap_scan32<T, NT>(L, sh, kLin, 0);
    gap_scan32<T, NT>(L, sh, kLin, 0);
    gap_scan32<T, NT>(L, sh, kLin, 1);
    gap_exact<T, NT>(L, z, sh, keys, codes);
    if (sh.g_state == kGActive) gap_finish<T, NT>(L, z, sh, keys, codes);
  }
  if (sh.g_state == kGDone) return sh.g_mu;
  // FP64 scans: a geometric window from the lower bound, then linear refinement until
  // the exact pass accepts the bracket
  __syncthreads();
  if (threadIdx.x == 0) sh.gap_fallbacks++;
  for (int rep = 0; rep < 64; ++rep) {
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.g_state = kGActive;
      sh.g_plan = kGeo;
      if (rep == 0) sh.g_sbase = sh.g_slb;
    }
    __syncthreads();
    gap_scan64<T, NT>(L, z, sh, kGeo, 0);
    if (sh.g_state != kGNeedMore) break;
  }
  for (int rep = 0; rep < 80 && sh.g_state == kGActive; ++rep) {
    gap_exact<T, NT>(L, z, sh, keys, codes);
    if (sh.g_state == kGActive) gap_finish<T, NT>(L, z, sh, keys, codes);
    if (sh.g_state == kGDone) break;
    __syncthreads();
    if (sh.g_shi - sh.g_slo <= 1e-15 * sh.g_shi) {
      __syncthreads();
      if (threadIdx.x == 0) {
        sh.g_mu = (sh.g_beta * sh.g_slo + sh.g_phi) / sh.g_r;
        sh.g_state = kGDone;
      }
      __syncthreads();
      break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.g_state = kGActive;
      sh.g_plan = kLin;
    }
    __syncthreads();
    gap_scan64<T, NT>(L, z, sh, kLin, 1);
  }
  __syncthreads();
  double mu = sh.g_mu;
  if (sh.g_state != kGDone) {
    mu = NAN;
    __syncthreads();
    if (threadIdx.x == 0) sh.gap_failures++;
  }
  __syncthreads();
  return mu;
}

// ---------------------------------------------------------------------------
// infeasibility detection (Sec. 3, App. C) on three candidate directions
// ---------------------------------------------------------------------------
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
__device__ __forceinline__ double proj_sbar(double v, bool lf, bool uf) {
  if (lf && uf) return 0.0;
  if (uf) return fmax(v, 0.0);
  if (lf) return fmin(v, 0.0);
  return v;
}

// Returns 0, PDLP_PRIMAL_INFEASIBLE or PDLP_DUAL_INFEASIBLE; sh.flag = candidate index.
template <class T, int NT, int B>
__device__ __noinline__ int cta_infeas(const BatchLP<T>& L, const BatchParams& P, Sh<T>& sh) {
  const OrigVecs& o = L.o;
  const int64_t m = L.m, n = L.n;
  const int cur = sh.cur;
  const T* y = L.Y[cur];
  const T* yp = L.Y[cur ^ 1];
  const T* x = L.X[cur];
  const T* xp = L.X[cur ^ 1];
  for (int64_t i = threadIdx.x; i < m; i += NT) {
    const bool lf = isfinite(o.lc[i]), uf = isfinite(o.uc[i]);
    L.yd[i] = (T)proj_y((double)y[i] - (double)yp[i], lf, uf);
  }
  double v3[3] = {0, 0, 0};
  for (int64_t j = threadIdx.x; j < n; j += NT) {
    const bool lf = isfinite(o.lv[j]), uf = isfinite(o.uv[j]);
    const T a = (T)proj_xbar((double)x[j] - (double)xp[j], lf, uf);
    const T b = (T)proj_xbar((double)x[j], lf, uf);
    const T c = (T)proj_xbar((double)L.Xa[j], lf, uf);
    L.xb[j] = a;
    L.xb[n + j] = b;
    L.xb[2 * n + j] = c;
    const double wgt = o.c[j] * o.d2[j];
    v3[0] += wgt * (double)a;
    v3[1] += wgt * (double)b;
    v3[2] += wgt * (double)c;
  }
  cta_sum<NT, 3>(v3, sh);
  double cx[3] = {sh.out[0], sh.out[1], sh.out[2]};
  using A = typename Acc<T>::type;
  A u0 = (A)0, u1 = (A)0;
  Epi<T> e{};
  e.src = L.yd;
  e.out0 = L.atyd;
  cta_spmv<T, NT, B, kEpPlain>(L.AT, L.at_col16, e, u0, u1);
  unsigned xmask = 0;
  for (int c = 0; c < 3; ++c) {
    if (!(cx[c] < 0.0)) continue;
    e.src = L.xb + c * n;
    e.out0 = L.axb + c * m;
    cta_spmv<T, NT, B, kEpPlain>(L.A, L.a_col16, e, u0, u1);
    xmask |= 1u << c;
  }
  __syncthreads();
  const T* yc[3] = {L.yd, y, L.Ya};
  const T* atyc[3] = {L.atyd, L.ATY[cur], L.ATYa};
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double mx[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < m; i += NT) {
    const double l = o.lc[i], u = o.uc[i];
    const bool lf = isfinite(l), uf = isfinite(u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double yy = (double)yc[c][i] * o.d1[i];
      if (yy > 0.0)
        v[c] += l * yy;
      else if (yy < 0.0)
        v[c] += u * yy;
      if (xmask & (1u << c)) {
        const double p = (double)L.axb[c * m + i] * o.inv_d1[i];
        mx[3 + c] = fmax(mx[3 + c], fabs(p + proj_sbar(-p, lf, uf)));
      }
    }
  }
  for (int64_t j = threadIdx.x; j < n; j += NT) {
    const double l = o.lv[j], u = o.uv[j];
    const bool lf = isfinite(l), uf = isfinite(u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double q = (double)atyc[c][j] * o.inv_d2[j];
      const double r = proj_y(-q, lf, uf);  // proj_R has the sign sets of proj_Y
      mx[c] = fmax(mx[c], fabs(q + r));
      if (r > 0.0)
        v[3 + c] += l * r;
      else if (r < 0.0)
        v[3 + c] += u * r;
      v[6 + c] += o.c[j] * ((double)L.xb[c * n + j] * o.d2[j]);
    }
  }
  cta_sum<NT, 9>(v, sh);
  double tot[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) tot[q] = sh.out[q];
  cta_max<NT, 6>(mx, sh);
  if (threadIdx.x == 0) {
    const double eps = P.eps_infeas;
    int res = 0, which = -1;
    for (int c = 0; c < 3 && !res; ++c) {
      const double yobj = tot[c] + tot[3 + c];
      if (yobj > 0.0 && sh.out[c] <= eps * yobj) {
        res = PDLP_PRIMAL_INFEASIBLE;
        which = c;
      }
    }
    for (int c = 0; c < 3 && !res; ++c) {
      const double xres = (xmask >> c) & 1u ? sh.out[3 + c] : INFINITY;
      if (tot[6 + c] < 0.0 && xres <= eps * fabs(tot[6 + c])) {
        res = PDLP_DUAL_INFEASIBLE;
        which = c;
      }
    }
    sh.im[0] = (double)res;
    sh.flag = which;
  }
  __syncthreads();
  return (int)sh.im[0];
}

// thread 0 adds the cycles since the last phase boundary to phase q's counter
template <class T>
__device__ __forceinline__ void batch_phase(Sh<T>& sh, int q) {
  if (threadIdx.x == 0) {
    const long long now = clock64();
    sh.cyc[q] += now - sh.mark;
    sh.mark = now;
  }
}

// One step attempt of Algorithm 1's inner loop (Eq. (3a); A x' with Eq. (3b); Algorithm 2
// on thread 0) and, when it is accepted, A'y' with the running sums.  A function of its
// own so that the hot loops get registers independently of the evaluation code around
// them.
template <class T, int NT, int B>
__device__ __noinline__ void step_attempt(const BatchLP<T>& L, const BatchParams& P, Sh<T>& sh,
                                          T* sx, T* sy) {
  using A = typename Acc<T>::type;
  const int64_t m = L.m, n = L.n;
  const int64_t period = P.check_period > 0 ? P.check_period : 1;
  const int cur = sh.cur, nx = cur ^ 1;
  {
    const T tau = sh.tau;
    const T* x = L.X[cur];
    const T* aty = L.ATY[cur];
    T* xn = L.X[nx];
    A dx2 = (A)0;
    for (int64_t j = threadIdx.x; j < n; j += NT) {
      const T xo = x[j];
      const T v = clampv<T>(xo - tau * (__ldg(L.c + j) - aty[j]), __ldg(L.lv + j), __ldg(L.uv + j));
      xn[j] = v;
      if (sx) sx[j] = v;
      const A d = (A)v - (A)xo;
      dx2 = fma(d, d, dx2);
    }
    __syncthreads();
    batch_phase(sh, 0);
    Epi<T> e{};
    e.src = sx ? sx : xn;
    e.out0 = L.AX[nx];
    e.out1 = L.Y[nx];
    e.stage1 = sy;
    e.in0 = L.AX[cur];
    e.in1 = L.Y[cur];
    e.lo = L.lc;
    e.hi = L.uc;
    e.sigma = sh.sigma;
    A c0 = (A)0, c1 = (A)0;
    cta_spmv<T, NT, B, kEpDual>(L.A, L.a_col16, e, c0, c1);
    A s3[3] = {dx2, c0, c1};
    cta_sum<NT, 3>(s3, sh);
  }
  if (threadIdx.x == 0) {
    // Algorithm 2 with the interaction taken in magnitude (Eq. (5) for K = -A)
    const double dx2 = sh.out[0], dy2 = sh.out[1], inter = sh.out[2];
    const double omega = sh.omega, eta = sh.eta;
    const double num = omega * dx2 + dy2 / omega;
    const double den = 2.0 * fabs(inter);
    const double eta_bar = den > 0.0 ? num / den : INFINITY;
    double red_f, grow_f;
    if (sh.k < P.step_len) {
      red_f = P.step_tab[2 * sh.k];
      grow_f = P.step_tab[2 * sh.k + 1];
    } else {
      const double kf = (double)(sh.k + 2);
      red_f = 1.0 - pow(kf, -0.3);
      grow_f = 1.0 + pow(kf, -0.6);
    }
    const bool fixed = P.fixed_step > 0.0;
    const double eta_new = fixed ? P.fixed_step : fmin(red_f * eta_bar, grow_f * eta);
    sh.attempts += 1;
    if (!(isfinite(eta_new) && isfinite(num))) {
      sh.err = 1;
      sh.accepted = 0;
    } else if (fixed || eta <= eta_bar) {
      sh.eta_acc = eta;
      sh.eta_hat = eta_new;
      sh.eta = eta_new;
      sh.cur = nx;
      sh.k += 1;
      sh.t += 1;
      sh.W += eta;
      sh.accepted = 1;
      sh.retries = 0;
      sh.wacc = (typename BatchSum<T>::type)eta;
      // evaluation points: checks, restart criterion (iii), the iteration limit
      const int64_t k = sh.k, t = sh.t;
      int ev = (k % period) == 0 ? 1 : 0;
      if ((double)t >= P.beta_art * (double)k) ev |= 2;
      if (k >= P.max_iters) ev |= 4;
      sh.ev = ev;
      if (ev) {
        sh.evaluations++;
        sh.winv = (typename BatchSum<T>::type)(1.0 / sh.W);
      }
    } else {
      sh.eta = eta_new;
      sh.accepted = 0;
      sh.retries += 1;
      sh.rejected += 1;
      if (sh.retries >= P.max_retries) sh.err = 2;
    }
    sh.tau = (T)(sh.eta / sh.omega);
    sh.sigma = (T)(sh.eta * sh.omega);
  }
  __syncthreads();
  batch_phase(sh, 1);
  if (sh.err || !sh.accepted) return;
  {
    // A'y' with the running sums of Algorithm 1 (the iterate just accepted is `nx`)
    using S = typename BatchSum<T>::type;
    const S wv = sh.wacc;
    const T* yn = sy ? sy : L.Y[nx];
    for (int64_t i = threadIdx.x; i < m; i += NT) L.Sy[i] = L.Sy[i] + wv * (S)yn[i];
    Epi<T> e{};
    e.src = yn;
    e.out0 = L.ATY[nx];
    e.in0 = sx ? sx : L.X[nx];
    e.acc0 = L.Sx;
    e.wacc = wv;
    A u0 = (A)0, u1 = (A)0;
    cta_spmv<T, NT, B, kEpAvg>(L.AT, L.at_col16, e, u0, u1);
    __syncthreads();
    batch_phase(sh, 2);
  }
}

// ---------------------------------------------------------------------------
// the whole method on one LP
// ---------------------------------------------------------------------------
template <class T, int NT, int B>
__device__ void solve_lp(const BatchLP<T>& L, const BatchParams& P, BatchResult* R, Sh<T>& sh,
                         unsigned char* dsm, int64_t stage_bytes) {
  using A = typename Acc<T>::type;
  const int64_t m = L.m, n = L.n;
  // gathered vectors staged in shared memory when they fit
  const size_t xb = sizeof(T) * (size_t)n, yb = sizeof(T) * (size_t)m;
  const size_t xb_al = (xb + 15) & ~(size_t)15;
  bool sx_on = false, sy_on = false;
  const size_t budget = (size_t)stage_bytes;
  if (budget) {
    if (xb_al + yb <= budget) {
      sx_on = true;
      sy_on = m > 0;
    } else if (xb <= budget) {
      sx_on = true;
    } else if (yb <= budget && m > 0) {
      sy_on = true;
    }
  }
  T* sx = sx_on ? reinterpret_cast<T*>(dsm) : nullptr;
  T* sy = sy_on ? reinterpret_cast<T*>(dsm + (sx_on ? xb_al : 0)) : nullptr;

  if (threadIdx.x == 0) {
    sh.k = sh.t = sh.attempts = sh.rejected = 0;
    sh.restarts[0] = sh.restarts[1] = sh.restarts[2] = 0;
    sh.evaluations = sh.gap_evals = sh.gap_fallbacks = sh.gap_failures = 0;
    sh.eta = P.fixed_step > 0.0 ? P.fixed_step : L.eta0;
    sh.eta_hat = sh.eta;
    sh.eta_acc = 0.0;
    sh.omega = P.fixed_omega > 0.0 ? P.fixed_omega : L.omega0;
    sh.W = 0.0;
    sh.mu_ref = 0.0;
    sh.mu_c_prev = INFINITY;
    sh.cur = 0;
    sh.accepted = 0;
    sh.retries = 0;
    sh.err = 0;
    sh.have_mu_ref = 0;
    sh.tau = (T)(sh.eta / sh.omega);
    sh.sigma = (T)(sh.eta * sh.omega);
    sh.t0 = global_ns();
    for (int q = 0; q < 8; ++q) sh.cyc[q] = 0;
    sh.mark = clock64();
  }

  // z^{0,0} = (proj_X(0), 0); sums 0
  for (int64_t j = threadIdx.x; j < n; j += NT) {
    const T lo = L.lv[j], hi = L.uv[j];
    const T v = (T)0 < lo ? lo : ((T)0 > hi ? hi : (T)0);
    L.X[0][j] = v;
    L.X0[j] = v;
    L.ATY[0][j] = (T)0;
    L.Sx[j] = 0;
  }
  for (int64_t i = threadIdx.x; i < m; i += NT) {
    L.Y[0][i] = (T)0;
    L.Y0[i] = (T)0;
    L.Sy[i] = 0;
  }
  __syncthreads();
  {
    A u0 = (A)0, u1 = (A)0;
    Epi<T> e{};
    e.src = L.X[0];
    e.out0 = L.AX[0];
    cta_spmv<T, NT, B, kEpPlain>(L.A, L.a_col16, e, u0, u1);
  }
  __syncthreads();

  int status = -1;
  int ray = 0;
  Pt<T> out{L.X[0], L.Y[0], L.AX[0], L.ATY[0]};
  // termination test on the start point
  cta_kkt<T, NT>(L, P, out, sh);
  if (converged(sh.kk, P)) status = PDLP_OPTIMAL;

  while (status < 0) {
    batch_phase(sh, 3);  // evaluation points (and the start) since the last boundary
    // ---- one step attempt ----
    step_attempt<T, NT, B>(L, P, sh, sx, sy);
    if (sh.err) {
      status = PDLP_NUMERICAL_ERROR;
      out = Pt<T>{L.X[sh.cur], L.Y[sh.cur], L.AX[sh.cur], L.ATY[sh.cur]};
      cta_kkt<T, NT>(L, P, out, sh);
      break;
    }
    if (!sh.accepted) continue;
    const int ev = sh.ev;
    if (!ev) continue;
    const bool is_check = ev & 1, is_art = (ev & 2) != 0, is_limit = (ev & 4) != 0;
    {
      // the average since the last restart (x kept inside [lv, uv])
      const auto wi = sh.winv;
      for (int64_t j = threadIdx.x; j < n; j += NT) {
        const T v = (T)(L.Sx[j] * wi);
        const T lo = L.lv[j], hi = L.uv[j];
        L.Xa[j] = v < lo ? lo : (v > hi ? hi : v);
      }
      for (int64_t i = threadIdx.x; i < m; i += NT) L.Ya[i] = (T)(L.Sy[i] * wi);
      __syncthreads();
      // A xbar and A'ybar by two products here rather than running sums of A x and A'y
      // updated every iteration (the same vectors by linearity, up to rounding): an
      // evaluation comes every few dozen iterations, the sums cost 16 (m + n) bytes each
      A u0 = (A)0, u1 = (A)0;
      Epi<T> e{};
      e.src = L.Xa;
      e.out0 = L.AXa;
      cta_spmv<T, NT, B, kEpPlain>(L.A, L.a_col16, e, u0, u1);
      e.src = L.Ya;
      e.out0 = L.ATYa;
      cta_spmv<T, NT, B, kEpPlain>(L.AT, L.at_col16, e, u0, u1);
      __syncthreads();
    }
    const int c2 = sh.cur;
    const Pt<T> zc{L.X[c2], L.Y[c2], L.AX[c2], L.ATY[c2]};
    const Pt<T> za{L.Xa, L.Ya, L.AXa, L.ATYa};
    batch_phase(sh, 3);
    const double mu_cur = cta_gap<T, NT>(L, zc, L.X0, L.Y0, sh.omega, sh, dsm);
    const double mu_avg = cta_gap<T, NT>(L, za, L.X0, L.Y0, sh.omega, sh, dsm);
    batch_phase(sh, 5);
    if (threadIdx.x == 0) {
      // GetRestartCandidate: the average unless the current iterate's gap is smaller
      const bool avg = !(mu_cur < mu_avg);
      sh.dec_avg = avg ? 1 : 0;
      sh.im[2] = avg ? mu_avg : mu_cur;
    }
    __syncthreads();
    const bool cand_avg = sh.dec_avg != 0;
    const Pt<T> cand = cand_avg ? za : zc;
    if (is_check || is_limit) {
      cta_kkt<T, NT>(L, P, cand, sh);
      batch_phase(sh, 6);
      if (threadIdx.x == 0) sh.dec_conv = converged(sh.kk, P) ? 1 : 0;
      __syncthreads();
      if (sh.dec_conv) {
        status = PDLP_OPTIMAL;
        out = cand;
        break;
      }
      if (P.detect_infeasibility) {
        const int inf = cta_infeas<T, NT, B>(L, P, sh);
        batch_phase(sh, 7);
        if (inf) {
          const int c = sh.flag;
          if (inf == PDLP_PRIMAL_INFEASIBLE) {
            const T* ys[3] = {L.yd, L.Y[c2], L.Ya};
            const T* atys[3] = {L.atyd, L.ATY[c2], L.ATYa};
            out = Pt<T>{L.X[c2], ys[c], L.AX[c2], atys[c]};
          } else {
            out = Pt<T>{L.xb + c * n, L.Y[c2], L.axb + c * m, L.ATY[c2]};
            ray = 1;
          }
          cta_kkt<T, NT>(L, P, out, sh);
          status = inf;
          break;
        }
      }
      if (is_limit) {
        status = PDLP_ITERATION_LIMIT;
        out = cand;
        break;
      }
      if (threadIdx.x == 0)
        sh.dec_time = (double)(global_ns() - sh.t0) * 1e-9 > P.time_limit_s ? 1 : 0;
      __syncthreads();
      if (sh.dec_time) {
        status = PDLP_TIME_LIMIT;
        out = cand;
        break;
      }
    }
    if (threadIdx.x == 0) {
      const double mu_c = sh.im[2];
      const int kind = restart_kind(is_check, is_art, sh.have_mu_ref != 0, mu_c, sh.mu_ref,
                                    sh.mu_c_prev, P.beta_suff, P.beta_nec);
      if (is_check) sh.mu_c_prev = mu_c;
      sh.flag = kind;
      if (kind) sh.restarts[kind - 1]++;
    }
    __syncthreads();
    if (sh.flag == 0) continue;
    // ---- restart the outer loop at the candidate (Algorithm 1), Algorithm 3 ----
    {
      T* x = L.X[c2];
      T* y = L.Y[c2];
      T* ax = L.AX[c2];
      T* aty = L.ATY[c2];
      double d[2] = {0.0, 0.0};
      for (int64_t j = threadIdx.x; j < n; j += NT) {
        if (cand_avg) {
          x[j] = L.Xa[j];
          aty[j] = L.ATYa[j];
        }
        const double dd = (double)x[j] - (double)L.X0[j];
        d[0] += dd * dd;
      }
      for (int64_t i = threadIdx.x; i < m; i += NT) {
        if (cand_avg) {
          y[i] = L.Ya[i];
          ax[i] = L.AXa[i];
        }
        const double dd = (double)y[i] - (double)L.Y0[i];
        d[1] += dd * dd;
      }
      cta_sum<NT, 2>(d, sh);
      if (threadIdx.x == 0) {
        const double dx = sqrt(sh.out[0]), dy = sqrt(sh.out[1]);
        const double om = P.fixed_omega > 0.0 ? P.fixed_omega
                                              : primal_weight(sh.omega, dx, dy, P.theta, P.eps_zero);
        sh.g_om = om;  // handed to the evaluation below
        sh.im[1] = om;
      }
      __syncthreads();
      const double om = sh.im[1];
      batch_phase(sh, 3);
      const double mu_ref = cta_gap<T, NT>(L, zc, L.X0, L.Y0, om, sh, dsm);
      batch_phase(sh, 5);
      for (int64_t j = threadIdx.x; j < n; j += NT) {
        L.X0[j] = x[j];
        L.Sx[j] = 0;
      }
      for (int64_t i = threadIdx.x; i < m; i += NT) {
        L.Y0[i] = y[i];
        L.Sy[i] = 0;
      }
      if (threadIdx.x == 0) {
        sh.mu_ref = mu_ref;
        sh.have_mu_ref = 1;
        sh.mu_c_prev = INFINITY;
        sh.omega = om;
        sh.W = 0.0;
        sh.t = 0;
        sh.tau = (T)(sh.eta / om);
        sh.sigma = (T)(sh.eta * om);
      }
      __syncthreads();
    }
  }

  // ---- output: x = D2 x~ (inside [lv, uv] unless it is a ray), y = D1 y~, in the
  // caller's numbering; statistics ----
  {
    const OrigVecs& o = L.o;
    for (int64_t j = threadIdx.x; j < n; j += NT) {
      const double v = o.d2[j] * (double)out.x[j];
      L.x_out[L.perm_c[j]] = ray ? v : fmin(fmax(v, o.lv[j]), o.uv[j]);
    }
    for (int64_t i = threadIdx.x; i < m; i += NT) L.y_out[L.perm_r[i]] = o.d1[i] * (double)out.y[i];
  }
  batch_phase(sh, 4);
  if (threadIdx.x == 0) {
    BatchResult r;
    for (int q = 0; q < 8; ++q) r.cycles[q] = sh.cyc[q];
    r.status = status;
    r.staged = (sx_on ? 1 : 0) | (sy_on ? 2 : 0);
    r.k = sh.k;
    r.attempts = sh.attempts;
    r.rejected = sh.rejected;
    for (int q = 0; q < 3; ++q) r.restarts[q] = sh.restarts[q];
    r.evaluations = sh.evaluations;
    r.gap_evals = sh.gap_evals;
    r.gap_fallbacks = sh.gap_fallbacks;
    r.gap_failures = sh.gap_failures;
    const Kkt& q = sh.kk;
    r.rel_kkt = q.rel_kkt;
    r.rel_primal = q.rel_primal;
    r.rel_dual = q.rel_dual;
    r.rel_gap = q.rel_gap;
    r.pres2 = q.pres2;
    r.dres2 = q.dres2;
    r.pres_inf = q.pres_inf;
    r.dres_inf = q.dres_inf;
    r.pobj = q.pobj;
    r.dobj = q.dobj;
    r.paper_gap = q.paper_gap;
    r.pres_rel_inf = q.pres_rel_inf;
    r.dres_rel_inf = q.dres_rel_inf;
    r.omega = sh.omega;
    r.eta_hat = sh.eta_hat;
    r.seconds = (double)(global_ns() - sh.t0) * 1e-9;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    r.sm = smid;
    *R = r;
  }
  __syncthreads();
}

template <class T, int NT, int PER_SM>
__global__ void __launch_bounds__(NT, PER_SM)
    k_batch(const BatchLP<T>* lps, const int32_t* order, int count, BatchParams prm,
            BatchResult* res, unsigned int* queue, int64_t stage_bytes) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ Sh<T> sh;
  __shared__ BatchLP<T> lp;
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int q = s_next;
    if (q >= count) break;
    const int idx = order[q];
    // the LP's descriptor, copied to shared memory word by word
    static_assert(sizeof(BatchLP<T>) % sizeof(int) == 0, "descriptor size");
    {
      const int words = (int)(sizeof(BatchLP<T>) / sizeof(int));
      const int* srcw = reinterpret_cast<const int*>(lps + idx);
      int* dstw = reinterpret_cast<int*>(&lp);
      for (int w = threadIdx.x; w < words; w += NT) dstw[w] = srcw[w];
    }
    __syncthreads();
    solve_lp<T, NT, (NT * PER_SM >= PDLP_BATCH_B_THRESHOLD ? PDLP_BATCH_B_SMALL_REGS : 8)>(lp, prm, res + idx, sh, dsm, stage_bytes);
  }
}

}  // namespace

template <class T, int NT, int PER_SM>
static int resident_impl(size_t smem) {
  static size_t set = 0;  // largest dynamic shared memory enabled so far
  if (smem > set) {
    PDLP_CUDA_CHECK(cudaFuncSetAttribute(k_batch<T, NT, PER_SM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    set = smem;
  }
  int occ = 0;
  PDLP_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<T, NT, PER_SM>, NT, smem));
  if (occ < 1) throw PdlpError(-3, "persistent batch kernel does not fit on an SM");
  return occ * num_sms();
}

template <class T>
static int resident_any(const BatchConfig& c) {
  const size_t smem = (size_t)c.smem_kb * 1024;
  if (c.threads == 1024) return resident_impl<T, 1024, 1>(smem);
  if (c.threads == 768) return resident_impl<T, 768, 1>(smem);
  if (c.per_sm == 2) return resident_impl<T, 512, 2>(smem);
  return resident_impl<T, 512, 1>(smem);
}

template <class T>
int batch_resident_ctas(int config) {
  if (config < 1 || config > kNumConfigs) throw PdlpError(-1, "unknown batch configuration");
  return resident_any<T>(kConfigs[config - 1]);
}

template <class T>
void launch_batch(const BatchLP<T>* lps, const int32_t* order, int count, const BatchParams& prm,
                  BatchResult* res, unsigned int* queue, int config, int ctas, cudaStream_t s) {
  if (config < 1 || config > kNumConfigs) throw PdlpError(-1, "unknown batch configuration");
  const BatchConfig& c = kConfigs[config - 1];
  resident_any<T>(c);
  const size_t smem = (size_t)c.smem_kb * 1024;
  const int64_t stage = c.stage ? (int64_t)smem : 0;
  if (c.threads == 1024)
    k_batch<T, 1024, 1><<<ctas, 1024, smem, s>>>(lps, order, count, prm, res, queue, stage);
  else if (c.threads == 768)
    k_batch<T, 768, 1><<<ctas, 768, smem, s>>>(lps, order, count, prm, res, queue, stage);
  else if (c.per_sm == 2)
    k_batch<T, 512, 2><<<ctas, 512, smem, s>>>(lps, order, count, prm, res, queue, stage);
  else
    k_batch<T, 512, 1><<<ctas, 512, smem, s>>>(lps, order, count, prm, res, queue, stage);
  PDLP_LAUNCH_CHECK();
}

}  // namespace pdlp
