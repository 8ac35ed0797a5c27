// Per-coordinate paths of the maximiser in the normalized duality gap (Sec. 3,
// "Adaptive restarts"), shared by the grid-wide kernels of gap.cu and the per-LP
// evaluation of the persistent batch kernel (batch_impl.cuh).
//
// For z = (x, y) and radius r,
//   r * rho_r(z) = max { L(x,yh) - L(xh,y) : zh in X x Y, ||zh - z||_omega <= r }.
// The objective is separable; with a multiplier on the ball, parametrised by s, every
// coordinate of the maximiser follows a path with at most three linear pieces (moving,
// parked at a bound or at 0, moving again), and along the path
//     ||zh(s) - z||_omega^2 = alpha(s) s^2 + gamma(s),   F(s) = beta(s) s + phi(s)
// with alpha, gamma, beta, phi piecewise constant, changing only at breakpoints.
#pragma once

#include <math.h>
#include <stdint.h>

namespace pdlp {

// Path of one column: g = c - A'y; it moves toward lv (g > 0) or uv (g < 0) at rate
// |g| / omega per unit s and parks after travelling `room`.
// The FP32 bracket scans of the batch kernel use the same paths in single precision
// (S = float); every exact step uses S = double.
template <class S>
struct XPathT {
  S g, ga, room;
  bool moves;
};
using XPath = XPathT<double>;
template <class S>
__device__ __forceinline__ XPathT<S> x_path_t(S x, S c, S aty, S lv, S uv) {
  XPathT<S> p;
  p.g = c - aty;
  p.ga = fabs(p.g);
  p.moves = p.g != (S)0;
  p.room = p.g > (S)0 ? x - lv : (p.g < (S)0 ? uv - x : (S)0);
  return p;
}
__device__ __forceinline__ XPath x_path(double x, double c, double aty, double lv, double uv) {
  return x_path_t<double>(x, c, aty, lv, uv);
}

// Path of one row (kind 0: fixed; 1: moves away forever with slope k1; 2: moves to 0
// with slope k1 and parks; 3: moves to 0, parks, then moves on with slope k2).
template <class S>
struct YPathT {
  S y, k1, k2;
  int kind;
};
using YPath = YPathT<double>;
template <class S>
__device__ __forceinline__ YPathT<S> y_path_t(S y, S lc, S uc, S ax) {
  YPathT<S> p;
  p.y = y;
  p.k1 = (S)0;
  p.k2 = (S)0;
  p.kind = 0;
  const bool lf = isfinite(lc), uf = isfinite(uc);
  const S a = lc - ax, b = uc - ax;
  if (y > (S)0) {
    if (a > (S)0) {
      p.kind = 1;
      p.k1 = a;
    } else if (a < (S)0) {
      p.k1 = a;
      if (uf && b < (S)0) {
        p.kind = 3;
        p.k2 = b;
      } else {
        p.kind = 2;
      }
    }
  } else if (y < (S)0) {
    if (b < (S)0) {
      p.kind = 1;
      p.k1 = b;
    } else if (b > (S)0) {
      p.k1 = b;
      if (lf && a > (S)0) {
        p.kind = 3;
        p.k2 = a;
      } else {
        p.kind = 2;
      }
    }
  } else {
    if (lf && a > (S)0) {
      p.kind = 1;
      p.k1 = a;
    } else if (uf && b < (S)0) {
      p.kind = 1;
      p.k1 = b;
    }
  }
  return p;
}
__device__ __forceinline__ YPath y_path(double y, double lc, double uc, double ax) {
  return y_path_t<double>(y, lc, uc, ax);
}

// Coefficients (alpha, gamma, beta, phi) of a column / row at s.
__device__ __forceinline__ void x_coef(const XPath& p, double s, double om, double iom,
                                       double* c4) {
  if (!p.moves) return;
  if (s * p.ga < om * p.room) {
    const double w = p.g * p.g * iom;
    c4[0] += w;
    c4[2] += w;
  } else {
    c4[1] += om * p.room * p.room;
    c4[3] += p.ga * p.room;
  }
}
__device__ __forceinline__ int y_piece(const YPath& p, double s, double om) {
  // 1 moving (first piece), 2 parked at 0, 3 moving again
  if (p.kind == 1) return 1;
  const double ay = fabs(p.y);
  if (s * (om * fabs(p.k1)) < ay) return 1;
  if (p.kind == 3 && s * (om * fabs(p.k2)) >= ay) return 3;
  return 2;
}
__device__ __forceinline__ void y_coef(const YPath& p, double s, double om, double iom,
                                       double* c4) {
  if (p.kind == 0) return;
  const int pc = y_piece(p, s, om);
  if (pc == 1) {
    const double w = om * p.k1 * p.k1;
    c4[0] += w;
    c4[2] += w;
  } else if (pc == 2) {
    c4[1] += p.y * p.y * iom;
    c4[3] += -p.k1 * p.y;
  } else {
    const double w = om * p.k2 * p.k2;
    c4[0] += w;
    c4[2] += w;
    c4[3] += (p.k2 - p.k1) * p.y;
  }
}

// Breakpoint of a column (where it parks) and the change of (alpha, gamma, beta, phi)
// there.
__device__ __forceinline__ void x_cand(const XPath& q, double om, double* bp, double* d4) {
  *bp = om * q.room / q.ga;
  const double w = q.g * q.g * (1.0 / om);
  d4[0] = -w;
  d4[1] = om * q.room * q.room;
  d4[2] = -w;
  d4[3] = q.ga * q.room;
}

// Breakpoint `which` of a row (1: it parks at 0; 2: it moves on along its third piece)
// and the coefficient change there.
__device__ __forceinline__ void y_cand(const YPath& q, int which, double om, double* bp,
                                       double* d4) {
  const double ay = fabs(q.y);
  if (which == 1) {
    *bp = ay / (om * fabs(q.k1));
    const double w = om * q.k1 * q.k1;
    d4[0] = -w;
    d4[1] = q.y * q.y * (1.0 / om);
    d4[2] = -w;
    d4[3] = -q.k1 * q.y;
  } else {
    *bp = ay / (om * fabs(q.k2));
    const double w = om * q.k2 * q.k2;
    d4[0] = w;
    d4[1] = -q.y * q.y * (1.0 / om);
    d4[2] = w;
    d4[3] = q.k2 * q.y;
  }
}

}  // namespace pdlp
