"""Independent reference computations used to pin the oracle.

Nothing here calls the oracle's arithmetic: each function restates a textbook
definition (vertex enumeration, the proximal operator as an explicit argmin, the
trust-region maximum by sorting breakpoints) so that an error in the oracle shows
up as a disagreement.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

import lpgen


def make_lp(A_dense, c, lc, uc, lv, uv, name="test") -> lpgen.LPInstance:
    A = sp.csr_matrix(np.asarray(A_dense, dtype=np.float64))
    A.sort_indices()
    m, n = A.shape
    return lpgen.LPInstance(
        m=m, n=n,
        row_ptr=A.indptr.astype(np.int64), col_idx=A.indices.astype(np.int32),
        val=A.data.astype(np.float64),
        c=np.asarray(c, float), lc=np.asarray(lc, float), uc=np.asarray(uc, float),
        lv=np.asarray(lv, float), uv=np.asarray(uv, float), name=name)


def random_bounded_lp(rng, m, n, density=0.7, eq_frac=0.3):
    """A small feasible LP with finite variable bounds (so it has an optimum)."""
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    x0 = rng.uniform(0, 4, n)
    ax0 = A @ x0
    lc = ax0 - rng.uniform(0, 1, m)
    uc = ax0 + rng.uniform(0, 1, m)
    neq = int(round(eq_frac * m))
    lc[:neq] = ax0[:neq]
    uc[:neq] = ax0[:neq]
    # a few one-sided / free rows
    if m >= 3:
        lc[m - 1] = -np.inf
        uc[m - 2] = np.inf
    return make_lp(A, rng.uniform(-1, 1, n), lc, uc, np.zeros(n), np.full(n, 4.0))


def brute_force_vertices(inst):
    """min c'x over the polytope by enumerating every vertex: choose n of the finite
    bound hyperplanes (row i at lc_i or uc_i, variable j at lv_j or uv_j), solve, keep
    the feasible solutions.  Only for n <= 6."""
    A = inst.scipy_csr().toarray()
    m, n = A.shape
    planes = []
    for i in range(m):
        for b in (inst.lc[i], inst.uc[i]):
            if np.isfinite(b):
                planes.append((A[i], b))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        for b in (inst.lv[j], inst.uv[j]):
            if np.isfinite(b):
                planes.append((e, b))
    best = math.inf
    best_x = None
    for combo in itertools.combinations(range(len(planes)), n):
        M = np.array([planes[k][0] for k in combo])
        rhs = np.array([planes[k][1] for k in combo])
        if abs(np.linalg.det(M)) < 1e-10:
            continue
        x = np.linalg.solve(M, rhs)
        ax = A @ x
        tol = 1e-8
        if np.all(ax >= inst.lc - tol) and np.all(ax <= inst.uc + tol) and \
                np.all(x >= inst.lv - tol) and np.all(x <= inst.uv + tol):
            v = float(inst.c @ x)
            if v < best:
                best, best_x = v, x
    return best, best_x


def prox_p_argmin(v, sigma, lc, uc):
    """prox of sigma*p(.; -uc, -lc) + indicator of Y, coordinate by coordinate, as the
    explicit argmin of  p(y) + (y - v)^2 / (2 sigma)  over the allowed signs:
    p(y; -uc, -lc) = -lc*y for y >= 0 and uc*(-y) for y <= 0 (Sec. 2's definition of
    p), so the stationary points are v + sigma*lc (on y >= 0, needs lc finite) and
    v + sigma*uc (on y <= 0, needs uc finite); 0 is always a candidate."""
    out = np.empty_like(v)
    for i in range(v.shape[0]):
        cands = [0.0]
        if np.isfinite(lc[i]):
            cands.append(max(0.0, v[i] + sigma * lc[i]))
        if np.isfinite(uc[i]):
            cands.append(min(0.0, v[i] + sigma * uc[i]))

        def obj(y):
            pv = 0.0
            if y > 0:
                pv = -lc[i] * y
            elif y < 0:
                pv = uc[i] * (-y)
            return pv + (y - v[i]) ** 2 / (2.0 * sigma)

        out[i] = min(cands, key=obj)
    return out


def _trial(lp, x, y, Ax, g, omega, s):
    lcf, ucf = np.isfinite(lp.lc), np.isfinite(lp.uc)
    xh = np.clip(x - s * g / omega, lp.lv, lp.uv)
    yh = np.zeros_like(y)
    for i in range(y.shape[0]):
        if lcf[i]:
            v = y[i] + s * omega * (lp.lc[i] - Ax[i])
            if v > 0:
                yh[i] = v
                continue
        if ucf[i]:
            v = y[i] + s * omega * (lp.uc[i] - Ax[i])
            if v < 0:
                yh[i] = v
    return xh, yh


def lagrangian(lp, x, y, Ax_of):
    """L(x, y) = c'x - y'Ax - p(y; -uc, -lc) with 0*inf = 0 (Sec. 2, Eq. (2))."""
    Ax = Ax_of(x)
    pv = 0.0
    for i in range(y.shape[0]):
        if y[i] > 0:
            pv += -lp.lc[i] * y[i]
        elif y[i] < 0:
            pv += lp.uc[i] * (-y[i])
    return float(lp.c @ x - y @ Ax - pv)


def exact_normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega):
    """The trust-region maximum of rho_r by sorting breakpoints instead of bisection:
    between consecutive breakpoints every coordinate of the maximiser moves affinely
    in s, so ||zh(s) - z||_omega^2 is an exact quadratic there; its root on the
    crossing interval gives s*, and the objective is evaluated from the Lagrangian
    definition directly (no shortcut formula)."""
    r = math.sqrt(omega * np.sum((x - xr) ** 2) + np.sum((y - yr) ** 2) / omega)
    if r == 0:
        return 0.0
    g = lp.c - ATy
    bps = set()
    for j in range(x.shape[0]):
        if g[j] > 0 and np.isfinite(lp.lv[j]):
            bps.add(omega * (x[j] - lp.lv[j]) / g[j])
        if g[j] < 0 and np.isfinite(lp.uv[j]):
            bps.add(omega * (lp.uv[j] - x[j]) / (-g[j]))
    for i in range(y.shape[0]):
        for bnd in (lp.lc[i], lp.uc[i]):
            if np.isfinite(bnd):
                sl = bnd - Ax[i]
                if sl != 0:
                    s = -y[i] / (omega * sl)
                    if s > 0:
                        bps.add(s)
    bps = sorted(b for b in bps if b > 0)

    def dist2(s):
        xh, yh = _trial(lp, x, y, Ax, g, omega, s)
        return omega * np.sum((xh - x) ** 2) + np.sum((yh - y) ** 2) / omega

    A_T = lp.A
    Axf = lambda v: A_T @ v  # noqa: E731

    def F(s):
        xh, yh = _trial(lp, x, y, Ax, g, omega, s)
        return lagrangian(lp, x, yh, Axf) - lagrangian(lp, xh, y, Axf)

    lo = 0.0
    pts = bps + [max(bps[-1] * 2.0, 1.0) if bps else 1.0]
    hi = None
    for b in pts:
        if dist2(b) >= r * r:
            hi = b
            break
        lo = b
    if hi is None:
        # saturated within the ball, or the crossing is past the last breakpoint
        if dist2(pts[-1] * 4) <= dist2(pts[-1]) * (1 + 1e-15):
            return F(pts[-1]) / r
        hi = pts[-1] * 2
        while dist2(hi) < r * r:
            lo, hi = hi, hi * 2
    # exact quadratic on [lo, hi]: in t = (s - lo)/(hi - lo) it is a t^2 + b t + c
    w = hi - lo
    ts = np.array([0.25, 0.5, 0.75])
    vals = np.array([dist2(lo + w * t) for t in ts])
    # interpolate exactly through the three samples
    c2 = (vals[0] - 2.0 * vals[1] + vals[2]) / (2.0 * 0.25 * 0.25)
    c1 = (vals[2] - vals[0]) / 0.5 - c2 * (ts[2] + ts[0])
    c0 = vals[1] - c2 * 0.25 - c1 * 0.5
    rr = r * r
    if abs(c2) < 1e-300:
        t_star = (rr - c0) / c1
    else:
        disc = max(c1 * c1 - 4.0 * c2 * (c0 - rr), 0.0)
        cands = [(-c1 + math.sqrt(disc)) / (2 * c2), (-c1 - math.sqrt(disc)) / (2 * c2)]
        cands = [t for t in cands if -1e-9 <= t <= 1 + 1e-9] or cands
        t_star = min(cands, key=lambda t: abs(t - 0.5))
    s_star = lo + w * min(max(t_star, 0.0), 1.0)
    return F(s_star) / r


def _p_rows(lp, Y):
    """p(y; -uc, -lc) for each row of Y (vectorised Sec. 2 definition, 0*inf = 0)."""
    lc = np.where(np.isfinite(lp.lc), lp.lc, 0.0)
    uc = np.where(np.isfinite(lp.uc), lp.uc, 0.0)
    return (-(np.maximum(Y, 0.0) * lc) + (np.maximum(-Y, 0.0) * uc)).sum(axis=1)


def sample_trust_region_max(lp, x, y, A_dense, r, omega, rng, nsamp=400000):
    """Monte-Carlo lower estimate of max {L(x,yh) - L(xh,y)} over zh in X x Y with
    ||zh - z||_omega <= r (for tiny n + m), by uniform samples in the ball; L is
    evaluated from its definition, Eq. (2)."""
    n, m = x.shape[0], y.shape[0]
    d = n + m
    u = rng.standard_normal((nsamp, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = rng.random(nsamp) ** (1.0 / d)
    pts = u * rad[:, None] * r
    xh = x + pts[:, :n] / math.sqrt(omega)
    yh = y + pts[:, n:] * math.sqrt(omega)
    ok = np.all((xh >= lp.lv) & (xh <= lp.uv), axis=1)
    for i in range(m):
        if not np.isfinite(lp.lc[i]):
            ok &= yh[:, i] <= 0
        if not np.isfinite(lp.uc[i]):
            ok &= yh[:, i] >= 0
    xh, yh = xh[ok], yh[ok]
    Ax = A_dense @ x
    L_x_yh = lp.c @ x - yh @ Ax - _p_rows(lp, yh)
    L_xh_y = xh @ lp.c - (xh @ A_dense.T) @ y - _p_rows(lp, y[None, :])[0]
    return float(np.max(L_x_yh - L_xh_y)) if xh.shape[0] else -math.inf


def lp_with_feasible_pair(rng, m, n, density=0.4):
    """A random LP with every kind of bound (two-sided, equality, one-sided, free rows;
    boxed, one-sided, free columns) built around a primal feasible x_F and a dual
    feasible y_F (sign pattern of Sec. 2's Y, reduced costs r_F in R, c = A'y_F + r_F),
    so that it has an optimum.  Returns (inst, x_F, y_F)."""
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    for i in range(m):  # no empty row
        if not A[i].any():
            A[i, rng.integers(n)] = 1.0
    x_F = rng.uniform(-2, 2, n)
    ax = A @ x_F
    kind_r = rng.integers(0, 5, m)  # 0 two-sided, 1 equality, 2 lower only, 3 upper only, 4 free
    lc = np.where(np.isin(kind_r, (0, 2)), ax - rng.uniform(0, 1, m), -np.inf)
    uc = np.where(np.isin(kind_r, (0, 3)), ax + rng.uniform(0, 1, m), np.inf)
    lc = np.where(kind_r == 1, ax, lc)
    uc = np.where(kind_r == 1, ax, uc)
    y_F = rng.standard_normal(m)
    y_F = np.where(kind_r == 2, np.abs(y_F), y_F)
    y_F = np.where(kind_r == 3, -np.abs(y_F), y_F)
    y_F = np.where(kind_r == 4, 0.0, y_F)
    kind_c = rng.integers(0, 4, n)  # 0 boxed, 1 lower only, 2 upper only, 3 free
    lv = np.where(np.isin(kind_c, (0, 1)), x_F - rng.uniform(0, 2, n), -np.inf)
    uv = np.where(np.isin(kind_c, (0, 2)), x_F + rng.uniform(0, 2, n), np.inf)
    r_F = rng.standard_normal(n)
    r_F = np.where(kind_c == 1, np.abs(r_F), r_F)
    r_F = np.where(kind_c == 2, -np.abs(r_F), r_F)
    r_F = np.where(kind_c == 3, 0.0, r_F)
    c = A.T @ y_F + r_F
    return make_lp(A, c, lc, uc, lv, uv, name="feasible-pair"), x_F, y_F
