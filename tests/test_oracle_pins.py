"""Pins of the CPU oracle against things other than itself: closed forms, brute force,
a second library solver, textbook operators, invariants the paper states.

Each test names the passage of the paper it checks.  All run on the CPU.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import lpgen
from oracle import pdlp_oracle as O
from tests import lp_helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _highs(inst):
    A = inst.scipy_csr().toarray()
    rows_ub, rhs_ub, rows_eq, rhs_eq = [], [], [], []
    for i in range(inst.m):
        if inst.lc[i] == inst.uc[i]:
            rows_eq.append(A[i]); rhs_eq.append(inst.lc[i])
            continue
        if np.isfinite(inst.uc[i]):
            rows_ub.append(A[i]); rhs_ub.append(inst.uc[i])
        if np.isfinite(inst.lc[i]):
            rows_ub.append(-A[i]); rhs_ub.append(-inst.lc[i])
    bounds = [(None if not np.isfinite(l) else l, None if not np.isfinite(u) else u)
              for l, u in zip(inst.lv, inst.uv)]
    r = so.linprog(inst.c, A_ub=np.array(rows_ub) if rows_ub else None,
                   b_ub=np.array(rhs_ub) if rhs_ub else None,
                   A_eq=np.array(rows_eq) if rows_eq else None,
                   b_eq=np.array(rhs_eq) if rhs_eq else None, bounds=bounds, method="highs")
    assert r.status == 0
    return r.fun


# ---------------------------------------------------------------------------
# whole solve: closed forms, brute force, a second solver
# ---------------------------------------------------------------------------

def test_box_only_closed_form():
    """m = 0 (Eq. (1) without rows): x_i = lv_i if c_i > 0 else uv_i."""
    rng = np.random.default_rng(1)
    n = 50
    lv = rng.uniform(-5, 0, n)
    uv = lv + rng.uniform(0.5, 3, n)
    c = rng.uniform(-1, 1, n)
    inst = H.make_lp(np.zeros((0, n)), c, [], [], lv, uv)
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-12))
    assert res.status == O.OPTIMAL
    x_star = np.where(c > 0, lv, uv)
    np.testing.assert_allclose(res.x, x_star, rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_vertices_and_highs(seed):
    """Small two-sided LPs (n <= 5): PDLP's objective equals the best vertex (Eq. (1))
    and scipy-HiGHS's optimum."""
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(2, 5)), int(rng.integers(2, 6))
    inst = H.random_bounded_lp(rng, m, n)
    best, _ = H.brute_force_vertices(inst)
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-10, max_iters=200000))
    assert res.status == O.OPTIMAL
    assert abs(res.stats["pobj"] - best) <= 1e-6 * (1 + abs(best))
    assert abs(_highs(inst) - best) <= 1e-7 * (1 + abs(best))


def test_diagonal_closed_form():
    """Diagonal A: every coordinate decouples; x_j* is the end of
    [max(lv, lc/a), min(uv, uc/a)] that c_j points to (Eq. (1))."""
    rng = np.random.default_rng(7)
    n = 300
    a = rng.uniform(0.5, 3.0, n) * np.where(rng.random(n) < 0.5, -1, 1)
    lv, uv = np.full(n, -2.0), np.full(n, 2.0)
    t_lo = rng.uniform(-1.5, 0.0, n)
    t_hi = t_lo + rng.uniform(0.2, 1.0, n)
    lc = np.where(a > 0, a * t_lo, a * t_hi)
    uc = np.where(a > 0, a * t_hi, a * t_lo)
    c = rng.uniform(-1, 1, n)
    inst = H.make_lp(np.diag(a), c, lc, uc, lv, uv)
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-11, max_iters=100000))
    assert res.status == O.OPTIMAL
    x_star = np.where(c > 0, np.maximum(lv, t_lo), np.minimum(uv, t_hi))
    np.testing.assert_allclose(res.x, x_star, atol=1e-7)


def test_continuous_knapsack_closed_form():
    """One equality row sum a_i x_i = b, 0 <= x <= u: greedy fill by c_i/a_i."""
    rng = np.random.default_rng(11)
    n = 40
    a = rng.uniform(0.5, 2.0, n)
    u = rng.uniform(0.5, 2.0, n)
    c = rng.uniform(-1, 1, n)
    b = 0.4 * float(a @ u)
    inst = H.make_lp(a[None, :], c, [b], [b], np.zeros(n), u)
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-11, max_iters=200000))
    assert res.status == O.OPTIMAL
    order = np.argsort(c / a)
    x = np.zeros(n)
    left = b
    for j in order:
        take = min(u[j], left / a[j])
        x[j] = take
        left -= take * a[j]
        if left <= 0:
            break
    assert abs(res.stats["pobj"] - c @ x) <= 1e-7 * (1 + abs(c @ x))


def test_golden_textbook_lp():
    """A hand-solved two-variable LP (Eq. (1)); primal and dual optimum derived by hand
    in the fixture."""
    with open(os.path.join(GOLDEN, "textbook_lp.json")) as f:
        g = json.load(f)
    inf = float("inf")
    conv = lambda v: [inf if s == "inf" else (-inf if s == "-inf" else s) for s in v]  # noqa
    inst = H.make_lp(g["A"], g["c"], conv(g["lc"]), conv(g["uc"]), conv(g["lv"]), conv(g["uv"]))
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-12, max_iters=100000))
    assert res.status == O.OPTIMAL
    np.testing.assert_allclose(res.x, g["x_star"], atol=1e-8)
    np.testing.assert_allclose(res.y, g["y_star"], atol=1e-8)
    assert abs(res.stats["pobj"] - g["obj"]) < 1e-8


def test_config0_matches_highs_and_kkt():
    """The small random LP reaches relative KKT 1e-8; objective equals HiGHS's; the
    residuals and the gap vanish (Sec. 7 termination quantities)."""
    inst = lpgen.config0()
    res = O.solve(inst, O.Params())
    assert res.status == O.OPTIMAL
    st = res.stats
    assert st["rel_kkt"] <= 1e-8
    ref = _highs(inst)
    assert abs(st["pobj"] - ref) <= 1e-6 * abs(ref)


def test_weak_duality_any_dual_point():
    """For a primal-feasible x and any y in Y with r = proj_R(c - A'y), the dual
    objective lc'y+ - uc'y- + lv'r+ - uv'r- never exceeds c'x when c - A'y - r = 0
    (Eq. (1)); with every variable boxed R is all of R^n, so any y in Y qualifies."""
    inst = lpgen.config0()
    A = inst.scipy_csr()
    rng = np.random.default_rng(3)
    for _ in range(20):
        y = rng.standard_normal(inst.m) * 3
        y = np.where(~np.isfinite(inst.lc) & (y > 0), 0.0, y)
        st = O.kkt_stats(inst, A, inst.x0, y)
        assert st["dual_res_l2"] == 0.0
        assert st["dobj"] <= st["pobj"] + 1e-9
        assert st["primal_res_l2"] <= 1e-9


def test_scaled_and_unscaled_same_objective():
    """Preconditioning changes the iterates, not the LP (Sec. 3): with and without it
    the objective agrees."""
    inst = lpgen.random_lp(60, 120, 4, seed=5)
    a = O.solve(inst, O.Params(eps_rel_kkt=1e-9, max_iters=300000))
    b = O.solve(inst, O.Params(eps_rel_kkt=1e-9, ruiz_iters=0, pc_alpha=0.0, max_iters=300000))
    assert a.status == O.OPTIMAL and b.status == O.OPTIMAL
    assert abs(a.stats["pobj"] - b.stats["pobj"]) <= 1e-6 * (1 + abs(a.stats["pobj"]))


# ---------------------------------------------------------------------------
# the PDHG step (Eq. (3), App. B)
# ---------------------------------------------------------------------------

def _rand_bounds(rng, m):
    lc = rng.standard_normal(m)
    uc = lc + rng.uniform(0, 2, m)
    kind = rng.integers(0, 5, m)
    lc = np.where(kind == 1, -np.inf, lc)
    uc = np.where(kind == 2, np.inf, uc)
    lc = np.where(kind == 3, -np.inf, lc)
    uc = np.where(kind == 3, np.inf, uc)
    uc = np.where(kind == 4, lc, uc)
    return lc, uc


def test_dual_step_equals_prox_argmin():
    """Eq. (3b) equals the PDHG dual step of App. B written as an explicit argmin of
    p(y; -uc, -lc) + ||y - (y_k - sigma A(2x'-x))||^2 / (2 sigma) over Y."""
    rng = np.random.default_rng(4)
    m = 400
    lc, uc = _rand_bounds(rng, m)
    for sigma in (0.01, 0.7, 5.0):
        y = rng.standard_normal(m)
        y = np.where(~np.isfinite(lc) & (y > 0), -y, y)
        y = np.where(~np.isfinite(uc) & (y < 0), -y, y)
        y = np.where(~np.isfinite(lc) & ~np.isfinite(uc), 0.0, y)
        Ax = rng.standard_normal(m)
        Axn = rng.standard_normal(m)
        got = O.dual_step(y, Ax, Axn, lc, uc, sigma)
        v = y - sigma * (2 * Axn - Ax)
        want = H.prox_p_argmin(v, sigma, lc, uc)
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-14 * np.abs(v).max())


def test_dual_step_literal_formula():
    """The evaluation order of R17 agrees with Eq. (3b) as printed,
    y - sigma q - sigma proj_[-uc,-lc](y/sigma - q), to rounding."""
    rng = np.random.default_rng(5)
    m = 1000
    lc, uc = _rand_bounds(rng, m)
    y = np.zeros(m)
    Ax = rng.standard_normal(m)
    Axn = rng.standard_normal(m)
    sigma = 0.37
    q = 2 * Axn - Ax
    lit = y - sigma * q - sigma * np.clip(y / sigma - q, -uc, -lc)
    got = O.dual_step(y, Ax, Axn, lc, uc, sigma)
    np.testing.assert_allclose(got, lit, rtol=1e-13, atol=1e-15)


def test_fixed_step_iterates_equal_chambolle_pock():
    """With restarts off and eta, omega fixed, PDLP's iterates are textbook PDHG
    (Chambolle-Pock with K = -A, App. B), dual prox as an explicit argmin."""
    inst = lpgen.random_lp(30, 50, 3, seed=9)
    prm = O.Params(ruiz_iters=0, pc_alpha=0.0, fixed_step=0.2, fixed_omega=1.3, restarts=False,
                   max_iters=40, eps_rel_kkt=0.0)
    res = O.solve(inst, prm, trace_iters=40)
    A = inst.scipy_csr()
    tau, sigma = 0.2 / 1.3, 0.2 * 1.3
    x = np.clip(np.zeros(inst.n), inst.lv, inst.uv)
    y = np.zeros(inst.m)
    for rec in res.trace:
        xn = np.clip(x - tau * (inst.c - A.T @ y), inst.lv, inst.uv)
        v = y - sigma * (A @ (2 * xn - x))
        yn = H.prox_p_argmin(v, sigma, inst.lc, inst.uc)
        np.testing.assert_allclose(rec["x"], xn, atol=1e-11)
        np.testing.assert_allclose(rec["y"], yn, atol=1e-11)
        x, y = xn, yn


def test_iterates_stay_in_X_and_Y_exactly():
    """Sec. 2's case analysis: y^{k+1} in Y and x^{k+1} in X, bit for bit, for every
    iterate (free rows keep y_i = 0 exactly)."""
    inst = lpgen.random_lp(80, 160, 4, seed=12)
    inst.lc[:10] = -np.inf
    inst.uc[10:20] = np.inf
    inst.lc[20:25] = -np.inf
    inst.uc[20:25] = np.inf
    lp = O.precondition(inst)
    res = O.solve(inst, O.Params(max_iters=300), trace_iters=300, lp=lp)
    for rec in res.trace:
        x, y = rec["x"], rec["y"]
        assert np.all(x >= lp.lv) and np.all(x <= lp.uv)
        assert np.all(y[:10] <= 0)
        assert np.all(y[10:20] >= 0)
        assert np.all(y[20:25] == 0)


def test_step_size_bound_and_acceptance():
    """Algorithm 2: the accepted eta satisfies Eq. (5), and eta_bar >= 1/||A||_2
    (Sec. 3, "Step size choice"), ||A||_2 from a dense SVD."""
    inst = lpgen.random_lp(40, 70, 4, seed=13)
    lp = O.precondition(inst)
    Ad = lp.A.toarray()
    nrm = np.linalg.svd(Ad, compute_uv=False)[0]
    rng = np.random.default_rng(14)
    for trial in range(30):
        x = np.clip(rng.standard_normal(inst.n) * 3, lp.lv, lp.uv)
        y = rng.standard_normal(inst.m)
        Ax, ATy = Ad @ x, Ad.T @ y
        omega = float(np.exp(rng.uniform(-2, 2)))
        for eta in (0.01, 1.0, 10.0):
            xn = O.primal_step(x, ATy, lp.c, lp.lv, lp.uv, eta / omega)
            yn = O.dual_step(y, Ax, Ad @ xn, lp.lc, lp.uc, eta * omega)
            dx, dy = xn - x, yn - y
            inter = abs(dy @ (Ad @ dx))
            if inter > 0:
                eta_bar = (omega * dx @ dx + dy @ dy / omega) / (2 * inter)
                assert eta_bar >= (1 - 1e-12) / nrm
        xo, yo, Axo, eta_acc, eta_new, att, ok = O.adaptive_step(
            lp, x, y, Ax, ATy, omega, 50.0, trial, 60)
        assert ok
        dx, dy = xo - x, yo - y
        inter = abs(dy @ (Axo - Ax))
        if inter > 0:
            assert eta_acc <= (omega * dx @ dx + dy @ dy / omega) / (2 * inter) * (1 + 1e-12)
        assert eta_new <= (1 + (trial + 2) ** -0.6) * eta_acc * (1 + 1e-15)


def test_running_average_and_linearity():
    """The weighted average since the last restart (Algorithm 1) equals the directly
    weighted mean of the traced iterates, and A x_bar from the running sums equals
    A (x_bar) (linearity, R18)."""
    inst = lpgen.random_lp(50, 90, 4, seed=15)
    lp = O.precondition(inst)
    res = O.solve(inst, O.Params(max_iters=60, restarts=False, eps_rel_kkt=0.0),
                  trace_iters=60, lp=lp)
    xs = np.array([r["x"] for r in res.trace])
    ys = np.array([r["y"] for r in res.trace])
    w = np.array([r["eta"] for r in res.trace])
    xbar = (w[:, None] * xs).sum(0) / w.sum()
    Axbar_sum = (w[:, None] * np.array([lp.A @ v for v in xs])).sum(0) / w.sum()
    np.testing.assert_allclose(lp.A @ xbar, Axbar_sum, atol=1e-12 * (1 + np.abs(Axbar_sum).max()))
    ybar = (w[:, None] * ys).sum(0) / w.sum()
    assert np.all(np.isfinite(ybar))


# ---------------------------------------------------------------------------
# normalized duality gap (Sec. 3, "Adaptive restarts")
# ---------------------------------------------------------------------------

def _rand_point(rng, lp, scale=1.0):
    with np.errstate(invalid="ignore"):
        x = np.clip(lp.lv + (lp.uv - lp.lv) * rng.random(lp.c.shape[0]), lp.lv, lp.uv)
    x = np.where(np.isfinite(x), x, rng.standard_normal(x.shape[0]))
    y = rng.standard_normal(lp.lc.shape[0]) * scale
    y = np.where(~np.isfinite(lp.lc) & (y > 0), -y, y)
    y = np.where(~np.isfinite(lp.uc) & (y < 0), -y, y)
    y = np.where(~np.isfinite(lp.lc) & ~np.isfinite(lp.uc), 0.0, y)
    return x, y


@pytest.mark.parametrize("seed", range(4))
def test_normalized_gap_vs_sorted_breakpoints(seed):
    """Bisection on the ball multiplier (oracle) vs an exact solve over sorted
    breakpoints with the Lagrangian evaluated from Eq. (2) (helper)."""
    rng = np.random.default_rng(200 + seed)
    inst = lpgen.random_lp(25, 40, 3, seed=300 + seed, free_frac=0.1)
    inst.lc[:4] = -np.inf
    inst.uc[4:8] = np.inf
    lp = O.precondition(inst)
    for _ in range(3):
        x, y = _rand_point(rng, lp)
        xr, yr = _rand_point(rng, lp)
        omega = float(np.exp(rng.uniform(-1, 1)))
        Ax, ATy = lp.A @ x, lp.AT @ y
        got = O.normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega)
        want = H.exact_normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega)
        assert abs(got - want) <= 1e-8 * (1 + abs(want))


@pytest.mark.parametrize("case", range(4))
def test_normalized_gap_vs_sampling_tiny(case):
    """n + m <= 3: the trust-region maximum is at least every sampled feasible value
    in the ball, and sampling gets within a small margin of it."""
    rng = np.random.default_rng(500 + case)
    m, n = (1, 1) if case < 2 else (1, 2)
    A = rng.standard_normal((m, n))
    lc = np.array([-0.5]) if case != 1 else np.array([-np.inf])
    uc = np.array([0.8])
    inst = H.make_lp(A, rng.uniform(-1, 1, n), lc, uc, np.full(n, -1.0), np.full(n, 1.5))
    lp = O.precondition(inst, ruiz_iters=0, pc_alpha=0.0)
    x, y = _rand_point(rng, lp)
    xr, yr = _rand_point(rng, lp)
    omega = 0.8
    Ad = lp.A.toarray()
    Ax, ATy = Ad @ x, Ad.T @ y
    mu = O.normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega)
    r = math.sqrt(omega * np.sum((x - xr) ** 2) + np.sum((y - yr) ** 2) / omega)
    best = H.sample_trust_region_max(lp, x, y, Ad, r, omega, rng)
    assert mu * r >= best - 1e-9
    assert mu * r <= best + 0.02 * (abs(best) + r)


def test_normalized_gap_zero_at_optimum():
    """rho_r(z) = 0 iff z is optimal (Sec. 3): tiny at a tightly converged point,
    clearly positive at the starting point."""
    inst = lpgen.random_lp(30, 60, 3, seed=21)
    lp = O.precondition(inst)
    res = O.solve(inst, O.Params(eps_rel_kkt=1e-12, max_iters=400000), lp=lp)
    assert res.status == O.OPTIMAL
    xs, ys = res.x / lp.d2, res.y / lp.d1
    Ax, ATy = lp.A @ xs, lp.AT @ ys
    rng = np.random.default_rng(22)
    xr, yr = _rand_point(rng, lp)
    mu_opt = O.normalized_gap(lp, xs, ys, Ax, ATy, xr, yr, 1.0)
    x0 = np.clip(np.zeros(inst.n), lp.lv, lp.uv)
    mu_0 = O.normalized_gap(lp, x0, np.zeros(inst.m), lp.A @ x0, np.zeros(inst.n), xr, yr, 1.0)
    assert abs(mu_opt) < 1e-6
    assert mu_0 > 1e-2


def test_normalized_gap_ball_inactive_is_duality_gap():
    """When every direction saturates inside the ball, r*rho_r(z) is the plain
    duality gap max_{zh in Z} L(x,yh) - L(xh,y): for boxed x it is attained at the box
    corner against g, and for rows with lc <= (Ax)_i <= uc every row term peaks at 0."""
    rng = np.random.default_rng(23)
    m, n = 6, 9
    A = rng.standard_normal((m, n))
    x = rng.uniform(-1, 1, n)
    ax = A @ x
    lc = ax - rng.uniform(1, 2, m)
    uc = ax + rng.uniform(1, 2, m)
    lc[:3] = -np.inf  # rows with yh <= 0 only
    inst = H.make_lp(A, rng.uniform(-1, 1, n), lc, uc, np.full(n, -1.0), np.full(n, 1.0))
    lp = O.precondition(inst, ruiz_iters=0, pc_alpha=0.0)
    y = rng.standard_normal(m)
    y[:3] = -np.abs(y[:3])
    Ad = lp.A.toarray()
    Ax, ATy = Ad @ x, Ad.T @ y
    g = lp.c - ATy
    xr = x + 1e6  # reference far away: the ball contains everything reachable
    yr = y
    omega = 1.0
    r = math.sqrt(omega * np.sum((x - xr) ** 2) + np.sum((y - yr) ** 2) / omega)
    mu = O.normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega)
    xh = np.where(g > 0, lp.lv, np.where(g < 0, lp.uv, x))
    yh = np.zeros(m)
    gap = H.lagrangian(lp, x, yh, lambda v: Ad @ v) - H.lagrangian(lp, xh, y, lambda v: Ad @ v)
    assert gap > 0
    assert abs(mu * r - gap) <= 1e-9 * (1 + abs(gap))


# ---------------------------------------------------------------------------
# preconditioning, primal weight
# ---------------------------------------------------------------------------

def test_ruiz_norms_go_to_one():
    """Ruiz (Sec. 3): applied iteratively, every row and column infinity norm tends
    to 1."""
    inst = lpgen.config1(scale=0.001)
    lp = O.precondition(inst, ruiz_iters=60, pc_alpha=0.0)
    A = abs(lp.A)
    rmax = A.max(axis=1).toarray().ravel()
    cmax = A.max(axis=0).toarray().ravel()
    assert np.all(np.abs(rmax[rmax > 0] - 1) < 1e-3)
    assert np.all(np.abs(cmax[cmax > 0] - 1) < 1e-3)
    # and the scaled matrix is D1 A D2 exactly as recorded
    A0 = inst.scipy_csr()
    D = sp.diags(lp.d1) @ A0 @ sp.diags(lp.d2)
    np.testing.assert_allclose(D.toarray() if D.shape[0] < 3000 else D.data,
                               lp.A.toarray() if D.shape[0] < 3000 else lp.A.data, rtol=1e-12)


def test_pock_chambolle_alpha1_row_col_l1():
    """Pock-Chambolle with alpha = 1 alone: row and column l1 norms of D1 A D2 with
    D1 = 1/sqrt(row l1), D2 = 1/sqrt(col l1), checked on a dense matrix."""
    rng = np.random.default_rng(24)
    Ad = rng.standard_normal((7, 5))
    Ad[2] = 0
    inst = H.make_lp(Ad, np.ones(5), -np.ones(7), np.ones(7), np.zeros(5), np.ones(5))
    lp = O.precondition(inst, ruiz_iters=0, pc_alpha=1.0)
    r = np.abs(Ad).sum(1)
    c = np.abs(Ad).sum(0)
    d1 = 1 / np.sqrt(np.where(r > 0, r, 1.0))  # a zero row keeps factor 1
    d2 = 1 / np.sqrt(c)
    np.testing.assert_allclose(lp.d1, d1, rtol=1e-15)
    np.testing.assert_allclose(lp.d2, d2, rtol=1e-15)
    np.testing.assert_allclose(lp.A.toarray(), d1[:, None] * Ad * d2[None, :], rtol=1e-14)
    assert lp.lv[0] == 0 and lp.uv[0] == pytest.approx(1 / d2[0], rel=1e-15)


@pytest.mark.parametrize("beta_art,num,den", [(0.5, 2, 1), (0.25, 4, 3)])
def test_artificial_restarts_follow_the_closed_form_schedule(beta_art, num, den):
    """Restart criterion (iii) of Sec. 3 alone (beta_suff = beta_nec = 0 switch (i) and
    (ii) off away from an exact optimum; no termination): a restart at k_j resets t, so
    the next one falls at the first k with k - k_j >= beta_art k, i.e.
    k_{j+1} = ceil(k_j / (1 - beta_art)) = ceil(num k_j / den), from k_1 = 1 -- powers of
    two for beta_art = 1/2.  Pins the counting of k and t (R3, R4) and the reset."""
    iters = 300
    prm = O.Params(beta_suff=0.0, beta_nec=0.0, beta_art=beta_art, eps_rel_kkt=0.0,
                   max_iters=iters, detect_infeasibility=False)
    res = O.solve(lpgen.config0(), prm, trace_iters=iters)
    got = [(r["k"], r["restart"]) for r in res.trace if r["restart"] != O.RESTART_NONE]
    want, k = [], 1
    while k < iters:
        want.append(k)
        k = -(-num * k // den)
    assert [k for k, _ in got] == want
    assert all(kind == O.RESTART_ARTIFICIAL for _, kind in got)
    assert res.stats["restarts"] == [0, 0, len(want)]


def test_sufficient_decay_restarts_only_at_checks():
    """Criterion (i) of Sec. 3 with beta_suff so large that it always holds: it is only
    evaluated at the periodic checks (every 64 iterations, R4), after the first restart
    has set mu(z^{n,0}, z^{n-1,0}) (R5), and it takes precedence over (iii) when both
    apply.  So (iii) restarts at k = 1, 2, 4, ..., 32 and (i) at every multiple of 64."""
    iters = 300
    prm = O.Params(beta_suff=1e300, beta_nec=0.0, eps_rel_kkt=0.0, max_iters=iters,
                   detect_infeasibility=False)
    res = O.solve(lpgen.config0(), prm, trace_iters=iters)
    got = [(r["k"], r["restart"]) for r in res.trace if r["restart"] != O.RESTART_NONE]
    want = [(2 ** j, O.RESTART_ARTIFICIAL) for j in range(6)]
    want += [(k, O.RESTART_SUFFICIENT) for k in range(64, iters, 64)]
    assert got == want


def _bilinear_1x1_schedule(a, b, c, eta, omega, period, iters, beta_suff, beta_nec, beta_art):
    """Restart schedule of fixed-step PDHG on  min c x  s.t.  a x = b  (x free, one
    equality row, no preconditioning), from closed forms written here, not the
    oracle's code.

    Iterates: in the coordinates u = sqrt(omega) (x - x*), v = (y - y*) / sqrt(omega)
    around the saddle point (x*, y*) = (b/a, c/a), one step of Eq. (3) with tau =
    eta/omega, sigma = eta omega is the linear map  u' = u + h v,
    v' = -h u + (1 - 2 h^2) v,  h = eta a.
    Normalized gap: with every bound infinite, L(x, yh) - L(xh, y) is linear in
    (xh - x, yh - y) with gradient (a y - c, -(a x - b)); its maximum over the ball of
    omega-radius r is r times the dual norm of that gradient, so
    mu(z, z_ref) = |a| sqrt(u^2 + v^2) for any z_ref != z, whatever the radius.
    The average since a restart is the plain mean (equal weights eta).
    Rules of Sec. 3: at the periodic checks (k a multiple of ``period``) once
    mu(z^{n,0}, z^{n-1,0}) exists, (i) mu_c <= beta_suff mu_ref, else (ii) mu_c <=
    beta_nec mu_ref with mu_c above the previous check's candidate gap in the same
    outer loop; else (iii) t >= beta_art k.  Returns the restarts [(k, kind)] and
    the candidate gap, mu_ref and kind at every evaluation {k: (mu_c, mu_ref, kind)}."""
    M = np.array([[1.0, eta * a], [-eta * a, 1.0 - 2.0 * (eta * a) ** 2]])
    w = np.array([math.sqrt(omega) * (0.0 - b / a), (0.0 - c / a) / math.sqrt(omega)])
    mu = lambda v: abs(a) * float(np.hypot(v[0], v[1]))  # noqa: E731
    k = t = 0
    mu_ref, mu_prev, acc = None, math.inf, np.zeros(2)
    out, ev = [], {}
    for _ in range(iters):
        w = M @ w
        acc = acc + w
        k, t = k + 1, t + 1
        check, art = k % period == 0, t >= beta_art * k
        if not (check or art):
            continue
        avg = acc / t
        cand = w if mu(w) < mu(avg) else avg
        mu_c = mu(cand)
        kind = 0
        if check and mu_ref is not None:
            if mu_c <= beta_suff * mu_ref:
                kind = 1
            elif mu_c <= beta_nec * mu_ref and mu_c > mu_prev:
                kind = 2
        if kind == 0 and art:
            kind = 3
        ev[k] = (mu_c, mu_ref, kind, mu(w), mu(avg))
        if check:
            mu_prev = mu_c
        if kind:
            out.append((k, kind))
            w, mu_ref, mu_prev, acc, t = cand.copy(), mu(cand), math.inf, np.zeros(2), 0
    return out, ev


# min -x s.t. x = 1: x* = 1, y* = -1; eta = 1/4, omega = 4 (tau = 1/16, sigma = 1: exact)
BILINEAR_SCHEDULE = [(1, 3), (2, 3), (4, 3), (8, 3), (16, 3), (32, 3), (64, 3), (90, 1),
                     (130, 2), (180, 1)]


def bilinear_instance():
    return H.make_lp(np.array([[1.0]]), np.array([-1.0]), np.array([1.0]), np.array([1.0]),
                     np.array([-np.inf]), np.array([np.inf]))


def test_restart_criteria_i_and_ii_at_the_paper_thresholds():
    """Criteria (i) and (ii) of Sec. 3 at beta_suff = 0.1, beta_nec = 0.9 (beta_art =
    0.5, checks every 10 iterations) on a closed-form trajectory: the rotating, not
    monotone, gap of fixed-step PDHG on a 1 x 1 equality-constrained LP with a free
    variable.  (iii) restarts at 1, 2, 4, ..., 64; (i) at k = 90, where the average's
    gap is 0.0885 of mu_ref; (ii) at k = 130, where the candidate gap (0.118 of mu_ref)
    rose above the k = 120 check's; (i) again at 180.  The facts that separate the
    schedule from plausible misreadings are asserted on the closed form too: at k = 64
    (a (iii) iteration, not a check) and at k = 70 (the first check after that restart)
    the candidate gap lies below 0.9 mu_ref and above the last check's, so evaluating
    (ii) between checks, or keeping the previous candidate gap across a restart, would
    restart by (ii) there; at k = 30 the gap is 0.41 of mu_ref, so swapped thresholds
    would restart by (i)."""
    iters = 200
    want, ev = _bilinear_1x1_schedule(1.0, 1.0, -1.0, 0.25, 4.0, 10, iters, 0.1, 0.9, 0.5)
    assert want == BILINEAR_SCHEDULE
    r = {k: v[0] / v[1] if v[1] else math.nan for k, v in ev.items()}
    assert r[90] < 0.1 and 0.1 < r[130] <= 0.9 and ev[130][0] > ev[120][0] and r[180] < 0.1
    assert 0.1 < r[64] <= 0.9 and ev[64][0] > ev[60][0]   # (ii) would hold at the (iii) step
    assert 0.1 < r[70] <= 0.9 and ev[70][0] > ev[60][0]   # ... and against a stale mu_c_prev
    assert 0.1 < r[30] <= 0.9                             # (i) with beta 0.9 would fire
    # every decision is away from its threshold by far more than rounding
    for k, (mu_c, mu_ref, _, mc, ma) in ev.items():
        if mu_ref:
            assert min(abs(mu_c - 0.1 * mu_ref), abs(mu_c - 0.9 * mu_ref)) > 1e-3 * mu_ref, k
    prm = O.Params(fixed_step=0.25, fixed_omega=4.0, check_period=10, ruiz_iters=0, pc_alpha=0.0,
                   eps_rel_kkt=-1.0, max_iters=iters, detect_infeasibility=False)
    res = O.solve(bilinear_instance(), prm, trace_iters=iters)
    got = [(rec["k"], rec["restart"]) for rec in res.trace if rec["restart"] != O.RESTART_NONE]
    assert got == BILINEAR_SCHEDULE
    assert res.stats["restarts"] == [2, 1, 7]
    # the oracle's normalized gap (bisection on the trust-region multiplier) equals the
    # closed form at every evaluation
    for rec in res.trace:
        if rec["k"] in ev:
            _, _, _, mc, ma = ev[rec["k"]]
            assert rec["mu_cur"] == pytest.approx(mc, rel=1e-11), rec["k"]
            assert rec["mu_avg"] == pytest.approx(ma, rel=1e-11), rec["k"]


SECOND_BILINEAR_SCHEDULE = [(1, 3), (2, 3), (4, 3), (8, 3), (16, 3), (32, 3), (48, 1), (69, 2),
                            (87, 1), (108, 2), (126, 1), (147, 2), (165, 1), (186, 2)]


def test_necessary_decay_needs_the_decay_bound():
    """The same LP with eta = 11/32, omega = 4 and checks every 3 iterations: (i) and (ii)
    alternate from k = 48 on.  After the (iii) restart at k = 8 the candidate gap rises
    from the k = 9 check to the k = 12 check but stays above 0.9 mu_ref, so (ii) must
    not fire there: its decay bound is what holds it back."""
    iters = 200
    want, ev = _bilinear_1x1_schedule(1.0, 1.0, -1.0, 11 / 32, 4.0, 3, iters, 0.1, 0.9, 0.5)
    assert want == SECOND_BILINEAR_SCHEDULE
    assert ev[12][0] > ev[9][0] and ev[12][0] > 0.9 * ev[12][1] and ev[12][2] == 0
    for k, (mu_c, mu_ref, _, _, _) in ev.items():
        if mu_ref:
            assert min(abs(mu_c - 0.1 * mu_ref), abs(mu_c - 0.9 * mu_ref)) > 1e-3 * mu_ref, k
    prm = O.Params(fixed_step=11 / 32, fixed_omega=4.0, check_period=3, ruiz_iters=0,
                   pc_alpha=0.0, eps_rel_kkt=-1.0, max_iters=iters, detect_infeasibility=False)
    res = O.solve(bilinear_instance(), prm, trace_iters=iters)
    got = [(rec["k"], rec["restart"]) for rec in res.trace if rec["restart"] != O.RESTART_NONE]
    assert got == SECOND_BILINEAR_SCHEDULE


# min x s.t. x = 2 with eta = omega = 1: the step map (h = 1) is nilpotent, so from
# z1 = (-1, 4) every iterate is the saddle point (2, 1)
NILPOTENT_SCHEDULE = [(1, 3), (10, 3)] + [(k, 1) for k in range(12, 40, 3)]


def nilpotent_instance():
    return H.make_lp(np.array([[1.0]]), np.array([1.0]), np.array([2.0]), np.array([2.0]),
                     np.array([-np.inf]), np.array([np.inf]))


def test_necessary_decay_needs_a_strict_increase():
    """Criterion (ii) asks the candidate gap to have *risen* since the previous check.
    On min x s.t. x = 2 (free x, eta = omega = 1) PDHG reaches the saddle point (2, 1)
    exactly at k = 2 and stays; the gap there is exactly 0.  With (i) switched off
    while mu_ref > 0 (beta_suff = -1), beta_art = 0.9 (so (iii) restarts at k = 1 and
    10) and checks every 3 iterations, the checks at k = 3, 6, 9 see mu_c = 0 = the
    previous candidate gap below 0.9 mu_ref = 0.9 mu(z1): no restart, because 0 > 0
    fails (a non-strict reading restarts at 6).  The restart at 10 makes the saddle
    point z^{n,0}, so mu_ref = 0 and (i) holds from then on (0 <= -0) at every check."""
    iters = 40
    want, ev = _bilinear_1x1_schedule(1.0, 2.0, 1.0, 1.0, 1.0, 3, iters, -1.0, 0.9, 0.9)
    assert want == NILPOTENT_SCHEDULE
    assert ev[3][0] == ev[6][0] == ev[9][0] == 0.0 and ev[6][1] > 0.0
    prm = O.Params(fixed_step=1.0, fixed_omega=1.0, check_period=3, beta_suff=-1.0,
                   beta_art=0.9, ruiz_iters=0, pc_alpha=0.0, eps_rel_kkt=-1.0, max_iters=iters,
                   detect_infeasibility=False)
    res = O.solve(nilpotent_instance(), prm, trace_iters=iters)
    assert list(res.trace[0]["x"]) == [-1.0] and list(res.trace[0]["y"]) == [4.0]
    assert all(list(r["x"]) == [2.0] and list(r["y"]) == [1.0] for r in res.trace[1:])
    got = [(rec["k"], rec["restart"]) for rec in res.trace if rec["restart"] != O.RESTART_NONE]
    assert got == NILPOTENT_SCHEDULE


def test_primal_weight_closed_form():
    """Algorithm 3 with theta = 1/2 is the geometric mean of omega and Dy/Dx; outside
    (eps0, 1/eps0) the weight is kept."""
    rng = np.random.default_rng(25)
    for _ in range(20):
        xo, yo = rng.standard_normal(5), rng.standard_normal(4)
        xn, yn = xo + rng.standard_normal(5), yo + rng.standard_normal(4)
        om = float(np.exp(rng.uniform(-3, 3)))
        dx, dy = np.linalg.norm(xn - xo), np.linalg.norm(yn - yo)
        assert abs(O.primal_weight_update(xn, yn, xo, yo, om) - math.sqrt(om * dy / dx)) \
            <= 1e-13 * math.sqrt(om * dy / dx)
    assert O.primal_weight_update(np.ones(3), np.ones(2), np.ones(3), np.zeros(2), 2.5) == 2.5
    assert O.primal_weight_update(np.ones(3) * 1e11, np.ones(2), np.zeros(3), np.zeros(2), 2.5) == 2.5


def test_initial_primal_weight_and_combine():
    """InitializePrimalWeight and Combine (Sec. 3) on a hand example."""
    lc = np.array([-np.inf, -3.0, 2.0, -np.inf])
    uc = np.array([4.0, 1.0, np.inf, np.inf])
    np.testing.assert_array_equal(O.combine(lc, uc), [4.0, 3.0, 2.0, 0.0])
    c = np.array([3.0, 4.0])
    assert O.initial_primal_weight(c, lc, uc) == pytest.approx(5.0 / math.sqrt(29.0), rel=1e-15)
    assert O.initial_primal_weight(np.zeros(2), lc, uc) == 1.0


def test_step_factors_first_step_positive():
    """Algorithm 2's reduction factor must be positive at the first step (R3)."""
    red, grow = O.step_factors(0)
    assert red == pytest.approx(1 - 2 ** -0.3) and grow == pytest.approx(1 + 2 ** -0.6)


def test_app_a_reduced_costs_closed_forms():
    """App. A: keep c_i - a_i'y only next to the bound it prices, measured against
    |x_i|.  Hand cases, and the golden LP's optimum, where complementary slackness makes
    both choices coincide (all measures ~0)."""
    g = np.array([-2.0, 3.0, 3.0, -1.0, 4.0])
    x = np.array([0.5, 0.5, -5.0, 9.0, 2.0])
    lv = np.array([0.0, 0.0, -np.inf, 0.0, 2.0])
    uv = np.array([1e12, 1e12, np.inf, 10.0, 2.0])
    r = O.reduced_costs_bound_proximity(g, x, lv, uv)
    # far from the huge upper bound: 0; near the lower bound: kept; free: 0;
    # upper bound 1 away from x = 9 (<= |x|): kept; fixed at 2: kept
    np.testing.assert_array_equal(r, [0.0, 3.0, 0.0, -1.0, 4.0])
    with open(os.path.join(GOLDEN, "textbook_lp.json")) as f:
        gold = json.load(f)
    inf = float("inf")
    conv = lambda v: [inf if s == "inf" else (-inf if s == "-inf" else s) for s in v]  # noqa
    inst = H.make_lp(gold["A"], gold["c"], conv(gold["lc"]), conv(gold["uc"]), conv(gold["lv"]),
                     conv(gold["uv"]))
    st = O.kkt_stats(inst, inst.scipy_csr(), np.array(gold["x_star"]), np.array(gold["y_star"]),
                     reduced_costs=1)
    assert st["rel_kkt"] <= 1e-12


def test_app_a_reduced_costs_huge_bound():
    """A variable with a huge, inactive upper bound: the natural reduced cost prices it
    at 1e12 and wrecks the dual objective; App. A's choice ignores it."""
    inst = H.make_lp([[1.0, 1.0]], [1.0, 2.0], [1.0], [1.0], [0.0, 0.0], [1e12, 1e12])
    x = np.array([1.0, 0.0])
    y = np.array([1.0 + 1e-9])  # slightly off the optimal multiplier 1
    nat = O.kkt_stats(inst, inst.scipy_csr(), x, y)
    app = O.kkt_stats(inst, inst.scipy_csr(), x, y, reduced_costs=1)
    assert nat["rel_gap"] > 1e-4      # -1e-9 * 1e12 enters the dual objective
    assert app["rel_kkt"] <= 1e-8


def test_app_a_reduced_costs_same_optimum():
    inst = lpgen.config0()
    a = O.solve(inst, O.Params(eps_rel_kkt=1e-8))
    b = O.solve(inst, O.Params(eps_rel_kkt=1e-8, reduced_costs=1))
    assert a.status == b.status == O.OPTIMAL
    assert abs(a.stats["pobj"] - b.stats["pobj"]) <= 1e-6 * abs(a.stats["pobj"])


def test_rescaled_criteria_q_and_w_by_hand():
    """Eq. (10)'s row and column scales on every case of Sec. 7's definition."""
    inf = math.inf
    lc = np.array([2.0, -inf, -3.0, -inf, 0.0, 0.0, -4.0, 5.0])
    uc = np.array([inf, 7.0, 6.0, inf, inf, 8.0, 0.0, 5.0])
    # only lc finite & nonzero | only uc | both | neither | lc = 0 (not counted), uc inf |
    # lc = 0, uc | lc, uc = 0 | equality row
    np.testing.assert_array_equal(O.row_scale_q(lc, uc), [2.0, 7.0, 6.0, 1.0, 1.0, 8.0, 4.0, 5.0])
    np.testing.assert_array_equal(O.col_scale_w(np.array([-3.0, 0.0, 0.5])), [3.0, 1.0, 0.5])


def test_rescaled_criteria_equal_absolute_residuals_of_the_rescaled_instance():
    """Sec. 7: the absolute l_inf criteria (Eq. (9)) on the paper's rescaled instance
    (Sec. 6: right-hand sides in {-inf, -1, 0, 1, inf} or scaled to max 1, objective in
    {-1, 0, 1}) are Eq. (10)'s scaled residuals on the LP as given.  The rescaling is
    built here explicitly -- row i divided by q_i, column j substituted x'_j = w_j x_j
    (so c'_j = c_j / w_j), y'_i = q_i y_i -- and kkt_stats of the transformed point on the
    rescaled LP must give, as absolute residuals, the scaled residuals of the original."""
    rng = np.random.default_rng(31)
    inf = math.inf
    m, n = 12, 9
    Ad = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6)
    c = rng.choice([-40.0, -2.5, 0.0, 0.3, 7.0, 90.0], n)
    lc = rng.choice([-inf, 0.0, -3.0, 12.0, 400.0], m)
    uc = np.where(np.isfinite(lc), lc + rng.choice([0.0, 5.0, inf], m), rng.choice([5.0, 300.0, inf], m))
    lv = rng.choice([-inf, 0.0, -2.0], n)
    uv = np.where(np.isfinite(lv), lv + rng.choice([1.0, 20.0, inf], n), rng.choice([4.0, inf], n))
    inst = H.make_lp(Ad, c, lc, uc, lv, uv)
    q, w = O.row_scale_q(lc, uc), O.col_scale_w(c)
    A2 = Ad / q[:, None] / w[None, :]
    resc = H.make_lp(A2, c / w, lc / q, uc / q, lv * w, uv * w)
    # the rescaled instance has the form of Sec. 6
    assert set(np.unique(resc.c)) <= {-1.0, 0.0, 1.0}
    for a, b in zip(resc.lc, resc.uc):
        fin = [abs(v) for v in (a, b) if math.isfinite(v) and v != 0]
        assert not fin or max(fin) == pytest.approx(1.0, rel=1e-15)
    for _ in range(5):
        x = rng.standard_normal(n) * 3
        x = np.clip(x, lv, uv)
        y = rng.standard_normal(m) * 2
        y = np.where(~np.isfinite(lc) & (y > 0), -y, y)
        y = np.where(~np.isfinite(uc) & (y < 0), -y, y)
        y = np.where(~np.isfinite(lc) & ~np.isfinite(uc), 0.0, y)  # y in Y
        st = O.kkt_stats(inst, inst.scipy_csr(), x, y)
        st2 = O.kkt_stats(resc, resc.scipy_csr(), x * w, y * q)
        assert st["primal_res_rel_inf"] == pytest.approx(st2["primal_res_inf"], rel=1e-13, abs=1e-15)
        assert st["dual_res_rel_inf"] == pytest.approx(st2["dual_res_inf"], rel=1e-13, abs=1e-15)
        # objectives and the relative gap of Eq. (8) are unchanged by the rescaling
        assert st["pobj"] == pytest.approx(st2["pobj"], rel=1e-13)
        assert st["paper_gap"] == pytest.approx(st2["paper_gap"], rel=1e-12, abs=1e-15)
