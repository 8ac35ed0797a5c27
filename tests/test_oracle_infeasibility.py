"""Pins of the oracle's infeasibility detection (Sec. 3 "Infeasibility detection",
App. C) against facts fixed outside it: HiGHS' status on the same LPs, App. C's
certificate conditions written out by hand, Farkas' lemma (a certificate bounds
every feasible point's constraint values into a contradiction), closed forms on a
2-variable LP, and no certificate on feasible bounded LPs."""
import numpy as np
import pytest
import scipy.optimize as so

import lpgen
from oracle import pdlp_oracle as O
from tests import lp_helpers as H

INF = np.inf


def _highs_status(inst):
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
    return r.status  # 0 optimal, 2 infeasible, 3 unbounded


def primal_infeasible_lp(seed):
    """A feasible random LP plus two rows a'x >= t + 1 and a'x <= t."""
    rng = np.random.default_rng(seed)
    inst, _, _ = H.lp_with_feasible_pair(rng, 25, 40)
    a = rng.standard_normal(inst.n)
    A = np.vstack([inst.scipy_csr().toarray(), a, a])
    t = rng.uniform(-2, 2)
    return H.make_lp(A, inst.c, np.r_[inst.lc, t + 1.0, -INF], np.r_[inst.uc, INF, t],
                     inst.lv, inst.uv, name="primal-infeasible")


def unbounded_lp(seed):
    """A feasible random LP plus a variable with only a lower bound, cost -1 and an
    empty column (so the LP is unbounded along it)."""
    rng = np.random.default_rng(seed)
    inst, _, _ = H.lp_with_feasible_pair(rng, 25, 40)
    A = np.hstack([inst.scipy_csr().toarray(), np.zeros((inst.m, 1))])
    return H.make_lp(A, np.r_[inst.c, -1.0], inst.lc, inst.uc, np.r_[inst.lv, 0.0],
                     np.r_[inst.uv, INF], name="unbounded")


def _check_primal_certificate(inst, y, eps=1e-9):
    """App. C by hand: y in Y, r in R with A'y + r ~ 0 chosen as the best r, positive
    dual objective of (y, r) and the ratio test."""
    lf, uf = np.isfinite(inst.lc), np.isfinite(inst.uc)
    assert np.all(y[lf & ~uf] >= 0) and np.all(y[~lf & uf] <= 0) and np.all(y[~lf & ~uf] == 0)
    q = inst.scipy_csr().T @ y
    vf, wf = np.isfinite(inst.lv), np.isfinite(inst.uv)
    r = np.where(vf & wf, -q, np.where(vf, np.maximum(-q, 0), np.where(wf, np.minimum(-q, 0), 0.0)))
    obj = 0.0
    for i in range(inst.m):
        obj += inst.lc[i] * y[i] if y[i] > 0 else (inst.uc[i] * y[i] if y[i] < 0 else 0.0)
    for j in range(inst.n):
        obj += inst.lv[j] * r[j] if r[j] > 0 else (inst.uv[j] * r[j] if r[j] < 0 else 0.0)
    assert obj > 0
    assert np.max(np.abs(q + r)) <= eps * obj
    return obj


def _check_ray(inst, x, eps=1e-9):
    """App. C by hand: x in the recession cone of the box, s in S-bar with Ax + s ~ 0,
    c'x < 0 and the ratio test."""
    vf, wf = np.isfinite(inst.lv), np.isfinite(inst.uv)
    assert np.all(x[vf & wf] == 0) and np.all(x[vf & ~wf] >= 0) and np.all(x[~vf & wf] <= 0)
    p = inst.scipy_csr() @ x
    lf, uf = np.isfinite(inst.lc), np.isfinite(inst.uc)
    s = np.where(lf & uf, 0.0, np.where(uf, np.maximum(-p, 0), np.where(lf, np.minimum(-p, 0), -p)))
    cx = float(inst.c @ x)
    assert cx < 0
    assert np.max(np.abs(p + s)) <= eps * abs(cx)


def test_bound_driven_infeasibility_closed_form():
    """x1 <= 1 as a row, x1 >= 2 as a bound: y = -1 gives A'y = -1, r = proj_R(1) = 1
    (only a lower bound: R^+), A'y + r = 0, and objective -uc y^- + lv r^+ = -1 + 2 = 1:
    the certificate's objective is positive only through the reduced-cost term."""
    b = H.make_lp([[1.0]], [0.0], [-INF], [1.0], [2.0], [INF])
    yb, obj, res = O.primal_infeasibility_measures(b, b.scipy_csr(), np.array([-1.0]))
    assert obj == 1.0 and res == 0.0
    r = O.solve(b, O.Params(max_iters=5000))
    assert r.status == O.PRIMAL_INFEASIBLE and _highs_status(b) == 2
    _check_primal_certificate(b, r.y)


def test_two_variable_closed_forms():
    """x1 + x2 >= 3 and x1 + x2 <= 1 over x >= 0: the direction y = (1, -1) gives
    A'y = 0, r = 0 and objective 3 - 1 = 2.  min -x1 s.t. x1 - x2 <= 1, x >= 0: the ray
    x = (1, 1) gives Ax = 0 and c'x = -1."""
    p = H.make_lp([[1, 1], [1, 1]], [1, 1], [3, -INF], [INF, 1], [0, 0], [INF, INF])
    yb, obj, res = O.primal_infeasibility_measures(p, p.scipy_csr(), np.array([1.0, -1.0]))
    assert obj == 2.0 and res == 0.0 and np.array_equal(yb, [1.0, -1.0])
    # a wrong-signed direction is projected onto Y: (-1, 1) -> (0, 0)
    yb, obj, res = O.primal_infeasibility_measures(p, p.scipy_csr(), np.array([-1.0, 1.0]))
    assert np.array_equal(yb, [0.0, 0.0]) and obj == 0.0
    d = H.make_lp([[1, -1]], [-1, 0], [-INF], [1], [0, 0], [INF, INF])
    xb, cx, res = O.dual_infeasibility_measures(d, d.scipy_csr(), np.array([1.0, 1.0]))
    assert cx == -1.0 and res == 0.0
    # (2, 1) is not a ray: A x = 1 > 0 would leave x1 - x2 <= 1, and S-bar = R^+ on that
    # row forces A x = -s <= 0, so the residual is 1
    xb, cx, res = O.dual_infeasibility_measures(d, d.scipy_csr(), np.array([2.0, 1.0]))
    assert cx == -2.0 and res == 1.0
    r1 = O.solve(p, O.Params(max_iters=5000))
    assert r1.status == O.PRIMAL_INFEASIBLE and _highs_status(p) == 2
    _check_primal_certificate(p, r1.y)
    r2 = O.solve(d, O.Params(max_iters=5000))
    assert r2.status == O.DUAL_INFEASIBLE and _highs_status(d) == 3
    _check_ray(d, r2.x)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_primal_infeasible_lps(seed):
    inst = primal_infeasible_lp(seed)
    assert _highs_status(inst) == 2
    res = O.solve(inst, O.Params(max_iters=100000))
    assert res.status == O.PRIMAL_INFEASIBLE
    obj = _check_primal_certificate(inst, res.y)
    # Farkas: every x in the box has A x outside [lc, uc] somewhere, because
    # y'(A x) = -r'x <= (lv'r+ - uv'r-) ... so y'(Ax) < lc'y+ - uc'y- for feasible-box x;
    # check it on random points of the box
    rng = np.random.default_rng(seed)
    lo = np.where(np.isfinite(inst.lv), inst.lv, -1e3)
    hi = np.where(np.isfinite(inst.uv), inst.uv, 1e3)
    A = inst.scipy_csr()
    y = res.y
    bound = sum(inst.lc[i] * y[i] if y[i] > 0 else (inst.uc[i] * y[i] if y[i] < 0 else 0.0)
                for i in range(inst.m))
    for _ in range(20):
        x = rng.uniform(lo, hi)
        assert y @ (A @ x) < bound + 1e-6 * obj * (1 + np.abs(x).max())


@pytest.mark.parametrize("seed", [4, 5])
def test_unbounded_lps(seed):
    inst = unbounded_lp(seed)
    assert _highs_status(inst) == 3
    res = O.solve(inst, O.Params(max_iters=100000))
    assert res.status == O.DUAL_INFEASIBLE
    _check_ray(inst, res.x)


def test_no_certificate_on_feasible_lps():
    """Feasible bounded LPs end OPTIMAL with detection on, and the three candidate
    directions at every check of the first 2000 iterations never pass either test."""
    for inst in (lpgen.config0(), H.lp_with_feasible_pair(np.random.default_rng(9), 40, 70)[0]):
        res = O.solve(inst, O.Params(eps_rel_kkt=1e-8))
        assert res.status == O.OPTIMAL
        lp = O.precondition(inst)
        seen = []

        def spy(cands):
            out = O.infeasibility_certificate(
                inst, lp.A_orig, [(lp.d2 * cx, lp.d1 * cy) for cx, cy in cands], 1e-9)
            seen.append(out)
            return None
        run = O.PdlpRun(lp, O.Params(), O.proj_box(np.zeros(inst.n), lp.lv, lp.uv),
                        np.zeros(inst.m), O.initial_primal_weight(lp.c, lp.lc, lp.uc),
                        1.0 / np.max(np.abs(lp.A.data)), lambda xs, ys: False, 2000, infeas=spy)
        run.run()
        assert len(seen) >= 2000 // 64 and all(s is None for s in seen)


def test_detection_off_runs_to_the_limit():
    inst = primal_infeasible_lp(1)
    res = O.solve(inst, O.Params(max_iters=3000, detect_infeasibility=False))
    assert res.status == O.ITERATION_LIMIT
