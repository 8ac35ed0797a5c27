"""Pins of the oracle's feasibility polishing (Sec. 5, Algorithm 4) against facts the
paper and the mathematics fix: the two feasibility problems, the distance property of
PDHG that polishing relies on (Sec. 5, second insight; App. C), the pause schedule and
phase budgets of Algorithm 4, and the result against a second LP solver."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import lp_helpers as H
from tests.test_oracle_pins import _highs

NEVER = lambda xs, ys: False  # noqa: E731


def _identity_lp(inst):
    return O.precondition(inst, ruiz_iters=0, pc_alpha=0.0)


def test_feasibility_problems_of_sec5():
    """Primal problem: objective 0, constraints unchanged.  Dual problem (as an LP):
    every finite bound becomes 0 and infinite bounds stay, so the sign sets Y and R
    (which bounds are finite) are unchanged and the dual objective vanishes."""
    inst, _, _ = H.lp_with_feasible_pair(np.random.default_rng(1), 12, 20)
    lp = _identity_lp(inst)
    lp_p = O.primal_feasibility_lp(lp)
    assert np.all(lp_p.c == 0.0)
    for f in ("lc", "uc", "lv", "uv"):
        assert np.array_equal(getattr(lp_p, f), getattr(lp, f))
    assert lp_p.A is lp.A and lp_p.AT is lp.AT
    lp_d = O.dual_feasibility_lp(lp)
    assert np.array_equal(lp_d.c, lp.c)
    for f in ("lc", "uc", "lv", "uv"):
        v, w = getattr(lp, f), getattr(lp_d, f)
        assert np.array_equal(np.isfinite(v), np.isfinite(w))
        assert np.all(w[np.isfinite(w)] == 0.0)
        assert np.array_equal(w[~np.isfinite(v)], v[~np.isfinite(v)])
    # the source instance is untouched
    assert np.any(lp.c != 0.0) and np.any(np.isfinite(lp.lc) & (lp.lc != 0.0))


def _m_dist2(A, x, y, xs, ys, tau, sigma):
    """||z - z*||^2 in the norm of PDHG with K = -A (App. B):
    ||dx||^2/tau + 2 dy'A dx + ||dy||^2/sigma, positive definite for tau sigma ||A||^2 < 1."""
    dx, dy = x - xs, y - ys
    return dx @ dx / tau + 2.0 * dy @ (A @ dx) + dy @ dy / sigma


@pytest.mark.parametrize("seed", [3, 4])
def test_phases_never_move_away_from_their_saddle_points(seed):
    """Sec. 5, second insight: PDHG's distance (in its own norm) to any saddle point
    never grows.  (x_F, 0) is a saddle point of the primal feasibility problem for
    every feasible x_F, and (0, y_F) one of the dual feasibility problem for every dual
    feasible y_F; both phases, run with a fixed step eta < 1/||A||_2 and no restarts,
    must therefore never move away from them."""
    rng = np.random.default_rng(seed)
    inst, x_F, y_F = H.lp_with_feasible_pair(rng, 15, 25)
    lp = _identity_lp(inst)
    A = inst.scipy_csr().toarray()
    eta = 0.9 / np.linalg.norm(A, 2)
    omega = 0.7
    tau, sigma = eta / omega, eta * omega
    prm = O.Params(fixed_step=eta, fixed_omega=omega, restarts=False)
    K = 400
    for lp_phase, x_s, y_s, x_start, y_start in (
            (O.primal_feasibility_lp(lp), x_F, np.zeros(inst.m),
             rng.uniform(-3, 3, inst.n).clip(inst.lv, inst.uv), np.zeros(inst.m)),
            (O.dual_feasibility_lp(lp), np.zeros(inst.n), y_F,
             np.zeros(inst.n), rng.standard_normal(inst.m))):
        run = O.PdlpRun(lp_phase, prm, x_start, y_start, omega, eta, NEVER, K, trace_iters=K)
        run.run()
        d = [_m_dist2(A, x_start, y_start, x_s, y_s, tau, sigma)]
        d += [_m_dist2(A, r["x"], r["y"], x_s, y_s, tau, sigma) for r in run.trace]
        d = np.array(d)
        assert d[0] > 0
        assert np.all(np.diff(d) <= 1e-12 * d[0]), np.max(np.diff(d))
        assert d[-1] < d[0]  # and it does move towards the feasible sets


def test_pause_resume_is_transparent():
    """Pausing a run at the Algorithm 4 pause points and resuming it gives the same
    trajectory, bit for bit, as one uninterrupted run."""
    inst = lpgen.config0()
    lp = O.precondition(inst)
    eta0 = 1.0 / np.max(np.abs(lp.A.data))
    om0 = O.initial_primal_weight(lp.c, lp.lc, lp.uc)
    x0 = O.proj_box(np.zeros(inst.n), lp.lv, lp.uv)
    prm = O.Params()
    a = O.PdlpRun(lp, prm, x0, np.zeros(inst.m), om0, eta0, NEVER, 900)
    out_a = a.run()
    b = O.PdlpRun(lp, prm, x0, np.zeros(inst.m), om0, eta0, NEVER, 900)
    for k in (100, 200, 400, 800):
        assert b.run(pause_at=k) is None and b.k == k
    out_b = b.run()
    assert out_a[0] == out_b[0] == O.ITERATION_LIMIT
    assert np.array_equal(out_a[1], out_b[1]) and np.array_equal(out_a[2], out_b[2])
    assert a.stats == b.stats and a.omega == b.omega and a.eta_hat == b.eta_hat


def _criteria_by_hand(inst, x, y):
    """The paper's polishing termination criteria (Sec. 7, Eq. (9) and the relative
    gap of Eq. (8)) written out with the reduced-cost rule of Sec. 2."""
    A = inst.scipy_csr().toarray()
    ax = A @ x
    pres = np.maximum(inst.lc - ax, 0) + np.maximum(ax - inst.uc, 0)
    g = inst.c - A.T @ y
    lf, uf = np.isfinite(inst.lv), np.isfinite(inst.uv)
    r = np.where(lf & uf, g, np.where(lf, np.maximum(g, 0), np.where(uf, np.minimum(g, 0), 0.0)))
    dres = g - r
    pobj = inst.c @ x
    dobj = 0.0
    for i in range(inst.m):
        if y[i] > 0:
            dobj += inst.lc[i] * y[i]
        elif y[i] < 0:
            dobj += inst.uc[i] * y[i]
    for j in range(inst.n):
        if r[j] > 0:
            dobj += inst.lv[j] * r[j]
        elif r[j] < 0:
            dobj += inst.uv[j] * r[j]
    return np.max(pres), np.max(np.abs(dres)), pobj, dobj


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_polished_solution_meets_paper_criteria_and_brackets_highs(seed):
    """Algorithm 4 with the experiments' criteria (l_inf residuals <= 1e-8, relative gap
    of Eq. (8) <= 1e-2): the returned pair meets them, checked by hand, and weak
    duality puts HiGHS' optimum between its dual and primal objectives."""
    inst, _, _ = H.lp_with_feasible_pair(np.random.default_rng(seed), 30, 50)
    prm = O.Params(termination_mode=1, eps_abs_feas=1e-8, eps_rel_gap=1e-2,
                   feasibility_polishing=True, max_iters=200000)
    res = O.solve(inst, prm)
    assert res.status == O.OPTIMAL
    pinf, dinf, pobj, dobj = _criteria_by_hand(inst, res.x, res.y)
    assert pinf <= 1e-8 and dinf <= 1e-8
    assert abs(pobj - dobj) <= 1e-2 * (abs(pobj) + abs(dobj))
    opt = _highs(inst)
    slack = 1e-6 * (1.0 + abs(opt))  # residuals of 1e-8 times modest multipliers
    assert dobj - slack <= opt <= pobj + slack


def test_pause_schedule_and_phase_budgets():
    """Algorithm 4's schedule: pauses after k = 100, 200, 400, ... iterations; a phase
    runs at most k/8 iterations; the dual phase runs only after a successful primal
    phase; only the last pause can be accepted, and the status is then OPTIMAL."""
    for inst in (lpgen.config0(),
                 H.lp_with_feasible_pair(np.random.default_rng(8), 40, 70)[0]):
        prm = O.Params(termination_mode=1, feasibility_polishing=True, max_iters=200000)
        res = O.solve(inst, prm)
        log = res.stats["polish"]
        assert res.status == O.OPTIMAL and log
        assert [e["k"] for e in log] == [100 * 2 ** j for j in range(len(log))]
        for e in log:
            assert e["primal_iters"] <= e["k"] // 8 and e["dual_iters"] <= e["k"] // 8
            if not e["primal_ok"]:
                assert e["dual_iters"] == 0 and not e["accepted"]
            if e["paper_gap"] >= prm.eps_rel_gap:
                assert e["primal_iters"] == 0
        assert all(not e["accepted"] for e in log[:-1])
        if log[-1]["accepted"]:
            assert res.stats["iterations"] == log[-1]["k"]
        assert res.stats["polish_primal_iters"] == sum(e["primal_iters"] for e in log)


def test_polishing_off_is_plain_pdlp():
    """With polishing off the solve is Algorithm 1 alone (no pause, no log)."""
    inst = lpgen.config0()
    a = O.solve(inst, O.Params(termination_mode=1, max_iters=3000))
    assert "polish" not in a.stats
