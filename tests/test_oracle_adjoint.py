"""Pins of the oracle's adjoint of unrolled PDHG (K steps of Eq. (3) with fixed step
sizes) against things outside it: central finite differences of the forward map along
valid directions for every parameter group, the closed forms of LP sensitivity at a
nondegenerate optimum (d obj/dc = x*, d obj/d lc = y*+, d obj/d uc = -y*-; the
hand-solved golden LP), and linearity of the vector-Jacobian product."""
import dataclasses
import json
import os

import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import lp_helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _off_zero_bounds(inst, rng):
    """Variable bounds away from 0 so that the start proj_X(0) = 0 is strictly inside
    (a kink exactly at the evaluation point would make the central difference average
    two one-sided slopes)."""
    lv = rng.uniform(-2.0, -0.5, inst.n)
    uv = rng.uniform(5.0, 10.0, inst.n)
    return dataclasses.replace(inst, lv=lv, uv=uv)


def _fd_cases(seed):
    rng = np.random.default_rng(seed)
    a = _off_zero_bounds(lpgen.random_lp(30, 60, 4, seed=seed), rng)
    b, _, _ = H.lp_with_feasible_pair(rng, 25, 45)  # one-sided, free rows and columns
    b = dataclasses.replace(b, lv=np.where(np.isfinite(b.lv), np.minimum(b.lv, -0.3), b.lv),
                            uv=np.where(np.isfinite(b.uv), np.maximum(b.uv, 0.3), b.uv))
    return [a, b]


def _loss(inst, K, eta, omega, gx, gy):
    x, y = O.unrolled_pdhg(inst, K, eta, omega)[K][:2]
    return float(gx @ x + gy @ y)


@pytest.mark.parametrize("seed", [5, 6])
def test_vjp_matches_central_differences(seed):
    """For L = gx'x_K + gy'y_K and every parameter group, the adjoint's directional
    derivative equals the central difference (h = 1e-6) along a random direction that
    keeps the LP valid: lc and uc alone only on inequality rows, b = lc = uc together on
    equality rows, finite bounds only."""
    for inst in _fd_cases(seed):
        rng = np.random.default_rng(seed + 100)
        A = inst.scipy_csr().toarray()
        eta = 0.9 / np.linalg.norm(A, 2)
        omega = 0.8
        K = 150
        gx, gy = rng.standard_normal(inst.n), rng.standard_normal(inst.m)
        _, _, g = O.unrolled_pdhg_vjp(inst, K, eta, omega, gx, gy)
        eq = inst.lc == inst.uc
        h = 1e-6
        dirs = {
            "c": ({"c": 1.0}, rng.standard_normal(inst.n), g["c"]),
            "lv": ({"lv": 1.0}, rng.standard_normal(inst.n) * np.isfinite(inst.lv), g["lv"]),
            "uv": ({"uv": 1.0}, rng.standard_normal(inst.n) * np.isfinite(inst.uv), g["uv"]),
            "lc": ({"lc": 1.0}, rng.standard_normal(inst.m) * (~eq & np.isfinite(inst.lc)), g["lc"]),
            "uc": ({"uc": 1.0}, rng.standard_normal(inst.m) * (~eq & np.isfinite(inst.uc)), g["uc"]),
            "b": ({"lc": 1.0, "uc": 1.0}, rng.standard_normal(inst.m) * eq, g["lc"] + g["uc"]),
        }
        for name, (keys, d, grad) in dirs.items():
            if not np.any(d):
                continue
            plus = dataclasses.replace(inst, **{k: getattr(inst, k) + h * d for k in keys})
            minus = dataclasses.replace(inst, **{k: getattr(inst, k) - h * d for k in keys})
            fd = (_loss(plus, K, eta, omega, gx, gy) - _loss(minus, K, eta, omega, gx, gy)) / (2 * h)
            an = float(grad @ d)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (inst.name, name, fd, an)


def test_sensitivity_closed_forms_at_the_optimum():
    """Unrolled to convergence on the hand-solved LP (unique, nondegenerate vertex):
    d obj/dc = x* (= x_K + J_c'c), d obj/d uc = -y*^- and d obj/d lc = y*^+ (no finite
    lower row bound here), to 1e-9."""
    with open(os.path.join(GOLDEN, "textbook_lp.json")) as f:
        gd = json.load(f)
    inf = float("inf")
    conv = lambda v: [inf if s == "inf" else (-inf if s == "-inf" else s) for s in v]  # noqa
    inst = H.make_lp(gd["A"], gd["c"], conv(gd["lc"]), conv(gd["uc"]), conv(gd["lv"]),
                     conv(gd["uv"]))
    A = inst.scipy_csr().toarray()
    xK, yK, g = O.unrolled_pdhg_vjp(inst, 3000, 0.9 / np.linalg.norm(A, 2), 1.0, inst.c,
                                    np.zeros(inst.m))
    xs, ys = np.array(gd["x_star"]), np.array(gd["y_star"])
    np.testing.assert_allclose(xK + g["c"], xs, atol=1e-9)
    np.testing.assert_allclose(g["uc"], -np.maximum(-ys, 0.0), atol=1e-9)
    np.testing.assert_allclose(g["lc"], 0.0, atol=1e-12)


def test_vjp_is_linear_in_the_upstream_gradient():
    inst = _fd_cases(7)[0]
    rng = np.random.default_rng(1)
    A = inst.scipy_csr().toarray()
    eta = 0.9 / np.linalg.norm(A, 2)
    u = [rng.standard_normal(inst.n), rng.standard_normal(inst.m)]
    v = [rng.standard_normal(inst.n), rng.standard_normal(inst.m)]
    _, _, gu = O.unrolled_pdhg_vjp(inst, 60, eta, 1.0, *u)
    _, _, gv = O.unrolled_pdhg_vjp(inst, 60, eta, 1.0, *v)
    _, _, gw = O.unrolled_pdhg_vjp(inst, 60, eta, 1.0, 2.0 * u[0] - v[0], 2.0 * u[1] - v[1])
    for k in gu:
        np.testing.assert_allclose(gw[k], 2.0 * gu[k] - gv[k], rtol=1e-10, atol=1e-10)


def test_forward_equals_the_solver_with_fixed_steps():
    """The differentiated forward map is the solver's own iteration with fixed step
    sizes, restarts off and no preconditioning (same iterates)."""
    inst = _fd_cases(8)[0]
    A = inst.scipy_csr().toarray()
    eta = 0.9 / np.linalg.norm(A, 2)
    traj = O.unrolled_pdhg(inst, 40, eta, 1.3)
    res = O.solve(inst, O.Params(ruiz_iters=0, pc_alpha=0.0, fixed_step=eta, fixed_omega=1.3,
                                 restarts=False, max_iters=40, eps_rel_kkt=0.0,
                                 detect_infeasibility=False), trace_iters=40)
    for k, rec in enumerate(res.trace, start=1):
        np.testing.assert_array_equal(rec["x"], traj[k][0])
        np.testing.assert_array_equal(rec["y"], traj[k][1])
