"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: iterates of the FP64 path track the oracle to a relative 1e-10 (infinity
norm, relative to max(1, |z|)) over the first 100 iterations; the objective at
relative KKT 1e-8 agrees to a relative 1e-6; component entry points (preconditioning,
normalized duality gap, KKT measures) agree to 1e-12 .. 1e-10 relative, which
bounds accumulated FP64 rounding of a few hundred reduction steps.
"""
import math

import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import gpu_helpers as GH

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-10
# The accepted step eta depends on eta_bar = ||dz||^2 / (2 |dy'(Ax' - Ax)|), a quotient
# whose denominator is a sum of products of differences of nearby quantities; ulp-level
# differences in summation order (tree vs sequential) are amplified by its conditioning,
# so eta is compared at 1e-9 while the iterates themselves keep the 1e-10 bound.
ETA_TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


def _trace_parity(pkg, inst, iters=100, **prm):
    res = pkg.solve_instance(inst, trace_iters=iters, max_iters=iters, eps_rel_kkt=0.0, **prm)
    ora = O.solve(inst, O.Params(max_iters=iters, eps_rel_kkt=0.0), trace_iters=iters)
    assert len(res.trace) == len(ora.trace) == iters
    errs = GH.trace_errors(res.trace, ora.trace)
    return res, ora, errs


def test_restart_schedules_in_closed_form(pkg):
    """The closed-form restart schedules the oracle is pinned to: (iii) alone restarts at
    k_{j+1} = ceil(k_j / (1 - beta_art)); an always-true (i) fires exactly at the checks
    and before (iii).  Exercises the host's look-ahead to the next (iii) iteration."""
    inst = lpgen.config0()
    iters = 300
    cases = []
    for beta_art, num, den in ((0.5, 2, 1), (0.25, 4, 3)):
        want, k = [], 1
        while k < iters:
            want.append((k, O.RESTART_ARTIFICIAL))
            k = -(-num * k // den)
        cases.append((dict(beta_suff=0.0, beta_nec=0.0, beta_art=beta_art), want))
    want = [(2 ** j, O.RESTART_ARTIFICIAL) for j in range(6)]
    want += [(k, O.RESTART_SUFFICIENT) for k in range(64, iters, 64)]
    cases.append((dict(beta_suff=1e300, beta_nec=0.0), want))
    for prm, want in cases:
        res = pkg.solve_instance(inst, trace_iters=iters, max_iters=iters, eps_rel_kkt=0.0,
                                 detect_infeasibility=0, **prm)
        got = [(r["k"], r["restart"]) for r in res.trace if r["restart"] != 0]
        assert got == want, prm


@pytest.mark.parametrize("case", ["paper_thresholds", "decay_bound", "strict_increase"])
def test_restart_criteria_i_ii_in_closed_form(pkg, case):
    """The closed-form schedules that pin criteria (i) and (ii) in the oracle (fixed-step
    PDHG on 1 x 1 equality-constrained LPs with a free variable, no preconditioning):
    (i) and (ii) at the paper's thresholds, (ii) held back by its decay bound, and (ii)
    needing a strict rise of the candidate gap.  The device's normalized gap must also
    equal the closed form mu = |a| ||(u, v)|| at every evaluation."""
    from tests import test_oracle_pins as P

    if case == "paper_thresholds":
        inst, iters, want = P.bilinear_instance(), 200, P.BILINEAR_SCHEDULE
        prm = dict(fixed_step=0.25, fixed_omega=4.0, check_period=10)
        cf = (1.0, 1.0, -1.0, 0.25, 4.0, 10, iters, 0.1, 0.9, 0.5)
    elif case == "decay_bound":
        inst, iters, want = P.bilinear_instance(), 200, P.SECOND_BILINEAR_SCHEDULE
        prm = dict(fixed_step=11 / 32, fixed_omega=4.0, check_period=3)
        cf = (1.0, 1.0, -1.0, 11 / 32, 4.0, 3, iters, 0.1, 0.9, 0.5)
    else:
        inst, iters, want = P.nilpotent_instance(), 40, P.NILPOTENT_SCHEDULE
        prm = dict(fixed_step=1.0, fixed_omega=1.0, check_period=3, beta_suff=-1.0, beta_art=0.9)
        cf = (1.0, 2.0, 1.0, 1.0, 1.0, 3, iters, -1.0, 0.9, 0.9)
    _, ev = P._bilinear_1x1_schedule(*cf)
    res = pkg.solve_instance(inst, trace_iters=iters, max_iters=iters, eps_rel_kkt=-1.0,
                             ruiz_iters=0, pc_alpha=0.0, detect_infeasibility=0, **prm)
    got = [(r["k"], r["restart"]) for r in res.trace if r["restart"] != 0]
    assert got == want
    for r in res.trace:
        if r["k"] in ev:
            _, _, _, mc, ma = ev[r["k"]]
            # the iterates drift from the closed form by rounding (~1e-16 of |z| ~ 1), so
            # late, small gaps (1e-6) are compared to an absolute 1e-14
            assert r["mu_cur"] == pytest.approx(mc, rel=1e-9, abs=1e-14), r["k"]
            assert r["mu_avg"] == pytest.approx(ma, rel=1e-9, abs=1e-14), r["k"]


def test_fixed_step_and_weight_rejected_when_invalid(pkg):
    inst = lpgen.config0()
    for bad in (dict(fixed_step=-1.0), dict(fixed_omega=math.inf), dict(beta_art=math.nan),
                dict(beta_art=-0.5)):
        with pytest.raises(pkg.PdlpError) as ei:
            pkg.solve_instance(inst, max_iters=10, **bad)
        assert ei.value.code == -1, bad


@pytest.mark.parametrize("name", ["config0", "edge", "edge_long", "powerlaw", "mcf"])
def test_trace_parity_first_100_iterations(pkg, name):
    """Iterates, accepted steps and restart decisions of the first 100 iterations.
    ``edge_long`` has a row of A and a row of A' that span several chunks of the
    long-row path (chunk sums combined by the last chunk to finish)."""
    if name == "config0":
        inst = lpgen.config0()
    elif name == "edge":
        inst = GH.edge_instance()
    elif name == "edge_long":
        inst = GH.edge_instance(seed=12, m=12000, n=24000, dense_row_nnz=20000,
                                dense_col_nnz=10000)
    elif name == "mcf":  # multicommodity flow: equality and capacity rows, hub rows of A
        inst = lpgen.multicommodity_flow_lp(200, 2000, 10, seed=7)
    else:
        inst = lpgen.config1(scale=0.002)
    res, ora, errs = _trace_parity(pkg, inst)
    worst = max(e["ez"] for e in errs)
    prof = [max(e["ez"] for e in errs[i:i + 10]) for i in range(0, len(errs), 10)]
    print(f"{name}: max relative iterate error per 10 iterations: "
          + " ".join(f"{v:.1e}" for v in prof))
    bad = [e for e in errs if not e["restart_same"]]
    assert not bad, f"restart decisions differ first at k={bad[0]['k']}: {bad[0]}"
    assert worst <= TRACE_TOL, max(errs, key=lambda e: e["ez"])
    assert max(e["eeta"] for e in errs) <= ETA_TOL
    # mu values at the evaluated iterations
    for e in errs:
        gc, oc, ga, oa = e["mu"]
        if not math.isnan(oc):
            assert abs(gc - oc) <= 1e-9 * max(1e-12, abs(oc)) + 1e-14
            assert abs(ga - oa) <= 1e-9 * max(1e-12, abs(oa)) + 1e-14


def _named_instance(name):
    if name == "config0":
        return lpgen.config0()
    if name == "edge":
        return GH.edge_instance()
    if name == "edge_long":
        return GH.edge_instance(seed=12, m=12000, n=24000, dense_row_nnz=20000,
                                dense_col_nnz=10000)
    if name == "mcf":
        return lpgen.multicommodity_flow_lp(200, 2000, 10, seed=7)
    return lpgen.config1(scale=0.002)


@pytest.mark.parametrize("name", ["config0", "edge", "edge_long", "powerlaw", "mcf"])
def test_returned_point_parity_without_trace(pkg, name):
    """The production path (no trace: many step attempts launched between the
    iterations where the host reads the device state) returns, at the 100-iteration
    limit, the oracle's candidate point (unscaled) to the trace tolerance, with the
    same restarts."""
    inst = _named_instance(name)
    res = pkg.solve_instance(inst, max_iters=100, eps_rel_kkt=0.0)
    ora = O.solve(inst, O.Params(max_iters=100, eps_rel_kkt=0.0))
    assert res.status == ora.status == O.ITERATION_LIMIT
    assert res.stats["restarts"] == list(ora.stats["restarts"])
    zo = np.concatenate([ora.x, ora.y])
    zg = np.concatenate([res.x, res.y])
    err = float(np.max(np.abs(zg - zo))) / max(1.0, float(np.max(np.abs(zo))))
    assert err <= TRACE_TOL, err


@pytest.mark.parametrize("name", ["config0", "edge"])
def test_solve_objective_at_rel_kkt_1e8(pkg, name):
    """Full solve to relative KKT 1e-8: same objective as the oracle (relative 1e-6),
    and the oracle's own measures of the returned point confirm the tolerance."""
    inst = lpgen.config0() if name == "config0" else GH.edge_instance()
    res = pkg.solve_instance(inst, eps_rel_kkt=1e-8)
    assert res.status == 0, res.status_name
    ref = O.solve(inst, O.Params(eps_rel_kkt=1e-8))
    assert ref.status == O.OPTIMAL
    assert abs(res.stats["pobj"] - ref.stats["pobj"]) <= 1e-6 * abs(ref.stats["pobj"])
    own = O.kkt_stats(inst, inst.scipy_csr(), res.x, res.y)
    assert own["rel_kkt"] <= 1.01e-8
    assert abs(own["pobj"] - res.stats["pobj"]) <= 1e-9 * abs(own["pobj"])
    assert np.all(res.x >= inst.lv) and np.all(res.x <= inst.uv)
    assert res.stats["gap_failures"] == 0, res.stats.get("gap_failure_message")
    # the call's device memory: at least the staged CSR (12 B per entry) and the vectors
    assert res.stats["device_bytes"] >= 12 * inst.nnz + 8 * 5 * (inst.m + inst.n)


def test_host_and_device_inputs_identical(pkg):
    import torch

    inst = lpgen.config0()
    a = pkg.solve_instance(inst, max_iters=500, eps_rel_kkt=0.0)
    b = pkg.solve_instance(inst, device=True, max_iters=500, eps_rel_kkt=0.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.x, b.x.cpu().numpy())
    np.testing.assert_array_equal(a.y, b.y.cpu().numpy())
    assert a.stats["iterations"] == b.stats["iterations"] == 500


def test_repeatable_bit_for_bit(pkg):
    inst = GH.edge_instance()
    a = pkg.solve_instance(inst, max_iters=300, eps_rel_kkt=0.0)
    b = pkg.solve_instance(inst, max_iters=300, eps_rel_kkt=0.0)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.y, b.y)


def test_precondition_parity(pkg):
    """D1, D2 and A~ = D1 A D2 of Sec. 3's preconditioner (10 Ruiz + Pock-Chambolle)."""
    for inst in (lpgen.config0(), GH.edge_instance(), lpgen.config1(scale=0.002)):
        d1, d2, sv = pkg.precondition(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val)
        lp = O.precondition(inst)
        np.testing.assert_allclose(d1, lp.d1, rtol=1e-13)
        np.testing.assert_allclose(d2, lp.d2, rtol=1e-13)
        np.testing.assert_allclose(sv, lp.A.data, rtol=1e-12)


def _rand_point(rng, inst):
    lv = np.where(np.isfinite(inst.lv), inst.lv, -5.0)
    uv = np.where(np.isfinite(inst.uv), inst.uv, 5.0)
    x = lv + (uv - lv) * rng.random(inst.n)
    mask = rng.random(inst.n) < 0.2
    x[mask] = np.where(rng.random(int(mask.sum())) < 0.5, lv[mask], uv[mask])
    y = rng.standard_normal(inst.m)
    y = np.where(~np.isfinite(inst.lc) & (y > 0), -y, y)
    y = np.where(~np.isfinite(inst.uc) & (y < 0), -y, y)
    y = np.where(~np.isfinite(inst.lc) & ~np.isfinite(inst.uc), 0.0, y)
    y[rng.random(inst.m) < 0.1] = 0.0
    return x, y


@pytest.mark.parametrize("name", ["config0", "edge", "powerlaw"])
def test_normalized_gap_parity(pkg, name):
    """mu(z, z_ref) of Sec. 3 from the GPU kernels vs the oracle's bisection."""
    inst = {"config0": lpgen.config0, "edge": GH.edge_instance,
            "powerlaw": lambda: lpgen.config1(scale=0.002)}[name]()
    lp = O.precondition(inst, ruiz_iters=0, pc_alpha=0.0)
    rng = np.random.default_rng(5)
    for trial in range(6):
        x, y = _rand_point(rng, inst)
        xr, yr = _rand_point(rng, inst)
        if trial == 4:
            xr, yr = x.copy(), y.copy()  # r = 0
        if trial == 5:
            xr = xr + 1e6  # far reference: ball contains the saturated point if bounded
        omega = float(np.exp(rng.uniform(-2, 2)))
        Ax, ATy = lp.A @ x, lp.AT @ y
        want = O.normalized_gap(lp, x, y, Ax, ATy, xr, yr, omega)
        got = pkg.normalized_gap(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val, inst.c,
                                 inst.lc, inst.uc, inst.lv, inst.uv, x, y, xr, yr, omega)
        assert abs(got - want) <= 1e-10 * max(abs(want), 1e-300) + 1e-15, (trial, got, want)


@pytest.mark.parametrize("reduced_costs", [0, 1])
def test_kkt_parity(pkg, reduced_costs):
    """Optimality measures with Sec. 2's reduced costs and with App. A's variant."""
    inst = GH.edge_instance()
    rng = np.random.default_rng(6)
    A = inst.scipy_csr()
    for _ in range(3):
        x, y = _rand_point(rng, inst)
        got = pkg.kkt(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val, inst.c, inst.lc,
                      inst.uc, inst.lv, inst.uv, x, y, reduced_costs=reduced_costs)
        want = O.kkt_stats(inst, A, x, y, reduced_costs=reduced_costs)
        for k in ("rel_kkt", "rel_primal", "rel_dual", "rel_gap", "primal_res_l2", "dual_res_l2",
                  "pobj", "dobj", "paper_gap"):
            assert abs(got[k] - want[k]) <= 1e-11 * max(1.0, abs(want[k])), k
        for k in ("primal_res_inf", "dual_res_inf"):
            assert abs(got[k] - want[k]) <= 1e-12 * max(1.0, abs(want[k])), k


def test_box_only_lp(pkg):
    """m = 0: x_i = lv_i if c_i > 0 else uv_i."""
    rng = np.random.default_rng(8)
    n = 3000
    lv = rng.uniform(-5, 0, n)
    uv = lv + rng.uniform(0.5, 3, n)
    c = rng.uniform(-1, 1, n)
    res = pkg.solve(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), c,
                    np.zeros(0), np.zeros(0), lv, uv, eps_rel_kkt=1e-12)
    assert res.status == 0
    np.testing.assert_allclose(res.x, np.where(c > 0, lv, uv), atol=1e-9)


def test_all_rows_empty_and_single_column(pkg):
    m, n = 5, 1
    res = pkg.solve(m, n, np.zeros(m + 1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                    np.array([1.0]), np.full(m, -1.0), np.full(m, 1.0), np.array([-2.0]),
                    np.array([3.0]), eps_rel_kkt=1e-10)
    assert res.status == 0
    assert abs(res.x[0] + 2.0) < 1e-9
    np.testing.assert_array_equal(res.y, np.zeros(m))


@pytest.mark.parametrize("mutation", ["unsorted", "col_range", "nan_c", "lc_gt_uc", "lv_inf",
                                      "row_ptr"])
def test_invalid_input_rejected(pkg, mutation):
    inst = lpgen.config0()
    rp, ci, va = inst.row_ptr.copy(), inst.col_idx.copy(), inst.val.copy()
    c, lc, uc, lv, uv = inst.c.copy(), inst.lc.copy(), inst.uc.copy(), inst.lv.copy(), inst.uv.copy()
    if mutation == "unsorted":
        b = rp[3]
        ci[b], ci[b + 1] = ci[b + 1], ci[b]
    elif mutation == "col_range":
        ci[10] = inst.n + 5
    elif mutation == "nan_c":
        c[4] = np.nan
    elif mutation == "lc_gt_uc":
        lc[7] = uc[7] + 1.0
    elif mutation == "lv_inf":
        lv[2] = np.inf
    elif mutation == "row_ptr":
        rp[5] = rp[6] + 1
    with pytest.raises(pkg.PdlpError) as ei:
        pkg.solve(inst.m, inst.n, rp, ci, va, c, lc, uc, lv, uv, max_iters=10)
    assert ei.value.code == -1


def test_fp32_bulk_reaches_1e4(pkg):
    """FP32 bulk: matrix, iterates and SpMV accumulation in FP32; FP64 KKT.  Reaches
    relative KKT 1e-4; objective error against the FP64 oracle stated and bounded."""
    inst = lpgen.config0()
    res = pkg.solve_instance(inst, precision=pkg.FP32_BULK, eps_rel_kkt=1e-4)
    assert res.status == 0
    ref = O.solve(inst, O.Params(eps_rel_kkt=1e-10))
    own = O.kkt_stats(inst, inst.scipy_csr(), res.x, res.y)
    assert own["rel_kkt"] <= 1.5e-4
    assert abs(res.stats["pobj"] - ref.stats["pobj"]) <= 1e-3 * abs(ref.stats["pobj"])


@pytest.mark.slow
def test_full_size_powerlaw_first_iterations(pkg):
    """The 2M x 5M power-law LP at full size, in the bench's configuration: the first
    3 iterations (scaled iterates) against the oracle, on every coordinate."""
    inst = lpgen.config1()
    iters = 3
    res = pkg.solve_instance(inst, trace_iters=iters, max_iters=iters, eps_rel_kkt=0.0)
    ora = O.solve(inst, O.Params(max_iters=iters, eps_rel_kkt=0.0), trace_iters=iters)
    errs = GH.trace_errors(res.trace, ora.trace)
    assert all(e["restart_same"] for e in errs)
    assert max(e["ez"] for e in errs) <= TRACE_TOL, errs


@pytest.mark.parametrize("precision", [0, 1])
def test_every_gap_evaluation_resolves(pkg, precision):
    """Over 1500 iterations of the power-law shape (10% free columns, 40% equality
    rows), every normalized-gap evaluation of the restart scheme is resolved by the
    bracket search (no NaN fallback), in both precisions."""
    inst = lpgen.config1(scale=0.05)
    res = pkg.solve_instance(inst, max_iters=1500, eps_rel_kkt=0.0, precision=precision)
    st = res.stats
    assert st["gap_evals"] > 20
    assert st["gap_failures"] == 0, st.get("gap_failure_message")
