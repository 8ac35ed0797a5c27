"""The persistent batch (pdlp_solve_batch_persistent): one launch, one CTA per LP at a
time, each LP running the whole method with its own step sizes, primal weight,
restarts and termination.  Its reductions run in another order than pdlp_solve's, so
it is held to the oracle with the single-LP tolerances: the returned point after 100
iterations within a relative 1e-10 of the oracle's (same restart decisions), and at
relative KKT 1e-8 the objective within 1e-6 with the oracle measuring the returned
point.  Every staging path of the gathered vectors is exercised (both in shared
memory, x' only, y' only, none)."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import gpu_helpers as GH
from tests import test_oracle_infeasibility as PI

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
TUNES = (1, 2, 3, 4, 5, 6)  # the launch configurations of pdlp_solve_batch_persistent
# every call is bounded on the device: the kernel tests its time limit at each check
BOUND = dict(time_limit_s=60.0, max_iters=200000)


def _solve(pkg, insts, **kw):
    args = dict(BOUND)
    args.update(kw)
    return pkg.solve_batch(insts, persistent=True, **args)


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


def _uneven(k, m_lo=150, m_hi=600):
    return lpgen.uneven_lp(lpgen.config_seed(2) * 4096 + 7000 + k, m_lo=m_lo, m_hi=m_hi)


def _large_uneven():
    """An LP whose x' (n = 26,000 entries: 208 KB in FP64) does not fit the 200 KB of
    shared memory while its y' does: the y'-only staging path in FP64, x'-only in FP32."""
    rng = np.random.default_rng(lpgen.config_seed(2) * 4096 + 9100)
    degrees = rng.integers(4, 13, size=26000).astype(np.int64)
    return lpgen._assemble(rng, 11000, 26000, degrees, lpgen._normal_values, eq_frac=0.3,
                           free_frac=0.0, name="uneven m=11000 n=26000")


def _rel_err(a, b):
    return float(np.max(np.abs(a - b))) / max(1.0, float(np.max(np.abs(b))))


@pytest.mark.parametrize("tune", TUNES)
def test_point_after_100_iterations_matches_oracle(pkg, tune):
    """max_iters = 100 with the tolerance 0: the returned point is the restart candidate
    at k = 100, after the checks at 64 (and the (iii) restarts at 1, 2, 4, ...), which
    must all decide as the oracle's."""
    insts = [lpgen.config0(), GH.edge_instance()] + [_uneven(k) for k in range(3)]
    got = _solve(pkg, insts, tune=tune, max_iters=100, eps_rel_kkt=0.0)
    for inst, r in zip(insts, got):
        ref = O.solve(inst, O.Params(max_iters=100, eps_rel_kkt=0.0))
        assert r.status == ref.status == O.ITERATION_LIMIT, inst.name
        assert r.stats["iterations"] == 100
        assert list(r.stats["restarts"]) == list(ref.stats["restarts"]), inst.name
        e = max(_rel_err(r.x, ref.x), _rel_err(r.y, ref.y))
        assert e <= ITER_TOL, (inst.name, e)
        assert r.stats["tune"] == tune


def test_staging_paths_match_oracle(pkg):
    """The LP whose x' does not fit shared memory (y' staged in FP64 with 200 KB, neither
    with 100 KB), against the oracle after 100 iterations, and with staging off."""
    inst = _large_uneven()
    ref = O.solve(inst, O.Params(max_iters=100, eps_rel_kkt=0.0))
    for tune in (1, 2, 5):
        r = _solve(pkg, [inst], tune=tune, max_iters=100, eps_rel_kkt=0.0)[0]
        assert r.status == O.ITERATION_LIMIT
        e = max(_rel_err(r.x, ref.x), _rel_err(r.y, ref.y))
        assert e <= ITER_TOL, (tune, e)


def test_solves_match_oracle_objective(pkg):
    insts = [lpgen.config0(), GH.edge_instance()] + [_uneven(k) for k in range(4)]
    got = _solve(pkg, insts, eps_rel_kkt=1e-8)
    assert got[0].stats["tune"] in TUNES
    for inst, r in zip(insts, got):
        ref = O.solve(inst, O.Params(eps_rel_kkt=1e-8))
        assert r.status == ref.status == O.OPTIMAL, inst.name
        own = O.kkt_stats(inst, inst.scipy_csr(), r.x, r.y)
        assert own["rel_kkt"] <= 1.01e-8, (inst.name, own["rel_kkt"])
        assert abs(own["pobj"] - ref.stats["pobj"]) <= 1e-6 * abs(ref.stats["pobj"])
        assert abs(r.stats["rel_kkt"] - own["rel_kkt"]) <= 1e-9


# The device tests relative KKT 1e-6 in FP64 on the FP32 iterate and its FP32 products
# A x, A'y; the oracle forms those products exactly.  An FP32 product of a row with L
# entries differs from the exact one by at most ~L eps_32 sum |a_ij x_j| (eps_32 = 6e-8,
# L <= 40 here), which moves the measured residuals by a few 1e-9 relative: the oracle's
# measure is held to 1e-6 + 5e-8.
FP32_KKT_TOL = 1.05e-6


def test_fp32_bulk_meets_tolerance_in_fp64(pkg):
    """FP32 bulk with FP64 checks at the batch's tolerance (relative KKT 1e-6): the
    oracle's FP64 measures of the returned points meet it."""
    insts = [lpgen.config0()] + [_uneven(k) for k in range(4)] + [_large_uneven()]
    got = _solve(pkg, insts, precision=1, eps_rel_kkt=1e-6)
    for inst, r in zip(insts, got):
        assert r.status == O.OPTIMAL, (inst.name, r.status_name)
        own = O.kkt_stats(inst, inst.scipy_csr(), r.x, r.y)
        assert own["rel_kkt"] <= FP32_KKT_TOL, (inst.name, own["rel_kkt"])
        assert r.stats["rel_kkt"] <= 1e-6


def test_deterministic_and_independent_of_neighbours(pkg):
    """A fixed configuration gives bit-identical results run to run, and an LP's result
    does not depend on which other LPs share the launch."""
    insts = [lpgen.config0(), GH.edge_instance()] + [_uneven(k) for k in range(6)]
    a = _solve(pkg, insts, tune=1, eps_rel_kkt=1e-8)
    b = _solve(pkg, insts, tune=1, eps_rel_kkt=1e-8)
    c = _solve(pkg, insts[::-1][:4], tune=1, eps_rel_kkt=1e-8)[::-1]
    for ra, rb in zip(a, b):
        assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.y, rb.y)
    for ra, rc in zip(a[4:], c):
        assert np.array_equal(ra.x, rc.x) and np.array_equal(ra.y, rc.y)
        assert ra.stats["iterations"] == rc.stats["iterations"]


def test_statuses_and_a_bad_problem(pkg):
    """One LP per outcome: optimal, primal infeasible, unbounded, iteration limit, and an
    invalid matrix (column index out of range), which fails alone; device arrays."""
    bad = lpgen.config0()
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[5] = bad.n + 3
    insts = [lpgen.config0(), PI.primal_infeasible_lp(1), PI.unbounded_lp(4), bad]
    got = _solve(pkg, insts, device=True, max_iters=100000)
    assert got[0].status == 0
    assert got[1].status == O.PRIMAL_INFEASIBLE
    assert got[2].status == O.DUAL_INFEASIBLE
    assert got[3].status == -1 and "problem 3" in got[3].stats.get("error", "")
    # the certificates check out on the LP as given (App. C)
    y = got[1].y.cpu().numpy()
    cert = O.infeasibility_certificate(insts[1], insts[1].scipy_csr(), [(np.zeros(insts[1].n), y)],
                                       1e-9)
    assert cert is not None and cert[0] == O.PRIMAL_INFEASIBLE
    lim = _solve(pkg, [GH.edge_instance()], max_iters=50)
    assert lim[0].status == O.ITERATION_LIMIT and lim[0].stats["iterations"] == 50


def test_time_limit_and_rejected_arguments(pkg):
    r = _solve(pkg, [GH.edge_instance()], time_limit_s=0.0, detect_infeasibility=0)[0]
    assert r.status == O.TIME_LIMIT and r.stats["iterations"] == 64
    from paper_2501_07018_gb300.binding import PdlpError

    with pytest.raises(PdlpError):
        _solve(pkg, [lpgen.config0()], feasibility_polishing=1)
    with pytest.raises(PdlpError):
        _solve(pkg, [lpgen.config0()], tune=7)


def test_box_only_lp_and_empty_batch(pkg):
    """An LP without rows (A is 0 x n) has the closed-form solution x_j = lv_j for
    c_j > 0, uv_j for c_j < 0 (Sec. 2's box constraints alone); it solves in a batch with a
    regular LP.  An empty batch returns at once."""
    from tests import lp_helpers as H

    rng = np.random.default_rng(3)
    n = 700
    c = rng.uniform(-1.0, 1.0, n)
    lv, uv = rng.uniform(-5.0, 0.0, n), rng.uniform(0.0, 5.0, n)
    box = H.make_lp(np.zeros((0, n)), c, [], [], lv, uv, name="box-only")
    for prec in (0, 1):
        got = _solve(pkg, [box, lpgen.config0()], precision=prec,
                     eps_rel_kkt=1e-8 if prec == 0 else 1e-6)
        assert got[0].status == 0 and got[1].status == 0
        want = np.where(c > 0, lv, uv)
        # FP32 bulk holds the scaled bounds in FP32: the returned x is within their rounding
        assert np.allclose(got[0].x, want, rtol=0, atol=(1e-9 if prec == 0 else 1e-6) * 5.0)
        assert got[0].y.size == 0
    assert _solve(pkg, []) == []
