"""Feasibility polishing (Sec. 5, Algorithm 4) on the CUDA path against the oracle.

The pause schedule and each phase's outcome (iterations, success) must be the
oracle's exactly: they are integer decisions taken on quantities that agree to
about 1e-10 relative.  The returned pair must meet the paper's criteria (l_inf
residuals <= 1e-8, relative gap of Eq. (8) <= 1e-2) as measured by the oracle's
FP64 definitions, and its objective must agree with the oracle's to 1e-6 relative
(the tolerance of the plain full-solve parity test)."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import gpu_helpers as GH
from tests import lp_helpers as H

pytestmark = pytest.mark.gpu

CRIT = dict(termination_mode=1, eps_abs_feas=1e-8, eps_rel_gap=1e-2, max_iters=30000)


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


def _instance(name):
    if name == "config0":
        return lpgen.config0()
    if name == "mixed_bounds":
        return H.lp_with_feasible_pair(np.random.default_rng(21), 300, 500, density=0.05)[0]
    if name == "edge":
        return GH.edge_instance()
    return lpgen.config1(scale=0.002)


@pytest.mark.parametrize("name", ["config0", "mixed_bounds", "edge", "powerlaw"])
def test_polished_solve_matches_oracle(pkg, name):
    inst = _instance(name)
    ref = O.solve(inst, O.Params(feasibility_polishing=True, **CRIT))
    got = pkg.solve_instance(inst, device=True, feasibility_polishing=1, **CRIT)
    assert ref.status == O.OPTIMAL
    assert got.status == 0, got.stats
    lg, lr = got.stats["polish"], ref.stats["polish"]
    print(name, [(e["k"], e["primal_iters"], e["dual_iters"], e["accepted"]) for e in lg])
    assert len(lg) == len(lr) == got.stats["polish_pauses"]
    for a, b in zip(lg, lr):
        for key in ("k", "primal_iters", "primal_ok", "dual_iters", "dual_ok", "accepted"):
            assert a[key] == b[key], (key, a, b)
        assert abs(a["paper_gap"] - b["paper_gap"]) <= 1e-6 * b["paper_gap"] + 1e-13
    assert got.stats["iterations"] == ref.stats["iterations"]
    assert got.stats["polish_accepted_k"] == lr[-1]["k"]
    assert got.stats["polish_primal_iters"] == ref.stats["polish_primal_iters"]
    assert got.stats["polish_dual_iters"] == ref.stats["polish_dual_iters"]
    x, y = got.x.cpu().numpy(), got.y.cpu().numpy()
    st = O.kkt_stats(inst, inst.scipy_csr(), x, y)
    assert st["primal_res_inf"] <= 1e-8 and st["dual_res_inf"] <= 1e-8
    assert st["paper_gap"] <= 1e-2
    assert abs(st["pobj"] - ref.stats["pobj"]) <= 1e-6 * abs(ref.stats["pobj"])
    assert got.stats["gap_failures"] == 0


def test_polishing_off_keeps_the_plain_path(pkg):
    """Polishing off: same iterations and objective as before (no pause, empty log)."""
    inst = lpgen.config0()
    a = pkg.solve_instance(inst, device=True, **CRIT)
    ref = O.solve(inst, O.Params(**CRIT))
    assert a.stats["polish_pauses"] == 0 and "polish" not in a.stats
    assert a.stats["iterations"] == ref.stats["iterations"]
    assert a.status == ref.status


def test_polished_fp32_bulk_meets_paper_criteria(pkg):
    """FP32 bulk arithmetic in normal PDLP, FP64 in the polishing phases: the returned
    pair meets the paper's criteria (1e-8 l_inf residuals, measured in FP64 by the
    oracle), which the FP32 iteration alone cannot reach."""
    inst = GH.edge_instance()
    got = pkg.solve_instance(inst, device=True, feasibility_polishing=1, precision=pkg.FP32_BULK,
                             **CRIT)
    print("fp32+polish", got.stats["iterations"], got.stats["polish_primal_iters"],
          got.stats["polish_dual_iters"], got.stats.get("polish"))
    assert got.status == 0, got.stats
    assert got.stats["polish_accepted_k"] > 0
    st = O.kkt_stats(inst, inst.scipy_csr(), got.x.cpu().numpy(), got.y.cpu().numpy())
    assert st["primal_res_inf"] <= 1e-8 and st["dual_res_inf"] <= 1e-8
    assert st["paper_gap"] <= 1e-2
    plain = pkg.solve_instance(inst, device=True, precision=pkg.FP32_BULK,
                               **dict(CRIT, max_iters=got.stats["iterations"]))
    assert plain.status != 0
