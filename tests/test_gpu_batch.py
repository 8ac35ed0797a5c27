"""Batched solve of LPs of uneven sizes (pdlp_solve_batch): every LP runs the whole
method with its own step sizes, primal weight, restarts and termination, so each
result must equal, bit for bit, the result of solving that LP alone (the path is
deterministic and the batch only changes which stream runs it), and agree with the
oracle's objective as in the single-LP parity tests."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import gpu_helpers as GH
from tests import test_oracle_infeasibility as PI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


def _batch():
    lps = [lpgen.uneven_lp(lpgen.config_seed(2) * 4096 + 7000 + k, m_lo=150, m_hi=600)
           for k in range(6)]
    return [lpgen.config0(), GH.edge_instance()] + lps


@pytest.mark.parametrize("concurrency", [1, 4, 16])
def test_batch_equals_single_solves(pkg, concurrency):
    insts = _batch()
    got = pkg.solve_batch(insts, concurrency=concurrency, eps_rel_kkt=1e-8)
    for inst, r in zip(insts, got):
        one = pkg.solve_instance(inst, eps_rel_kkt=1e-8)
        assert r.status == one.status == 0, (inst.name, r.status)
        assert np.array_equal(r.x, one.x) and np.array_equal(r.y, one.y), inst.name
        assert r.stats["iterations"] == one.stats["iterations"]


def test_batch_objectives_match_oracle(pkg):
    insts = _batch()[2:6]
    got = pkg.solve_batch(insts, device=True, eps_rel_kkt=1e-8)
    for inst, r in zip(insts, got):
        ref = O.solve(inst, O.Params(eps_rel_kkt=1e-8))
        assert r.status == ref.status == O.OPTIMAL
        own = O.kkt_stats(inst, inst.scipy_csr(), r.x.cpu().numpy(), r.y.cpu().numpy())
        assert own["rel_kkt"] <= 1.01e-8
        assert abs(own["pobj"] - ref.stats["pobj"]) <= 1e-6 * abs(ref.stats["pobj"])


def test_batch_mixed_statuses_and_a_bad_problem(pkg):
    """One LP per outcome: optimal, primal infeasible, unbounded, iteration limit, and an
    invalid matrix (column index out of range), which fails alone."""
    bad = lpgen.config0()
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[5] = bad.n + 3
    insts = [lpgen.config0(), PI.primal_infeasible_lp(1), PI.unbounded_lp(4), GH.edge_instance(),
             bad]
    got = pkg.solve_batch(insts, concurrency=3, max_iters=100000)
    assert got[0].status == 0
    assert got[1].status == O.PRIMAL_INFEASIBLE
    assert got[2].status == O.DUAL_INFEASIBLE
    assert got[4].status == -1 and "problem 4" in got[4].stats.get("error", "")
    lim = pkg.solve_batch([GH.edge_instance()], max_iters=50)
    assert lim[0].status == O.ITERATION_LIMIT and lim[0].stats["iterations"] == 50
