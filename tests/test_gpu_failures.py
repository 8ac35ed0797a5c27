"""Finished solves that end without meeting the tolerance, with the failure made on the
host side (a parameter or the input data), never on the GPU: the statuses
PDLP_TIME_LIMIT and PDLP_NUMERICAL_ERROR of Sec. 3's "Periodic checks" (termination is
also checked on a numerical error), each with x and y written."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import lp_helpers as H

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


def ones_lp():
    """4 x 4 all-ones matrix: the first step estimate 1/max|a_ij| = 1 exceeds the largest
    acceptable step (about 1/||A||_2 = 1/4), so Algorithm 2 rejects the first attempt."""
    return H.make_lp(np.ones((4, 4)), np.array([1.0, -1.0, 2.0, -2.0]),
                     np.array([1.0, -np.inf, 0.5, 0.0]), np.array([1.0, 3.0, np.inf, 5.0]),
                     np.zeros(4), 10.0 * np.ones(4))


@pytest.mark.parametrize("device", [False, True])
def test_time_limit_zero_stops_at_the_first_check(pkg, device):
    """time_limit_s = 0: the limit is tested at the periodic checks, so the solve stops at
    the first one (k = 64) with status TIME_LIMIT and the restart candidate written."""
    inst = lpgen.config0()
    res = pkg.solve_instance(inst, device=device, time_limit_s=0.0, detect_infeasibility=0)
    assert res.status == 2, res.status_name
    assert res.stats["iterations"] == 64
    x = res.x.cpu().numpy() if device else res.x
    y = res.y.cpu().numpy() if device else res.y
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(y))
    assert np.all(x >= inst.lv) and np.all(x <= inst.uv)
    # the same point the oracle's measures call far from optimal, but a real iterate
    st = O.kkt_stats(inst, inst.scipy_csr(), x, y)
    assert 0.0 < st["rel_kkt"] < 1.0


def test_step_retry_cap_gives_numerical_error(pkg):
    """max_step_retries = 1 on an LP whose first attempt Algorithm 2 rejects: the retry cap
    (read R16) ends the solve with NUMERICAL_ERROR before any accepted iteration, and
    the returned point is the start z^{0,0} = (proj_X(0), 0), as in the oracle."""
    inst = ones_lp()
    ora = O.solve(inst, O.Params(max_iters=100000, eps_rel_kkt=1e-8))
    assert O.solve(inst, O.Params(max_iters=2, eps_rel_kkt=0.0), trace_iters=2).trace[0]["attempts"] == 2
    ora1 = O.solve(inst, O.Params(max_iters=20, eps_rel_kkt=0.0, max_step_retries=1))
    assert ora1.status == O.NUMERICAL_ERROR and ora.status == O.OPTIMAL
    res = pkg.solve_instance(inst, max_iters=20, eps_rel_kkt=0.0, max_step_retries=1)
    assert res.status == 5, res.status_name
    assert res.stats["iterations"] == 0 and res.stats["rejected_steps"] == 1
    np.testing.assert_array_equal(res.x, ora1.x)
    np.testing.assert_array_equal(res.y, ora1.y)
    # with the default cap the same LP solves
    ok = pkg.solve_instance(inst, max_iters=100000, eps_rel_kkt=1e-8)
    assert ok.status == 0 and ok.stats["rejected_steps"] >= 1


def test_overflowing_objective_gives_numerical_error(pkg):
    """A finite objective whose scale overflows the step quantities (c times 1e200):
    the oracle stops with NUMERICAL_ERROR at once, and so does the library, with x and y
    written."""
    import dataclasses

    inst = lpgen.config0()
    big = dataclasses.replace(inst, c=inst.c * 1e200)
    with np.errstate(all="ignore"):
        ora = O.solve(big, O.Params(max_iters=200))
    assert ora.status == O.NUMERICAL_ERROR
    res = pkg.solve_instance(big, max_iters=200)
    assert res.status == 5, res.status_name
    assert res.stats["iterations"] == 0
    # the point returned is the start z^{0,0}, like the oracle's
    np.testing.assert_array_equal(res.x, ora.x)
    np.testing.assert_array_equal(res.y, ora.y)
