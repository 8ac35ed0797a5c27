"""Infeasibility detection (Sec. 3, App. C) on the CUDA path against the oracle.

On the small closed-form LPs the certificate is found at the first check, where the
trajectories agree, so status and detection iteration must equal the oracle's.  On the
random LPs detection happens after thousands of iterations, beyond the horizon where
the two trajectories agree (see test_gpu_polishing), so the status must match and the
returned certificate must pass App. C's conditions written out by hand (ratio
threshold 2e-9 instead of 1e-9 for the rounding of A'y between the two sides)."""
import numpy as np
import pytest

from oracle import pdlp_oracle as O
from tests import lp_helpers as H
from tests import test_oracle_infeasibility as PI

pytestmark = pytest.mark.gpu
INF = np.inf


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


SMALL = {
    "primal": lambda: H.make_lp([[1, 1], [1, 1]], [1, 1], [3, -INF], [INF, 1], [0, 0], [INF, INF]),
    "bound": lambda: H.make_lp([[1.0]], [0.0], [-INF], [1.0], [2.0], [INF]),
    "dual": lambda: H.make_lp([[1, -1]], [-1, 0], [-INF], [1], [0, 0], [INF, INF]),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_closed_form_certificates(pkg, name):
    inst = SMALL[name]()
    ref = O.solve(inst, O.Params(max_iters=5000))
    got = pkg.solve_instance(inst, max_iters=5000)
    assert got.status == ref.status and got.status in (O.PRIMAL_INFEASIBLE, O.DUAL_INFEASIBLE)
    assert got.stats["iterations"] == ref.stats["iterations"]
    if got.status == O.PRIMAL_INFEASIBLE:
        PI._check_primal_certificate(inst, got.y, eps=2e-9)
        np.testing.assert_allclose(got.y, ref.y, rtol=1e-9)
    else:
        PI._check_ray(inst, got.x, eps=2e-9)
        np.testing.assert_allclose(got.x, ref.x, rtol=1e-9)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_primal_infeasible_random(pkg, seed):
    inst = PI.primal_infeasible_lp(seed)
    got = pkg.solve_instance(inst, device=True, max_iters=100000)
    assert got.status == O.PRIMAL_INFEASIBLE, got.stats
    PI._check_primal_certificate(inst, got.y.cpu().numpy(), eps=2e-9)


@pytest.mark.parametrize("seed", [4, 5])
def test_unbounded_random(pkg, seed):
    inst = PI.unbounded_lp(seed)
    got = pkg.solve_instance(inst, device=True, max_iters=100000)
    assert got.status == O.DUAL_INFEASIBLE, got.stats
    PI._check_ray(inst, got.x.cpu().numpy(), eps=2e-9)


def test_detection_off(pkg):
    inst = PI.primal_infeasible_lp(1)
    got = pkg.solve_instance(inst, max_iters=3000, detect_infeasibility=0)
    assert got.status == O.ITERATION_LIMIT


def test_fp32_bulk_detects(pkg):
    """FP32 bulk iterates, FP64 measures: the closed-form cases are detected too."""
    for name in SMALL:
        inst = SMALL[name]()
        got = pkg.solve_instance(inst, max_iters=5000, precision=pkg.FP32_BULK)
        assert got.status in (O.PRIMAL_INFEASIBLE, O.DUAL_INFEASIBLE), (name, got.stats)
