"""The allocation-free entry point pdlp_kkt_products_noalloc, checked through the C ABI
against pdlp_kkt on the same point and against the FP64 oracle's measures (kkt_stats),
on two calls in a row (the second call must not see the first call's leftovers in the
shared scratch array).

It is for callers that cannot let a library allocate device memory while they run
(their own pool owns the device, or an allocation could stall a latency-bound loop);
they pass device arrays including the products A x and A'y they already hold.
This file is collected last so that a stopping run has executed every other test.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import gpu_helpers as GH

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


def _point(rng, inst):
    lv = np.where(np.isfinite(inst.lv), inst.lv, -5.0)
    uv = np.where(np.isfinite(inst.uv), inst.uv, 5.0)
    x = lv + (uv - lv) * rng.random(inst.n)
    y = rng.standard_normal(inst.m)
    y = np.where(~np.isfinite(inst.lc) & (y > 0), -y, y)
    y = np.where(~np.isfinite(inst.uc) & (y < 0), -y, y)
    y = np.where(~np.isfinite(inst.lc) & ~np.isfinite(inst.uc), 0.0, y)
    return x, y


@pytest.mark.parametrize("name", ["edge", "powerlaw"])
def test_noalloc_matches_kkt_twice(pkg, name):
    import torch

    inst = GH.edge_instance() if name == "edge" else lpgen.config1(scale=0.01)
    A = inst.scipy_csr()
    rng = np.random.default_rng(17)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()  # noqa: E731
    vecs = [dev(v) for v in (inst.c, inst.lc, inst.uc, inst.lv, inst.uv)]
    results = []
    for call in range(2):
        x, y = _point(rng, inst)
        ref = pkg.kkt(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val, inst.c, inst.lc,
                      inst.uc, inst.lv, inst.uv, x, y)
        got = pkg.kkt_products_noalloc(inst.m, inst.n, *vecs, dev(x), dev(y), dev(A @ x),
                                       dev(A.T @ y))
        torch.cuda.synchronize()
        for k, v in ref.items():
            assert abs(got[k] - v) <= 1e-11 * max(1.0, abs(v)), (call, k, got[k], v)
        ora = O.kkt_stats(inst, A, x, y)
        for k in ("rel_kkt", "rel_primal", "rel_dual", "rel_gap", "pobj", "dobj",
                  "primal_res_inf", "dual_res_inf"):
            assert abs(got[k] - ora[k]) <= 1e-10 * max(1.0, abs(ora[k])), (call, k, got[k], ora[k])
        results.append(got)
    assert results[0] != results[1]  # two different points, no stale scratch


def test_noalloc_rejects_bad_sizes(pkg):
    import torch

    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.PdlpError) as ei:
        pkg.kkt_products_noalloc(-1, 4, t, t, t, t, t, t, t, t, t)
    assert ei.value.code == -1
    with pytest.raises(pkg.PdlpError):
        pkg.kkt_products_noalloc(4, 2 ** 31, t, t, t, t, t, t, t, t, t)
