"""The seeded input generators (lpgen) against the recipes they state: shapes, degree
laws, equality / free fractions, value laws, feasibility of the point each instance is
built from, and the structure of the multicommodity-flow LP.  CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen


def _csr_valid(inst):
    rp, col = inst.row_ptr, inst.col_idx
    assert rp.dtype == np.int64 and col.dtype == np.int32 and inst.val.dtype == np.float64
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(col) == len(inst.val)
    assert np.all((col >= 0) & (col < inst.n))
    for i in range(inst.m):  # strictly increasing columns within a row
        seg = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0)


def _feasible_point(inst, rtol=1e-12):
    ax0 = inst.scipy_csr() @ inst.x0
    scale = 1.0 + np.abs(ax0)
    assert np.all(inst.lc - ax0 <= rtol * scale)
    assert np.all(ax0 - inst.uc <= rtol * scale)
    assert np.all(inst.x0 >= inst.lv) and np.all(inst.x0 <= inst.uv)


def _column_degrees(inst):
    return np.bincount(inst.col_idx, minlength=inst.n)


def test_small_random_lp_recipe():
    inst = lpgen.config0()
    assert (inst.m, inst.n) == (200, 400)
    _csr_valid(inst)
    assert np.all(_column_degrees(inst) == 5)
    assert int(np.sum(inst.lc == inst.uc)) == 60  # 30% equality rows
    assert np.all(inst.lv == 0.0) and np.all(inst.uv == 10.0)
    assert np.all(np.abs(inst.c) <= 1.0)
    _feasible_point(inst)
    # two-sided rows: the slacks are U[0,1] on each side
    ax0 = inst.scipy_csr() @ inst.x0
    ineq = inst.lc < inst.uc
    assert np.all(ax0[ineq] - inst.lc[ineq] <= 1.0) and np.all(inst.uc[ineq] - ax0[ineq] <= 1.0)


def test_seeded_generators_are_deterministic():
    a, b, c = lpgen.config0(), lpgen.config0(), lpgen.config0(instance=1)
    for f in ("row_ptr", "col_idx", "val", "c", "lc", "uc"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.val, c.val)
    assert lpgen.config_seed(1, 3) == lpgen.BASE_SEED + 1003


def test_power_law_exponent_gives_the_stated_mean():
    s = lpgen.zipf_mean_exponent(2, 5000, 10.0)
    k = np.arange(2, 5001, dtype=np.float64)
    w = k ** (-s)
    assert abs((k * w).sum() / w.sum() - 10.0) < 1e-9
    assert 2.0 < s < 2.2


def test_power_law_lp_recipe():
    inst = lpgen.config1(scale=0.01)  # 20,000 x 50,000, the same recipe
    assert (inst.m, inst.n) == (20000, 50000)
    _csr_valid(inst)
    deg = _column_degrees(inst)
    assert deg.min() >= 2 and deg.max() <= 5000
    assert abs(deg.mean() - 10.0) < 0.5
    assert np.quantile(deg, 0.5) <= 4  # heavy tail: the median is far below the mean
    assert int(np.sum(inst.lc == inst.uc)) == 8000  # 40% equality rows
    free = np.isinf(inst.lv) & np.isinf(inst.uv)
    assert int(free.sum()) == 5000  # 10% free columns
    assert np.all(inst.lv[~free] == 0.0) and np.all(inst.uv[~free] == 10.0)
    logs = np.log(np.abs(inst.val))
    assert abs(np.median(logs)) < 0.03 and abs(logs.std() - 1.0) < 0.03
    assert abs(np.mean(inst.val > 0) - 0.5) < 0.01
    _feasible_point(inst)
    # rows draw their entries uniformly: row degrees have mean nnz/m and no heavy tail
    rdeg = np.diff(inst.row_ptr)
    assert abs(rdeg.mean() - inst.nnz / inst.m) < 1e-9
    assert rdeg.max() < 5 * rdeg.mean()


def test_multicommodity_flow_structure():
    nodes, arcs, K = 60, 500, 3
    inst = lpgen.multicommodity_flow_lp(nodes, arcs, K, seed=7)
    assert inst.m == K * nodes + arcs and inst.n == K * arcs and inst.nnz == 3 * inst.n
    _csr_valid(inst)
    A = sp.csc_matrix(inst.scipy_csr())
    A.sort_indices()
    assert np.all(np.diff(A.indptr) == 3)
    for j in range(inst.n):  # +1 at (k, tail), -1 at (k, head), +1 at the capacity row
        k, a = divmod(j, arcs)
        rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
        vals = A.data[A.indptr[j]:A.indptr[j + 1]]
        cons = rows < K * nodes
        assert cons.sum() == 2 and np.all(rows[cons] // nodes == k)
        assert sorted(vals[cons]) == [-1.0, 1.0]
        assert rows[~cons][0] == K * nodes + a and vals[~cons][0] == 1.0
    cons_rows = np.arange(K * nodes)
    assert np.all(inst.lc[cons_rows] == inst.uc[cons_rows])  # conservation: equalities
    assert np.all(np.isneginf(inst.lc[K * nodes:]))  # capacity rows: <= cap
    for k in range(K):  # supplies of each commodity sum to zero
        assert abs(inst.lc[k * nodes:(k + 1) * nodes].sum()) < 1e-8
    assert np.all(inst.c >= 1.0) and np.all(inst.c <= 100.0)
    assert np.array_equal(inst.c[:arcs], inst.c[arcs:2 * arcs])  # costs shared
    assert np.all(inst.lv == 0.0) and np.all(np.isposinf(inst.uv))
    _feasible_point(inst, rtol=1e-12)
    # Zipf tails: the busiest node owns far more than a uniform share of the arcs
    out = np.diff(inst.row_ptr[:nodes + 1])  # commodity 0: out- plus in-arcs per node
    assert out.max() > 5 * (2 * arcs / nodes)


def test_uneven_batch_recipe():
    batch = lpgen.config2(count=6)
    assert len({(i.m, i.n) for i in batch}) == 6
    for inst in batch:
        assert 500 <= inst.m <= 20000 and int(1.5 * inst.m) <= inst.n <= 3 * inst.m
        deg = _column_degrees(inst)
        assert deg.min() >= 4 and deg.max() <= 12
        assert int(np.sum(inst.lc == inst.uc)) == int(round(0.3 * inst.m))
        _feasible_point(inst)


def test_degree_above_row_count_is_rejected():
    rng = np.random.default_rng(0)
    with pytest.raises(ValueError):
        lpgen._rows_without_replacement(rng, 3, np.array([2, 4]))
