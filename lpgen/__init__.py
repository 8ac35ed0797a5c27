"""Seeded synthetic LP instances of the form  min c'x  s.t.  lc <= Ax <= uc,  lv <= x <= uv.

This module only draws random numbers and assembles arrays; it holds none of the
PDLP arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA path consume the
exact same bytes produced here, so neither side's input depends on the other.

The instances stand in for the large-scale LP suite of the paper (Sec. 6), whose
files are not available: every instance is feasible by construction (a point x0
satisfies all constraints), rows are two-sided with a chosen fraction of equality
rows, and column degrees follow either a fixed count or a truncated power law.

Draw order (fixed, so an instance is a pure function of its seed):
  1. column degrees, 2. row indices (without replacement per column),
  3. matrix values, 4. x0, 5. which columns are free, 6. which rows are equalities,
  7. row-bound slack draws, 8. objective c.

Layout: CSR of A with int64 row pointers, int32 column indices (strictly
increasing within a row) and float64 values; +-inf marks a missing bound.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20250107


@dataclasses.dataclass
class LPInstance:
    """A two-sided LP in CSR form (all arrays are plain numpy, host side)."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64[m+1]
    col_idx: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    c: np.ndarray  # float64[n]
    lc: np.ndarray  # float64[m]
    uc: np.ndarray  # float64[m]
    lv: np.ndarray  # float64[n]
    uv: np.ndarray  # float64[n]
    name: str = ""
    x0: np.ndarray | None = None  # the feasible point the instance was built from

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy_csr(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.m, self.n))


def config_seed(config: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of synthetic configuration ``config``."""
    return BASE_SEED + 1000 * config + instance


def _rows_without_replacement(rng: np.random.Generator, m: int, degrees: np.ndarray):
    """Per column j, ``degrees[j]`` distinct row indices drawn uniformly from [0, m).

    Returns (col_ptr int64[n+1], rows int64[nnz]) with rows sorted inside each column.
    Duplicates from an initial with-replacement draw are redrawn until none remain.
    """
    n = degrees.shape[0]
    if n and int(degrees.max(initial=0)) > m:
        raise ValueError("a column degree exceeds the number of rows")
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(degrees, out=col_ptr[1:])
    nnz = int(col_ptr[-1])
    col = np.repeat(np.arange(n, dtype=np.int64), degrees)
    rows = rng.integers(0, m, size=nnz, dtype=np.int64) if nnz else np.zeros(0, np.int64)
    while nnz:
        key = np.sort(col * m + rows)
        rows = key % m
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        ndup = int(dup.sum())
        if ndup == 0:
            break
        rows[dup] = rng.integers(0, m, size=ndup, dtype=np.int64)
    return col_ptr, rows


def _assemble(rng, m, n, degrees, values_fn, eq_frac, free_frac, x_hi=10.0, name=""):
    import scipy.sparse as sp

    col_ptr, rows = _rows_without_replacement(rng, m, degrees)
    nnz = rows.shape[0]
    vals = values_fn(rng, nnz)
    csc = sp.csc_matrix((vals, rows, col_ptr), shape=(m, n))
    A = csc.tocsr()
    A.sort_indices()
    x0 = rng.uniform(0.0, x_hi, size=n)
    lv = np.zeros(n)
    uv = np.full(n, x_hi)
    n_free = int(round(free_frac * n))
    if n_free:
        free = rng.permutation(n)[:n_free]
        lv[free] = -np.inf
        uv[free] = np.inf
    ax0 = A @ x0
    n_eq = int(round(eq_frac * m))
    eq = rng.permutation(m)[:n_eq]
    slack_lo = rng.uniform(0.0, 1.0, size=m)
    slack_hi = rng.uniform(0.0, 1.0, size=m)
    lc = ax0 - slack_lo
    uc = ax0 + slack_hi
    lc[eq] = ax0[eq]
    uc[eq] = ax0[eq]
    c = rng.uniform(-1.0, 1.0, size=n)
    return LPInstance(
        m=m,
        n=n,
        row_ptr=A.indptr.astype(np.int64),
        col_idx=A.indices.astype(np.int32),
        val=A.data.astype(np.float64),
        c=c,
        lc=lc,
        uc=uc,
        lv=lv,
        uv=uv,
        name=name,
        x0=x0,
    )


def _normal_values(rng, nnz):
    return rng.standard_normal(nnz)


def _signed_lognormal_values(rng, nnz):
    mag = rng.lognormal(0.0, 1.0, size=nnz)
    sign = np.where(rng.random(nnz) < 0.5, -1.0, 1.0)
    return mag * sign


def random_lp(m: int, n: int, nnz_per_col: int, seed: int, eq_frac: float = 0.3,
              free_frac: float = 0.0, name: str = "") -> LPInstance:
    """Uniform-degree random LP: every column has ``nnz_per_col`` N(0,1) entries at
    distinct uniform random rows; x0 ~ U[0,10]^n; bounds [0,10] (free columns get
    (-inf, inf)); row bounds Ax0 -/+ U[0,1] with ``eq_frac`` of rows equalities;
    c ~ U[-1,1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    degrees = np.full(n, min(nnz_per_col, m), dtype=np.int64)
    return _assemble(rng, m, n, degrees, _normal_values, eq_frac, free_frac, name=name)


def zipf_mean_exponent(kmin: int, kmax: int, mean: float) -> float:
    """Exponent s of the truncated power law p(k) ~ k^-s on [kmin, kmax] whose mean is
    ``mean`` (solved by bisection; the mean decreases in s)."""
    k = np.arange(kmin, kmax + 1, dtype=np.float64)

    def mean_of(s):
        w = k ** (-s)
        return float((k * w).sum() / w.sum())

    lo, hi = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mean_of(mid) > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw_degrees(rng, n, kmin, kmax, s):
    """``n`` i.i.d. draws of the truncated power law p(k) ~ k^-s on [kmin, kmax]
    by inverse-CDF lookup."""
    k = np.arange(kmin, kmax + 1, dtype=np.float64)
    w = k ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    idx = np.searchsorted(cdf, u, side="right")
    idx = np.minimum(idx, len(k) - 1)
    return (kmin + idx).astype(np.int64)


def powerlaw_lp(m: int, n: int, seed: int, kmin: int = 2, kmax: int = 5000,
                mean_degree: float = 10.0, eq_frac: float = 0.4, free_frac: float = 0.1,
                name: str = "") -> LPInstance:
    """Large-LP shape: power-law column degrees on [kmin, kmax] with the exponent
    solved so that the mean degree is ``mean_degree``; values +-lognormal(0,1);
    ``eq_frac`` equality rows and ``free_frac`` free columns."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = zipf_mean_exponent(kmin, min(kmax, m), mean_degree)
    degrees = powerlaw_degrees(rng, n, kmin, min(kmax, m), s)
    return _assemble(rng, m, n, degrees, _signed_lognormal_values, eq_frac, free_frac,
                     name=name)


def config0(instance: int = 0) -> LPInstance:
    """Small random LP: m=200, n=400, 5 nonzeros per column, 30% equality rows."""
    return random_lp(200, 400, 5, config_seed(0, instance), eq_frac=0.3, name="random-200x400")


def config1(instance: int = 0, scale: float = 1.0) -> LPInstance:
    """Single large LP: m=2e6, n=5e6, ~5e7 nonzeros with power-law column degrees
    (min 2, max 5000, mean 10), +-lognormal values, 40% equality rows, 10% free
    columns.  ``scale`` < 1 shrinks m and n proportionally (same recipe) for
    tests that need the shape but not the size."""
    m = max(8, int(round(2_000_000 * scale)))
    n = max(8, int(round(5_000_000 * scale)))
    return powerlaw_lp(m, n, config_seed(1, instance), name=f"powerlaw-{m}x{n}")


def multicommodity_flow_lp(nodes: int, arcs: int, commodities: int, seed: int,
                           zipf_a: float = 1.3) -> LPInstance:
    """Multicommodity min-cost flow: a directed graph with ``nodes`` nodes and ``arcs``
    arcs whose tails are drawn by rank from a Zipf(``zipf_a``) law over a random node
    order (a few hub nodes own most arcs), heads uniform among the other nodes; one flow
    variable f_{k,a} >= 0 per commodity k and arc a (column k * arcs + a); rows:
      * conservation, one per commodity and node (row k * nodes + v):
            sum_{a out of v} f_{k,a} - sum_{a into v} f_{k,a} = b_{k,v}   (equality)
      * capacity, one per arc (row commodities * nodes + a):
            sum_k f_{k,a} <= cap_a                                         (lc = -inf)
    Costs U[1,100] per arc (shared by the commodities), capacities U[10,1000].  The
    supplies come from a feasible flow f0_{k,a} = cap_a U[0,1] / commodities
    (b_k = N f0_k, summing to zero), so the LP is feasible; with nonnegative costs it is
    bounded.  Draw order: node order, tail ranks, heads, costs, capacities, f0."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(nodes)
    w = np.arange(1, nodes + 1, dtype=np.float64) ** (-zipf_a)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    ranks = np.minimum(np.searchsorted(cdf, rng.random(arcs), side="right"), nodes - 1)
    tail = order[ranks]
    head = rng.integers(0, nodes - 1, arcs)
    head = head + (head >= tail)  # uniform among the nodes other than the tail
    cost = rng.uniform(1.0, 100.0, arcs)
    cap = rng.uniform(10.0, 1000.0, arcs)
    K = commodities
    f0 = cap[None, :] * rng.random((K, arcs)) / K
    # node-arc incidence per commodity: +1 at the tail, -1 at the head
    b = np.zeros((K, nodes))
    for k in range(K):
        b[k] = np.bincount(tail, weights=f0[k], minlength=nodes) - \
            np.bincount(head, weights=f0[k], minlength=nodes)
    # CSR rows of the conservation block of one commodity (same pattern for every k):
    # row v holds the out-arcs of v (+1) and the in-arcs of v (-1), columns increasing
    ends = np.concatenate([tail, head])
    arc_of = np.concatenate([np.arange(arcs), np.arange(arcs)])
    sgn = np.concatenate([np.ones(arcs), -np.ones(arcs)])
    o = np.lexsort((arc_of, ends))
    ends, arc_of, sgn = ends[o], arc_of[o], sgn[o]
    cnt = np.bincount(ends, minlength=nodes).astype(np.int64)
    m = K * nodes + arcs
    n = K * arcs
    nnz = 3 * n
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_len = np.concatenate([np.tile(cnt, K), np.full(arcs, K, dtype=np.int64)])
    np.cumsum(row_len, out=row_ptr[1:])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    blk = 2 * arcs
    for k in range(K):
        col[k * blk:(k + 1) * blk] = (k * arcs + arc_of).astype(np.int32)
        val[k * blk:(k + 1) * blk] = sgn
    # capacity rows: columns a, arcs + a, ..., (K-1) arcs + a
    cap_cols = (np.arange(K)[None, :] * arcs + np.arange(arcs)[:, None]).reshape(-1)
    col[K * blk:] = cap_cols.astype(np.int32)
    val[K * blk:] = 1.0
    lc = np.concatenate([b.reshape(-1), np.full(arcs, -np.inf)])
    uc = np.concatenate([b.reshape(-1), cap])
    c = np.tile(cost, K)
    x0 = f0.reshape(-1)
    return LPInstance(m=m, n=n, row_ptr=row_ptr, col_idx=col, val=val, c=c, lc=lc, uc=uc,
                      lv=np.zeros(n), uv=np.full(n, np.inf),
                      name=f"mcf nodes={nodes} arcs={arcs} commodities={K}", x0=x0)


def config4(scale: float = 1.0, instance: int = 0) -> LPInstance:
    """The multicommodity-flow LP sized for one GPU's HBM: 2e6 nodes, 2e7 arcs with
    Zipf(1.3) out-degrees, 50 commodities (m = 1.2e8, n = 1e9, 3e9 nonzeros); ``scale``
    shrinks nodes and arcs proportionally (same recipe)."""
    nodes = max(8, int(round(2_000_000 * scale)))
    arcs = max(16, int(round(20_000_000 * scale)))
    return multicommodity_flow_lp(nodes, arcs, 50, config_seed(4, instance))


def uneven_lp(seed: int, m_lo: int = 500, m_hi: int = 20000) -> LPInstance:
    """One LP of the batch of uneven sizes: m ~ U{m_lo..m_hi}, n ~ U{1.5m..3m}, each
    column with U{4..12} N(0,1) entries at distinct uniform rows, otherwise the 200 x 400
    recipe (x0 ~ U[0,10], bounds [0,10], rows A x0 -/+ U[0,1], 30% equalities,
    c ~ U[-1,1]).  Draw order: m, n, column degrees, then as ``random_lp``."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(m_lo, m_hi + 1))
    n = int(rng.integers(int(1.5 * m), 3 * m + 1))
    degrees = rng.integers(4, 13, size=n).astype(np.int64)
    return _assemble(rng, m, n, degrees, _normal_values, eq_frac=0.3, free_frac=0.0,
                     name=f"uneven m={m} n={n}")


def config2(count: int = 1024, instance: int = 0, m_lo: int = 500, m_hi: int = 20000):
    """The batch of ``count`` LPs of uneven sizes (``uneven_lp`` with per-LP seeds)."""
    base = config_seed(2, instance) * 4096
    return [uneven_lp(base + k, m_lo, m_hi) for k in range(count)]
