"""Shared fixtures of the GPU tests: seeded edge-case instances and trace comparison."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

import lpgen


def edge_instance(seed=11, m=1500, n=3000, dense_row_nnz=2500, dense_col_nnz=1300):
    """A feasible LP exercising every structural case of the kernels: empty rows and
    columns, a row longer than one shared-memory chunk (A side), a column longer than
    the long-row threshold (transpose side), one-sided, free and equality rows, free
    and fixed variables.  Bounds are derived from a feasible x0 after the pattern is
    fixed, so the instance stays feasible; free variables get c = 0, so it stays
    bounded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols = [], []
    for j in range(n):
        if j % 97 == 5:
            continue  # empty column
        k = 4 if j != 7 else min(dense_col_nnz, m)
        r = rng.choice(m, size=k, replace=False)
        rows.append(r)
        cols.append(np.full(k, j))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    # a dense row (A-side long row, several chunks)
    dr = 3
    dcols = rng.choice(n, size=min(dense_row_nnz, n), replace=False)
    rows = np.concatenate([rows, np.full(dcols.size, dr)])
    cols = np.concatenate([cols, dcols])
    vals = rng.standard_normal(rows.size)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    # empty rows
    keep = np.ones(m, bool)
    keep[::113] = False
    keep[dr] = True
    D = sp.diags(keep.astype(float))
    A = (D @ A).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    x0 = rng.uniform(0, 10, n)
    lv = np.zeros(n)
    uv = np.full(n, 10.0)
    free = rng.choice(n, size=n // 20, replace=False)
    lv[free], uv[free] = -np.inf, np.inf
    fixed = rng.choice(np.setdiff1d(np.arange(n), free), size=n // 40, replace=False)
    lv[fixed] = uv[fixed] = x0[fixed]
    ax0 = A @ x0
    lc = ax0 - rng.uniform(0, 1, m)
    uc = ax0 + rng.uniform(0, 1, m)
    kind = rng.integers(0, 6, m)
    lc = np.where(kind == 1, -np.inf, lc)
    uc = np.where(kind == 2, np.inf, uc)
    lc = np.where(kind == 3, ax0, lc)
    uc = np.where(kind == 3, ax0, uc)
    lc = np.where(kind == 4, -np.inf, lc)
    uc = np.where(kind == 4, np.inf, uc)
    c = rng.uniform(-1, 1, n)
    c[free] = 0.0
    return lpgen.LPInstance(m=m, n=n, row_ptr=A.indptr.astype(np.int64),
                            col_idx=A.indices.astype(np.int32), val=A.data.astype(np.float64),
                            c=c, lc=lc, uc=uc, lv=lv, uv=uv, name="edge", x0=x0)


def trace_errors(gpu_trace, ora_trace):
    """Per accepted iteration: relative infinity-norm distance of the iterates, the
    relative difference of the accepted step, and whether the restart kinds agree."""
    out = []
    for g, o in zip(gpu_trace, ora_trace):
        zo = np.concatenate([o["x"], o["y"]])
        zg = np.concatenate([g["x"], g["y"]])
        ez = float(np.max(np.abs(zg - zo))) / max(1.0, float(np.max(np.abs(zo))))
        ee = abs(g["eta"] - o["eta"]) / abs(o["eta"])
        out.append(dict(k=o["k"], ez=ez, eeta=ee, restart_same=g["restart"] == o["restart"],
                        mu=(g["mu_cur"], o["mu_cur"], g["mu_avg"], o["mu_avg"])))
    return out
