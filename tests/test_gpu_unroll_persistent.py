"""The persistent unrolled-PDHG batch (pdlp_unrolled_pdhg_batch_persistent): one launch,
one CTA per LP, each LP's K fixed steps of Eq. (3), checkpoints and reverse pass -- held
to the oracle's reverse-mode derivative at the tolerance of the single-call tests
(1e-9 relative to the largest entry), to the single calls themselves (the same per-row
summation order: 1e-12), and to its own recomputation from checkpoints (bit for bit
across checkpoint spacings)."""
import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import test_oracle_adjoint as PA

pytestmark = pytest.mark.gpu
KEYS = ("c", "lc", "uc", "lv", "uv")


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


def _close(a, b, rel):
    scale = max(1.0, float(np.max(np.abs(b)))) if b.size else 1.0
    return float(np.max(np.abs(a - b))) <= rel * scale if b.size else True


def _single(pkg, it, **prm):
    inst = it["lp"]
    return pkg.binding.unrolled_pdhg(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val,
                                     inst.c, inst.lc, inst.uc, inst.lv, inst.uv, it["K"],
                                     it["eta"], it.get("omega", 1.0), gx=it.get("gx"),
                                     gy=it.get("gy"), checkpoint_every=it.get("checkpoint_every", 50),
                                     **prm)


def _items(seeds=(5, 6, 7), K=150, every=9):
    items = []
    for seed in seeds:
        for inst in PA._fd_cases(seed):
            rng = np.random.default_rng(seed)
            eta = 0.9 / np.linalg.norm(inst.scipy_csr().toarray(), 2)
            items.append(dict(lp=inst, K=K, eta=eta, omega=0.8, gx=rng.standard_normal(inst.n),
                              gy=rng.standard_normal(inst.m), checkpoint_every=every))
    return items


def test_matches_oracle_and_single_calls(pkg):
    items = _items()
    items.append(dict(lp=items[0]["lp"], K=150, eta=items[0]["eta"], omega=0.8))  # forward only
    got = pkg.binding.unrolled_pdhg_batch(items, persistent=True)
    for it, (st, x, y, g) in zip(items, got):
        assert st == 0
        inst = it["lp"]
        one = _single(pkg, it)
        assert _close(x, one[0], 1e-12) and _close(y, one[1], 1e-12), inst.name
        if it.get("gx") is None:
            assert g is None
            continue
        xo, yo, go = O.unrolled_pdhg_vjp(inst, it["K"], it["eta"], it["omega"], it["gx"], it["gy"])
        assert _close(x, xo, 1e-9) and _close(y, yo, 1e-9), inst.name
        for k in KEYS:
            assert _close(g[k], go[k], 1e-9), (inst.name, k)
            assert _close(g[k], one[2][k], 1e-12), (inst.name, k)


def test_checkpoint_spacings_recompute_bit_for_bit(pkg):
    base = _items(seeds=(8,), K=100)
    ref = None
    for every in (1, 7, 50, 1000):
        items = [dict(it, checkpoint_every=every) for it in base]
        got = pkg.binding.unrolled_pdhg_batch(items, persistent=True)
        if ref is None:
            ref = got
            continue
        for (st, x, y, g), (_, xr, yr, gr) in zip(got, ref):
            assert st == 0 and np.array_equal(x, xr) and np.array_equal(y, yr)
            for k in KEYS:
                assert np.array_equal(g[k], gr[k]), (every, k)


def _config3_item(k):
    rng = np.random.default_rng(lpgen.config_seed(3) + k)
    inst = lpgen.random_lp(2000, 5000, 8, seed=lpgen.config_seed(3, k))
    A = inst.scipy_csr()
    eta = 0.9 / np.sqrt(float(abs(A).sum(axis=0).max()) * float(abs(A).sum(axis=1).max()))
    K = 2000
    target = rng.uniform(0.0, 10.0, inst.n)
    xK = O.unrolled_pdhg(inst, K, eta, 1.0)[K][0]
    return dict(lp=inst, K=K, eta=eta, omega=1.0, gx=2.0 * (xK - target), gy=np.zeros(inst.m),
                checkpoint_every=50)


def test_differentiable_batch_shape_matches_oracle(pkg):
    """Two LPs of the differentiable-batch shape (2000 x 5000, 8 entries per column,
    K = 2000, checkpoints every 50, loss ||x_K - x_target||^2) in one launch, against
    the oracle's reverse-mode derivative element by element; device arrays."""
    import torch

    items = [_config3_item(k) for k in (0, 1)]
    dev = [dict(it, gx=torch.as_tensor(it["gx"]).cuda(), gy=torch.as_tensor(it["gy"]).cuda())
           for it in items]
    got = pkg.binding.unrolled_pdhg_batch(dev, device=True, persistent=True)
    for it, (st, x, y, g) in zip(items, got):
        assert st == 0
        inst = it["lp"]
        xo, yo, go = O.unrolled_pdhg_vjp(inst, it["K"], it["eta"], 1.0, it["gx"], it["gy"])
        assert _close(x.cpu().numpy(), xo, 1e-9) and _close(y.cpu().numpy(), yo, 1e-9)
        for k in KEYS:
            assert _close(g[k].cpu().numpy(), go[k], 1e-9), k


def test_fp32_forward_matches_single_call(pkg):
    """FP32 forward with the FP64 reverse pass: the same arithmetic as the single call
    (x_K within 1e-6, gradients within 1e-6 relative l2), and the FP64 oracle's
    derivative in direction and size."""
    it = _config3_item(0)
    (st, x, y, g), = pkg.binding.unrolled_pdhg_batch([it], persistent=True, precision=pkg.FP32_BULK)
    assert st == 0
    xs, ys, gs = _single(pkg, it, precision=pkg.FP32_BULK)
    assert _close(x, xs, 1e-6) and _close(y, ys, 1e-6)
    _, _, go = O.unrolled_pdhg_vjp(it["lp"], it["K"], it["eta"], 1.0, it["gx"], it["gy"])
    for k in KEYS:
        a, b = g[k], go[k]
        nb = float(np.linalg.norm(b))
        if nb == 0.0:
            assert float(np.linalg.norm(a)) == 0.0
            continue
        assert float(np.linalg.norm(a - gs[k])) <= 1e-6 * max(nb, 1e-300), k
        assert float(np.linalg.norm(a - b)) / nb <= 1e-2, k
        assert float(a @ b) / (float(np.linalg.norm(a)) * nb) >= 0.9999, k


def test_an_lp_too_large_fails_alone(pkg):
    small = _items(seeds=(5,), K=20)[0]
    big = lpgen.random_lp(4000, 9000, 4, seed=17)  # 2 (m + n) FP64 values + adjoints > 200 KB
    items = [small, dict(lp=big, K=5, eta=0.1, omega=1.0)]
    got = pkg.binding.unrolled_pdhg_batch(items, persistent=True)
    assert got[0][0] == 0
    assert got[1][0] == -1
    assert "too large" in pkg.binding.load_library().pdlp_last_error().decode()


def test_box_only_lp_and_empty_batch(pkg):
    """An LP without rows: K steps of Eq. (3a) alone, x_K = proj_X(x - K tau c) reached
    step by step, and the gradient of x_K wrt c is -tau K on the columns that never hit a
    bound (each step moves x by -tau c); the single call gives the same."""
    from tests import lp_helpers as H

    rng = np.random.default_rng(4)
    n = 300
    c = rng.uniform(-1.0, 1.0, n)
    lv, uv = np.full(n, -1e3), np.full(n, 1e3)
    box = H.make_lp(np.zeros((0, n)), c, [], [], lv, uv, name="box-only")
    it = dict(lp=box, K=40, eta=0.05, omega=1.0, gx=np.ones(n), gy=np.zeros(0), checkpoint_every=7)
    (st, x, y, g), = pkg.binding.unrolled_pdhg_batch([it], persistent=True)
    assert st == 0
    tau = 0.05
    assert np.allclose(x, -it["K"] * tau * c, rtol=1e-12, atol=1e-12)
    assert np.allclose(g["c"], -it["K"] * tau, rtol=1e-12)
    one = _single(pkg, it)
    assert np.array_equal(x, one[0]) and np.array_equal(g["c"], one[2]["c"])
    assert pkg.binding.unrolled_pdhg_batch([], persistent=True) == []


FD_H = 1e-6


def _fd_instance(k):
    """Instance k of the 16 central-difference LPs (the differentiable-batch shape), one
    objective coordinate j and one equality row i to perturb, and the loss target."""
    rng = np.random.default_rng(lpgen.config_seed(3) + 100 + k)
    inst = lpgen.random_lp(2000, 5000, 8, seed=lpgen.config_seed(3, 100 + k))
    A = inst.scipy_csr()
    eta = 0.9 / np.sqrt(float(abs(A).sum(axis=0).max()) * float(abs(A).sum(axis=1).max()))
    j = int(rng.integers(0, inst.n))
    i = int(rng.choice(np.flatnonzero(inst.lc == inst.uc)))
    return inst, eta, j, i, rng.uniform(0.0, 10.0, inst.n)


def _moved(inst, kind, idx, step):
    import dataclasses

    if kind == "c":
        c = inst.c.copy()
        c[idx] += step
        return dataclasses.replace(inst, c=c)
    lc, uc = inst.lc.copy(), inst.uc.copy()  # an equality row: b_i moves both sides
    lc[idx] += step
    uc[idx] += step
    return dataclasses.replace(inst, lc=lc, uc=uc)


def test_differentiable_batch_central_differences_on_16_instances(pkg):
    """Sixteen LPs of the differentiable-batch shape (2000 x 5000, 8 entries per column,
    K = 2000, checkpoints every 50), loss ||x_K - x_target||^2: the adjoint's derivative
    along one objective coordinate c_j and along one equality row's b_i (lc_i = uc_i
    moved together) against the central difference (L(h) - L(-h)) / 2h with h = 1e-6,
    every forward pass run by the same persistent launch in FP64.

    x_K is piecewise affine in (c, b): the clamps of Eq. (3) switch where an iterate
    meets a bound.  The central difference equals the derivative on one affine piece;
    x_K(h) - x_K(0) against x_K(0) - x_K(-h) measures how far [-h, h] strays from one
    piece (over 5000 x 2000 clamp decisions a few flip), and an instance whose second
    difference r exceeds 1e-3 of the first is not a nondegenerate one and is left out
    (at most 4 of 16).  The kinks inside [-h, h] move the central difference by about r
    relative, the rounding of the 2000 steps by ~1e-5 absolute (1e-13 per entry of
    x+ - x-, over 5000 entries, divided by 2h): the bound is 20 r |an| + 1e-4 max(1, |an|).
    Measured in FP64 on the CPU for these 16: r up to 1.5e-3 along c_j (two instances
    above 1e-3), under 1e-6 along b_i but one at 6e-5; |fd - an| at most 6.2 r |an| where r
    exceeds 1e-5, otherwise at most 3.4e-5 relative and 2.5e-6 absolute.  The loss
    difference is formed as (x+ - x-)'(x+ + x- - 2 x_target), equal to L(h) - L(-h)
    without its cancellation.  The FP32-forward adjoint is held to the same differences at
    1e-2 (relative l2 over the instances used)."""
    cases = [_fd_instance(k) for k in range(16)]
    fwd = []
    for inst, eta, j, i, _ in cases:
        fwd.append(dict(lp=inst, K=2000, eta=eta, omega=1.0))
        for kind, idx in (("c", j), ("b", i)):
            for s in (1.0, -1.0):
                fwd.append(dict(lp=_moved(inst, kind, idx, s * FD_H), K=2000, eta=eta, omega=1.0))
    got = pkg.binding.unrolled_pdhg_batch(fwd, persistent=True)
    assert all(st == 0 for st, *_ in got)
    xs = [x for _, x, _, _ in got]
    grad_items = []
    for k, (inst, eta, j, i, t) in enumerate(cases):
        grad_items.append(dict(lp=inst, K=2000, eta=eta, omega=1.0, gx=2.0 * (xs[5 * k] - t),
                               gy=np.zeros(inst.m), checkpoint_every=50))
    g64 = pkg.binding.unrolled_pdhg_batch(grad_items, persistent=True)
    g32 = pkg.binding.unrolled_pdhg_batch(grad_items, persistent=True, precision=pkg.FP32_BULK)
    used = {"c": 0, "b": 0}
    fd_all, an32_all = [], []
    for k, (inst, eta, j, i, t) in enumerate(cases):
        assert g64[k][0] == 0 and g32[k][0] == 0
        x0 = xs[5 * k]
        for d, (kind, idx) in enumerate((("c", j), ("b", i))):
            xp, xm = xs[5 * k + 1 + 2 * d], xs[5 * k + 2 + 2 * d]
            dp, dm = xp - x0, x0 - xm
            r = float(np.linalg.norm(dp - dm)) / float(np.linalg.norm(dp))
            if r > 1e-3:
                continue
            used[kind] += 1
            fd = float((xp - xm) @ (xp + xm - 2.0 * t)) / (2.0 * FD_H)
            g, gf = g64[k][3], g32[k][3]
            an = g["c"][idx] if kind == "c" else g["lc"][idx] + g["uc"][idx]
            an32 = gf["c"][idx] if kind == "c" else gf["lc"][idx] + gf["uc"][idx]
            bound = 20.0 * r * abs(an) + 1e-4 * max(1.0, abs(an))
            assert abs(fd - an) <= bound, (k, kind, fd, an, r)
            fd_all.append(fd)
            an32_all.append(an32)
    assert used["c"] >= 12 and used["b"] >= 12, used
    fd_all, an32_all = np.array(fd_all), np.array(an32_all)
    assert np.linalg.norm(an32_all - fd_all) <= 1e-2 * np.linalg.norm(fd_all)
