"""The adjoint of unrolled PDHG on the CUDA path (pdlp_unrolled_pdhg and the torch
autograd layer) against the oracle's reverse-mode derivative, against central finite
differences of the GPU forward map, and against the LP sensitivity closed forms.

Fixed-step PDHG is non-expansive, so the GPU and oracle iterates stay within rounding
of each other (no amplification as with the adaptive step); gradients are compared at
1e-9 relative to the largest entry."""
import json
import os

import numpy as np
import pytest

from oracle import pdlp_oracle as O
from tests import lp_helpers as H
from tests import test_oracle_adjoint as PA

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
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


def _run(pkg, inst, K, eta, omega, gx=None, gy=None, every=50):
    return pkg.binding.unrolled_pdhg(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val, inst.c,
                                     inst.lc, inst.uc, inst.lv, inst.uv, K, eta, omega, gx=gx,
                                     gy=gy, checkpoint_every=every)


def _close(a, b, rel=1e-9):
    scale = max(1.0, float(np.max(np.abs(b)))) if b.size else 1.0
    return float(np.max(np.abs(a - b))) <= rel * scale if b.size else True


@pytest.mark.parametrize("seed", [5, 6])
def test_gradients_match_oracle_for_every_checkpoint_spacing(pkg, seed):
    for inst in PA._fd_cases(seed):
        rng = np.random.default_rng(seed)
        A = inst.scipy_csr().toarray()
        eta, omega, K = 0.9 / np.linalg.norm(A, 2), 0.8, 150
        gx, gy = rng.standard_normal(inst.n), rng.standard_normal(inst.m)
        xo, yo, go = O.unrolled_pdhg_vjp(inst, K, eta, omega, gx, gy)
        ref = None
        for every in (1, 7, 50, 1000):
            x, y, g = _run(pkg, inst, K, eta, omega, gx, gy, every)
            assert _close(x, xo) and _close(y, yo), inst.name
            for k in KEYS:
                assert _close(g[k], go[k]), (inst.name, k, every)
            if ref is None:
                ref = (x, y, g)
            else:  # recomputation from checkpoints is bit-identical
                assert np.array_equal(x, ref[0]) and np.array_equal(y, ref[1])
                for k in KEYS:
                    assert np.array_equal(g[k], ref[2][k]), (k, every)


@pytest.mark.parametrize("k", [0, 1])
def test_differentiable_batch_shape_matches_oracle(pkg, k):
    """The differentiable-batch shape at full size: an LP of 2000 rows x 5000 columns
    with 8 N(0,1) entries per column, K = 2000 fixed steps eta = 0.9 /
    sqrt(||A||_1 ||A||_inf) (<= 0.9 / ||A||_2), checkpoints every 50, loss
    ||x_K - x_target||^2 with x_target ~ U[0,10]: x_K, y_K and the gradients with
    respect to c, lc, uc, lv, uv equal the oracle's reverse-mode derivative element by
    element (1e-9 relative to the largest entry)."""
    import lpgen

    rng = np.random.default_rng(lpgen.config_seed(3) + k)
    inst = lpgen.random_lp(2000, 5000, 8, seed=lpgen.config_seed(3, k))
    A = inst.scipy_csr()
    eta = 0.9 / np.sqrt(float(abs(A).sum(axis=0).max()) * float(abs(A).sum(axis=1).max()))
    K = 2000
    target = rng.uniform(0.0, 10.0, inst.n)
    xK = O.unrolled_pdhg(inst, K, eta, 1.0)[K][0]
    gx, gy = 2.0 * (xK - target), np.zeros(inst.m)
    xo, yo, go = O.unrolled_pdhg_vjp(inst, K, eta, 1.0, gx, gy)
    x, y, g = _run(pkg, inst, K, eta, 1.0, gx, gy, 50)
    assert _close(x, xo) and _close(y, yo)
    for key in KEYS:
        assert _close(g[key], go[key]), key


def test_fp32_forward_with_fp64_gradient(pkg):
    """FP32 forward (precision = FP32 bulk: matrix, iterates, products and checkpoints in
    FP32) with the FP64 reverse pass, on the differentiable-batch shape (2000 x 5000, 8
    entries per column, K = 2000, checkpoints every 50): x_K is the FP64 oracle's to FP32
    accuracy, and the gradients agree with the FP64 oracle's reverse-mode derivative in
    direction and size (the reverse pass follows the FP32 trajectory's clamp branches,
    which differ from the FP64 trajectory's only where an iterate sits within rounding of
    a bound); the FP32 and FP64 forward passes of the library both run through the C ABI."""
    import lpgen

    rng = np.random.default_rng(lpgen.config_seed(3))
    inst = lpgen.random_lp(2000, 5000, 8, seed=lpgen.config_seed(3, 0))
    A = inst.scipy_csr()
    eta = 0.9 / np.sqrt(float(abs(A).sum(axis=0).max()) * float(abs(A).sum(axis=1).max()))
    K = 2000
    target = rng.uniform(0.0, 10.0, inst.n)
    xK = O.unrolled_pdhg(inst, K, eta, 1.0)[K][0]
    gx, gy = 2.0 * (xK - target), np.zeros(inst.m)
    xo, yo, go = O.unrolled_pdhg_vjp(inst, K, eta, 1.0, gx, gy)
    x, y, g = pkg.binding.unrolled_pdhg(inst.m, inst.n, inst.row_ptr, inst.col_idx, inst.val,
                                        inst.c, inst.lc, inst.uc, inst.lv, inst.uv, K, eta, 1.0,
                                        gx=gx, gy=gy, checkpoint_every=50, precision=pkg.FP32_BULK)
    ex = float(np.max(np.abs(x - xo))) / max(1.0, float(np.max(np.abs(xo))))
    ey = float(np.max(np.abs(y - yo))) / max(1.0, float(np.max(np.abs(yo))))
    print(f"FP32 forward: x_K error {ex:.2e}, y_K error {ey:.2e}")
    assert ex <= 1e-4 and ey <= 1e-4
    for key in KEYS:
        a, b = g[key], go[key]
        nb = float(np.linalg.norm(b))
        if nb == 0.0:
            assert float(np.linalg.norm(a)) == 0.0, key
            continue
        rel = float(np.linalg.norm(a - b)) / nb
        cos = float(a @ b) / (float(np.linalg.norm(a)) * nb)
        frac = float(np.mean(np.abs(a - b) <= 1e-4 * max(1.0, float(np.max(np.abs(b))))))
        print(f"  grad {key}: relative l2 error {rel:.2e}, cosine {cos:.8f}, entries within 1e-4: {frac:.4f}")
        assert rel <= 1e-2 and cos >= 0.9999, key


def test_gradients_match_central_differences_of_the_gpu_forward(pkg):
    import dataclasses

    inst = PA._fd_cases(9)[1]
    rng = np.random.default_rng(2)
    A = inst.scipy_csr().toarray()
    eta, omega, K = 0.9 / np.linalg.norm(A, 2), 1.1, 120
    gx, gy = rng.standard_normal(inst.n), rng.standard_normal(inst.m)
    _, _, g = _run(pkg, inst, K, eta, omega, gx, gy, 25)

    def loss(i2):
        x, y, _ = _run(pkg, i2, K, eta, omega)
        return float(gx @ x + gy @ y)
    eq = inst.lc == inst.uc
    h = 1e-6
    for key, keys, d in (("c", ("c",), rng.standard_normal(inst.n)),
                         ("uv", ("uv",), rng.standard_normal(inst.n) * np.isfinite(inst.uv)),
                         ("lc", ("lc",), rng.standard_normal(inst.m) * (~eq & np.isfinite(inst.lc))),
                         ("b", ("lc", "uc"), rng.standard_normal(inst.m) * eq)):
        if not np.any(d):
            continue
        plus = dataclasses.replace(inst, **{k: getattr(inst, k) + h * d for k in keys})
        minus = dataclasses.replace(inst, **{k: getattr(inst, k) - h * d for k in keys})
        fd = (loss(plus) - loss(minus)) / (2 * h)
        an = float(sum(g[k] for k in keys) @ d)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (key, fd, an)


def test_sensitivity_closed_forms(pkg):
    with open(os.path.join(GOLDEN, "textbook_lp.json")) as f:
        gd = json.load(f)
    inf = float("inf")
    conv = lambda v: [inf if s == "inf" else (-inf if s == "-inf" else s) for s in v]  # noqa
    inst = H.make_lp(gd["A"], gd["c"], conv(gd["lc"]), conv(gd["uc"]), conv(gd["lv"]),
                     conv(gd["uv"]))
    A = inst.scipy_csr().toarray()
    x, y, g = _run(pkg, inst, 3000, 0.9 / np.linalg.norm(A, 2), 1.0, inst.c, np.zeros(inst.m))
    np.testing.assert_allclose(x + g["c"], gd["x_star"], atol=1e-9)
    np.testing.assert_allclose(g["uc"], -np.maximum(-np.array(gd["y_star"]), 0.0), atol=1e-9)


def test_autograd_layer(pkg):
    """loss = ||x_K - x_target||^2 through the torch layer: the gradients equal the
    library's vector-Jacobian product with gx = 2 (x_K - x_target), gy = 0."""
    import torch

    from paper_2501_07018_gb300.autograd import SparseLp, unrolled_pdhg_layer

    inst = PA._fd_cases(11)[0]
    A = inst.scipy_csr().toarray()
    eta = 0.9 / np.linalg.norm(A, 2)
    dev = lambda a: torch.as_tensor(np.asarray(a)).cuda()  # noqa: E731
    lp = SparseLp(inst.m, inst.n, dev(inst.row_ptr), dev(inst.col_idx), dev(inst.val))
    params = [dev(v).clone().requires_grad_(True) for v in (inst.c, inst.lc, inst.uc, inst.lv, inst.uv)]
    target = torch.linspace(0, 3, inst.n, dtype=torch.float64, device="cuda")
    x, y = unrolled_pdhg_layer(lp, *params, K=100, eta=eta, omega=1.0, checkpoint_every=10)
    loss = ((x - target) ** 2).sum()
    loss.backward()
    gx = 2.0 * (x.detach() - target)
    _, _, go = O.unrolled_pdhg_vjp(inst, 100, eta, 1.0, gx.cpu().numpy(), np.zeros(inst.m))
    for p_, k in zip(params, KEYS):
        assert _close(p_.grad.cpu().numpy(), go[k]), k


def test_batch_equals_single_calls(pkg):
    """pdlp_unrolled_pdhg_batch: every LP's outputs and gradients equal, bit for bit, a
    single call on it (forward-only items included)."""
    items, singles = [], []
    for seed in (5, 6, 7):
        for inst in PA._fd_cases(seed):
            rng = np.random.default_rng(seed)
            eta = 0.9 / np.linalg.norm(inst.scipy_csr().toarray(), 2)
            gx, gy = rng.standard_normal(inst.n), rng.standard_normal(inst.m)
            items.append(dict(lp=inst, K=80, eta=eta, omega=0.9, gx=gx, gy=gy, checkpoint_every=9))
            singles.append(_run(pkg, inst, 80, eta, 0.9, gx, gy, 9))
    items.append(dict(lp=items[0]["lp"], K=80, eta=items[0]["eta"], omega=0.9))
    singles.append(_run(pkg, items[0]["lp"], 80, items[0]["eta"], 0.9))
    got = pkg.binding.unrolled_pdhg_batch(items, concurrency=4)
    for (st, x, y, g), (xs, ys, gs) in zip(got, singles):
        assert st == 0
        assert np.array_equal(x, xs) and np.array_equal(y, ys)
        if gs is None:
            assert g is None
        else:
            for k in KEYS:
                assert np.array_equal(g[k], gs[k]), k
