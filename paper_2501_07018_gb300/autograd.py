"""Differentiable unrolled PDHG for PyTorch: a torch.autograd.Function whose forward and
backward are the library's pdlp_unrolled_pdhg (CUDA kernels; this module only passes
tensors through).

    x, y = unrolled_pdhg_layer(lp, c, lc, uc, lv, uv, K, eta, omega)
    loss(x, y).backward()      # gradients in c.grad, lc.grad, ... (float64 CUDA tensors)

``lp`` holds the constraint matrix (m, n, row_ptr, col_idx, val as CUDA tensors); the
objective and the bounds are the differentiable inputs.  The backward recomputes the
forward iterates from checkpoints (see include/pdlp.h), so nothing but the inputs is kept
between the two calls."""
from __future__ import annotations

import dataclasses

import torch

from . import binding


@dataclasses.dataclass
class SparseLp:
    m: int
    n: int
    row_ptr: torch.Tensor  # int64 CUDA
    col_idx: torch.Tensor  # int32 CUDA
    val: torch.Tensor      # float64 CUDA


class _Unrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, lc, uc, lv, uv, lp, K, eta, omega, checkpoint_every):
        x, y, _ = binding.unrolled_pdhg(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, c, lc, uc, lv,
                                        uv, K, eta, omega, checkpoint_every=checkpoint_every)
        ctx.save_for_backward(c, lc, uc, lv, uv)
        ctx.cfg = (lp, K, eta, omega, checkpoint_every)
        return x, y

    @staticmethod
    def backward(ctx, gx, gy):
        c, lc, uc, lv, uv = ctx.saved_tensors
        lp, K, eta, omega, every = ctx.cfg
        gx = torch.zeros(lp.n, dtype=torch.float64, device=c.device) if gx is None else gx
        gy = torch.zeros(lp.m, dtype=torch.float64, device=c.device) if gy is None else gy
        _, _, g = binding.unrolled_pdhg(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, c, lc, uc,
                                        lv, uv, K, eta, omega, gx=gx.contiguous(),
                                        gy=gy.contiguous(), checkpoint_every=every)
        return g["c"], g["lc"], g["uc"], g["lv"], g["uv"], None, None, None, None, None


def unrolled_pdhg_layer(lp: SparseLp, c, lc, uc, lv, uv, K: int, eta: float, omega: float = 1.0,
                        checkpoint_every: int = 50):
    """(x_K, y_K) of K PDHG steps of Eq. (3) with steps tau = eta/omega, sigma = eta*omega,
    differentiable with respect to c, lc, uc, lv, uv (float64 CUDA tensors)."""
    return _Unrolled.apply(c, lc, uc, lv, uv, lp, K, eta, omega, checkpoint_every)
