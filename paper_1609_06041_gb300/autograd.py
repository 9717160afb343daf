"""Differentiable forms of the operators and of the unrolled solve.

Project / Backproject: A and A^T as torch.autograd.Functions, each the
other's backward (A^T is the adjoint of A).  UnrolledPDTV: K iterations of
Algorithm 1 / 2 with learnable taps of D and beta; forward and backward are
the library's ct_unrolled_forward / ct_unrolled_backward (checkpointed
forward, hand-written adjoint kernels).  These classes only route tensors to
the C ABI.
"""
from __future__ import annotations

import torch

from . import ctpd as _c


class Project(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, x):
        ctx.g = g
        return _c.ct_project(g, x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return None, _c.ct_backproject(ctx.g, gy.contiguous())


class Backproject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, y):
        ctx.g = g
        return _c.ct_backproject(g, y.contiguous())

    @staticmethod
    def backward(ctx, gx):
        return None, _c.ct_project(ctx.g, gx.contiguous())


def project(g, x):
    return Project.apply(g, x)


def backproject(g, y):
    return Backproject.apply(g, y)


class UnrolledPDTV(torch.autograd.Function):
    """x_K = unrolled solve(b, w; taps, beta).  Gradients flow to `taps`
    (2h-1 centred values) and `beta` (a 0-d tensor)."""

    @staticmethod
    def forward(ctx, taps, beta, g, b, w, tau, sigma, mode, iters, tv_iters):
        taps = taps.detach().contiguous().float()
        bval = float(beta.detach())
        batch = b.numel() // (g.n_views * g.n_bins)
        half = (taps.numel() + 1) // 2
        ws = torch.empty(_c.ct_unrolled_workspace_bytes(g, batch, half, iters, tv_iters), dtype=torch.uint8,
                         device=b.device)
        x = _c.ct_unrolled_forward(g, b, w, taps, tau, sigma, bval, mode, iters, tv_iters, ws)
        ctx.args = (g, b, w, taps, tau, sigma, bval, mode, iters, tv_iters, ws)
        return x

    @staticmethod
    def backward(ctx, gx):
        g, b, w, taps, tau, sigma, bval, mode, iters, tv_iters, ws = ctx.args
        grad = _c.ct_unrolled_backward(g, b, w, taps, tau, sigma, bval, mode, iters, tv_iters, gx, ws)
        n = taps.numel()
        return grad[:n], grad[n], None, None, None, None, None, None, None, None


class UnrolledReconstructor(torch.nn.Module):
    """K unrolled iterations of Algorithm 1 with a learnable log beta and a
    learnable symmetric preconditioner: `half` one-sided taps t[0..half-1],
    mirrored to 2 half - 1 centred taps.  tau and sigma stay fixed."""

    def __init__(self, g, taps_centred: torch.Tensor, beta: float, tau: float, sigma: float,
                 iters: int = 10, tv_iters: int = 10, half: int = 128, mode: int = _c.CT_LOWDOSE):
        super().__init__()
        h0 = (taps_centred.numel() + 1) // 2
        one_sided = taps_centred[h0 - 1:h0 - 1 + half].detach().clone().float()
        self.taps_half = torch.nn.Parameter(one_sided)
        self.log_beta = torch.nn.Parameter(torch.tensor(float(beta)).log().to(taps_centred.device))
        self.g, self.tau, self.sigma, self.iters, self.tv_iters, self.mode = g, tau, sigma, iters, tv_iters, mode

    def taps(self):
        t = self.taps_half
        return torch.cat([t.flip(0)[:-1], t])

    def forward(self, b, w):
        return UnrolledPDTV.apply(self.taps(), self.log_beta.exp(), self.g, b, w, self.tau, self.sigma,
                                  self.mode, self.iters, self.tv_iters)
