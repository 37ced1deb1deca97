"""torch.autograd wrappers of the library calls for gradients through a solve.

The forward and backward passes are library calls (hm_solve, hm_solve with
trans = 1, hm_matvec with trans = 1, hm_potential and its adjoint); only the
elementwise scaling by the per-panel coefficients is written in torch.

    alpha = DensitySolve.apply(A, f, c, opts)  solves  H diag(c) alpha = f
    phi   = Potential.apply(tree, points, alpha) is  E alpha,  E the
            single-layer potential of the panel basis at the points (Sec. 2.1)

Backward of the solve (adjoint method): with g = dL/dalpha the adjoint lam
solves (H diag(c))^T lam = g, i.e. H^T lam = g / c, and

    dL/df = lam,        dL/dc = -alpha * (H^T lam).

No Krylov basis of the forward solve is kept: the adjoint solve starts from
scratch and needs only alpha and c.
"""
from __future__ import annotations

import torch

from . import hm_matvec, hm_potential, hm_solve


def _solve(A, b, trans, opts):
    x = torch.zeros_like(b)
    info = hm_solve(A, b.contiguous(), x, trans=trans, **opts)
    return x, info


class DensitySolve(torch.autograd.Function):
    """alpha with H diag(c) alpha = f (f, c: CUDA float64 [n], original order)."""

    @staticmethod
    def forward(ctx, A, f, c, opts):
        y, _ = _solve(A, f.detach(), 0, opts)
        alpha = y / c.detach()
        ctx.A, ctx.opts = A, opts
        ctx.save_for_backward(alpha, c.detach())
        return alpha

    @staticmethod
    def backward(ctx, g):
        alpha, c = ctx.saved_tensors
        lam, _ = _solve(ctx.A, (g / c).contiguous(), 1, ctx.opts)
        h = torch.empty_like(lam)
        hm_matvec(ctx.A, lam, h, trans=1)
        return None, lam, -alpha * h, None


class Potential(torch.autograd.Function):
    """E alpha at the points ([n_points, 3] CUDA float64)."""

    @staticmethod
    def forward(ctx, tree, points, alpha):
        ctx.tree = tree
        ctx.save_for_backward(points)
        return hm_potential(tree, points, alpha.detach().contiguous())

    @staticmethod
    def backward(ctx, g):
        (points,) = ctx.saved_tensors
        return None, None, hm_potential(ctx.tree, points, g.contiguous(), trans=1)


def misfit_loss(A, tree, f, c, points, target, opts):
    """L = mean_k (E alpha - target)_k^2 with H diag(c) alpha = f."""
    alpha = DensitySolve.apply(A, f, c, opts)
    phi = Potential.apply(tree, points, alpha)
    return torch.mean((phi - target) ** 2)
