"""torch.autograd wrappers of the library calls for gradients through a solve.

The forward and backward passes are library calls only (hm_solve_scaled and
its transposed form, hm_matvec_scaled, hm_potential and its adjoint); this
module marshals tensors between them and autograd.

    alpha = DensitySolve.apply(A, f, c, opts)  solves  H diag(c) alpha = f
    phi   = Potential.apply(tree, points, alpha) is  E alpha,  E the
            single-layer potential of the panel basis at the points (Sec. 2.1)

Backward of the solve (adjoint method): with g = dL/dalpha the adjoint lam
solves (H diag(c))^T lam = g, and

    dL/df = lam,        dL/dc = -alpha * (H^T lam)   (hm_matvec_scaled).

No Krylov basis of the forward solve is kept: the adjoint solve starts from
scratch and needs only alpha and c.
"""
from __future__ import annotations

import torch

from . import hm_matvec_scaled, hm_potential, hm_solve_scaled


class DensitySolve(torch.autograd.Function):
    """alpha with H diag(c) alpha = f (f, c: CUDA float64 [n], original order)."""

    @staticmethod
    def forward(ctx, A, f, c, opts):
        c = c.detach().contiguous()
        alpha = torch.empty_like(f)
        hm_solve_scaled(A, f.detach().contiguous(), c, alpha, trans=0, **opts)
        ctx.A, ctx.opts = A, opts
        ctx.save_for_backward(alpha, c)
        return alpha

    @staticmethod
    def backward(ctx, g):
        alpha, c = ctx.saved_tensors
        lam = torch.empty_like(alpha)
        hm_solve_scaled(ctx.A, g.contiguous(), c, lam, trans=1, **ctx.opts)
        dc = torch.empty_like(alpha)
        hm_matvec_scaled(ctx.A, lam, dc, trans=1, left=alpha, alpha=-1.0)
        return None, lam, dc, None


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
