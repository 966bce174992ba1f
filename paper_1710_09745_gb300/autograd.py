"""Differentiable block solve x = A(U)^-1 phi for PyTorch autograd.

Forward: the block-CGrQ solve of the library (Algorithm 1 with reliable
updates) for the links U = (fat, long) and the right-hand sides phi.
Backward, given g = dL/dx: the adjoint block lam = A^-1 g is a second block
solve with the same handle (A is Hermitian, Sec. 3.2), the gradient with
respect to phi is lam, and the gradient with respect to the links comes from
the library's outer-product kernel (blockcg_link_grad):
    dL = Re[lam^dag dD_eo y] + Re[x^dag dD_eo mu],  y = D_oe x, mu = D_oe lam.
Gradients follow PyTorch's convention for complex inputs of a real loss,
dL/dRe + i dL/dIm.  All arithmetic runs in the library's kernels; this module
only orders the calls.
"""
from __future__ import annotations

import torch

from .binding import BlockCG, BlockCGError


class HisqSolve(torch.autograd.Function):
    """x = A(fat, lng)^-1 phi with phi of shape (N, V/2, 3), complex128."""

    @staticmethod
    def forward(ctx, fat, lng, phi, solver: BlockCG, tol: float):
        fat_d, lng_d = fat.detach(), lng.detach()
        solver.load_gauge(fat_d, lng_d)
        X, info = solver.solve(phi.detach(), tol=tol)
        if info["status"] != 0:
            raise BlockCGError(info["status"], "forward solve did not converge")
        ctx.save_for_backward(X, fat_d, lng_d)
        ctx.solver, ctx.tol = solver, tol
        return X

    @staticmethod
    def backward(ctx, gX):
        X, fat_d, lng_d = ctx.saved_tensors
        solver = ctx.solver
        need_f, need_l, need_phi = ctx.needs_input_grad[:3]
        if not (need_f or need_l or need_phi):
            return None, None, None, None, None
        keep = getattr(solver, "_links_keepalive", (None, None))
        if keep[0] is not fat_d or keep[1] is not lng_d:  # links changed since forward
            solver.load_gauge(fat_d, lng_d)
        Lam, info = solver.solve(gX.resolve_conj().contiguous(), tol=ctx.tol)
        if info["status"] != 0:
            raise BlockCGError(info["status"], "adjoint solve did not converge")
        gf = gl = None
        if need_f or need_l:
            gf, gl = solver.link_grad(X, Lam, fat=need_f, lng=need_l)
        return gf, gl, (Lam if need_phi else None), None, None


def hisq_solve(fat, lng, phi, solver: BlockCG, tol: float = 1e-10):
    """Differentiable x = A^-1 phi; phi (N, V/2, 3) or (V/2, 3) complex128."""
    squeeze = phi.dim() == 2
    if squeeze:
        phi = phi.unsqueeze(0)
    x = HisqSolve.apply(fat, lng, phi, solver, tol)
    return x[0] if squeeze else x
