"""``PhiSOX``: the Luttinger-Ward functional of SOX as a torch.autograd.Function.

Forward calls ``phi_sox`` (phi[s] = 1/4 sum_j w_j Tr[Sigma(tau_j) G(-tau_j)])
and keeps Sigma; backward turns the kept Sigma into dPhi/dG with
``phi_sox_grad_G`` (the conserving identity, no recomputation) and calls the
adjoint ``phi_sox_backward`` for X and V.  All of it runs in the library's CUDA
kernels; this module only moves pointers.
"""
from __future__ import annotations

import torch

from . import _binding as B


class PhiSOX(torch.autograd.Function):
    """phi = PhiSOX.apply(G, X, V, w, handle, problem) -> tensor [n_spin].

    G [n_spin][1][n_tau][n][n], X [1][N][n], V [1][N][N], w [n_tau]; float64
    CUDA tensors.  Gradients flow to G, X and V.
    """

    @staticmethod
    def forward(ctx, G, X, V, w, handle, prob):
        phi = torch.empty(prob.n_spin, dtype=torch.float64, device=G.device)
        sigma = torch.empty_like(G) if ctx.needs_input_grad[0] else None
        B.phi_sox(handle, prob, G, X, V, w, phi, sigma)
        ctx.save_for_backward(G, X, V, w, sigma)
        ctx.handle, ctx.prob = handle, prob
        return phi

    @staticmethod
    def backward(ctx, dphi):
        G, X, V, w, sigma = ctx.saved_tensors
        need_g, need_x, need_v = ctx.needs_input_grad[:3]
        dphi = dphi.contiguous()
        dG = torch.empty_like(G) if need_g else None
        dX = torch.empty_like(X) if need_x else None
        dV = torch.empty_like(V) if need_v else None
        if need_g:
            B.phi_sox_grad_G(ctx.handle, ctx.prob, sigma, w, dphi, dG)
        if need_x or need_v:
            B.phi_sox_backward(ctx.handle, ctx.prob, G, X, V, w, dphi, None, dX, dV)
        return dG, dX, dV, None, None, None
