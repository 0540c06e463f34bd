"""torch.autograd.Function for the pseudofermion action (Sec. 2, eq. "pseudo
fermions"; Sec. 2.2, fermion force through dD^-1 = -D^-1 dD D^-1).

``FermionAction.apply(omega, U, phi, kappa, mu, params)`` returns
S = phi^+ (Mhat^+ Mhat)^-1 phi for the gauge field U and the even-site
pseudofermion phi.  omega (float64 [4, V, 8]) holds the algebra coordinates
of a variation U_mu(x) -> exp(i omega^a T^a) U_mu(x) and must be zero: the
function is evaluated at the field U itself (the point where the HMC needs
the force), and dS/domega there is the derivative with respect to every
link.  A nonzero omega raises ValueError rather than returning the action
of the wrong field.  The forward pass calls ``lqcd_fermion_force`` (one CG
solve X = (Mhat^+ Mhat)^-1 phi and one adjoint kernel over all links) and
keeps the [4, V, 8] gradient for the backward pass, which scales it by the
incoming gradient.  With ``recompute=True`` the forward pass computes the
action alone (the solve, no force kernel, no gradient buffer) and the
backward pass solves for X again and runs the force kernel: a second solve
traded for the memory of the gradient between the two passes.
"""
from __future__ import annotations

import torch

from . import lqcd


class FermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx_, omega: torch.Tensor, U: "lqcd.Gauge", phi: "lqcd.lqcd_field", kappa: float,
                mu: float, params: "lqcd.lqcd_cg_params", recompute: bool = False):
        if omega.dtype != torch.float64 or not omega.is_cuda or omega.dim() != 3:
            raise ValueError("omega must be a CUDA float64 tensor [4, V, 8]")
        # two reductions, no temporary of omega's size (recompute keeps memory flat)
        if omega.amax().item() != 0.0 or omega.amin().item() != 0.0:
            raise ValueError("FermionAction is evaluated at omega = 0 (the field U itself); "
                             "apply the variation to U instead")
        ctx_.U, ctx_.phi, ctx_.kappa, ctx_.mu, ctx_.params = U, phi, kappa, mu, params
        ctx_.recompute = recompute
        if recompute:  # the action alone: no force kernel, no gradient kept
            S, _ = lqcd.lqcd_fermion_force(U.ctx, U, phi, None, kappa, mu, params)
            ctx_.grad = None
            ctx_.shape = omega.shape
        else:
            grad = torch.empty_like(omega)
            S, _ = lqcd.lqcd_fermion_force(U.ctx, U, phi, grad, kappa, mu, params)
            ctx_.grad = grad
        return omega.new_tensor(S)

    @staticmethod
    def backward(ctx_, grad_out):
        if ctx_.recompute:
            grad = torch.empty(ctx_.shape, dtype=torch.float64, device="cuda")
            lqcd.lqcd_fermion_force(ctx_.U.ctx, ctx_.U, ctx_.phi, grad, ctx_.kappa, ctx_.mu,
                                    ctx_.params)
        else:
            grad = ctx_.grad
        return grad * grad_out, None, None, None, None, None, None
