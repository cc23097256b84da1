"""torch.autograd.Function wrappers over the library's analytic adjoint.

LocalGP        d (per location), g  ->  local predictive mean and scale s2
               (Eqs. predgp, preds2 on fixed local designs);
LocalLogLik    d (per location), g  ->  local log-likelihood of Eq. (gpk).
Forward values come from lagp_predict / lagp_mle_step (max_iter = 0);
backward uses lagp_predict_grad, whose FP64 kernel differentiates the
equations through d(K^{-1}) = -K^{-1} dK K^{-1}.  The gradients are with
respect to d (one per location) and the shared nugget g (a scalar: the sum
over locations).  Inputs X, Y, Xref, sel are treated as constants.
"""
from __future__ import annotations

import torch

from . import lagp as _L


class LocalGP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, g, X, Y, Xref, sel, n):
        gval = float(g.detach().item()) if isinstance(g, torch.Tensor) else float(g)
        out = _L.lagp_predict(X, Y, Xref, sel, n, d.detach(), gval)
        ctx.save_for_backward(d.detach())
        ctx.args = (X, Y, Xref, sel, n, gval, isinstance(g, torch.Tensor))
        return out["mean"], out["s2"]

    @staticmethod
    def backward(ctx, gmean, gs2):
        (d,) = ctx.saved_tensors
        X, Y, Xref, sel, n, gval, g_is_tensor = ctx.args
        r = _L.lagp_predict_grad(X, Y, Xref, sel, n, d, gval)
        gmean = torch.zeros_like(d) if gmean is None else gmean
        gs2 = torch.zeros_like(d) if gs2 is None else gs2
        grad_d = gmean * r["dmean_dd"] + gs2 * r["ds2_dd"]
        grad_g = (gmean * r["dmean_dg"] + gs2 * r["ds2_dg"]).sum() if g_is_tensor else None
        return grad_d, grad_g, None, None, None, None, None


class LocalLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, d, g, X, Y, Xref, sel, n):
        gval = float(g.detach().item()) if isinstance(g, torch.Tensor) else float(g)
        r = _L.lagp_predict_grad(X, Y, Xref, sel, n, d.detach(), gval)
        ll = _L.lagp_mle_step(X, Y, sel, n, d.detach(), gval, 1e-300, 1e300, 0)["llik"]
        ctx.save_for_backward(r["dllik_dd"], r["dllik_dg"])
        ctx.g_is_tensor = isinstance(g, torch.Tensor)
        return ll

    @staticmethod
    def backward(ctx, gl):
        dd, dg = ctx.saved_tensors
        grad_g = (gl * dg).sum() if ctx.g_is_tensor else None
        return gl * dd, grad_g, None, None, None, None, None


def local_gp(d, g, X, Y, Xref, sel, n):
    """Differentiable local predictive (mean, s2) as functions of d and g."""
    return LocalGP.apply(d, g, X, Y, Xref, sel, n)


def local_loglik(d, g, X, Y, Xref, sel, n):
    """Differentiable local log-likelihood as a function of d and g."""
    return LocalLogLik.apply(d, g, X, Y, Xref, sel, n)
