"""torch.autograd front ends of the library (argument marshalling only).

NegLogPosterior: L(s) = -ln P(s | N) up to constants (Sec. 2.1 likelihood,
Sec. 2.3 prior) as a differentiable scalar of s.  The forward pass is one
plc_logpost_grad call, which produces L and its gradient (Sec. 3.1.2)
g = S^-1 (s - mu) + nbar w e^s - N in the same pipeline; the backward pass
returns grad_out * g.  Works in the context's field precision (FP64, or FP32
for a mixed context).

MapField: the MAP s*(N, ln A) of plc_newton_krylov_map as a differentiable
function of the counts (taken as reals) and of the log-amplitude ln A of the
prior power spectrum (P -> A P).  Its backward pass is the implicit adjoint
plc_map_vjp: the stationarity condition g(s*) = 0 gives ds*/dN = H^-1 and
ds*/d ln A = H^-1 S^-1 (s* - mu), so a cotangent u costs one CG solve
lam = H^-1 u at the converged state (nothing is stored per iteration).
The forward pass records the prior it solved with (the scaled table, mu and
the DC inverse eigenvalue); the backward pass puts that prior back on the
context if another call has changed it since, so several MAP fields taken on
one context each get the adjoint of their own amplitude.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import torch

from ._lib import Context


class NegLogPosterior(torch.autograd.Function):
    """f = NegLogPosterior.apply(s, ctx, N, w, nbar) -> 0-d float64 tensor."""

    @staticmethod
    def forward(fctx, s: torch.Tensor, ctx: Context, N: torch.Tensor,
                w: Optional[torch.Tensor], nbar: float):
        need = s.requires_grad
        f, g = ctx.logpost_grad(s.detach(), N, w, nbar, want_grad=need)
        if need:
            fctx.save_for_backward(g)
        return torch.tensor(f, dtype=torch.float64, device=s.device)

    @staticmethod
    def backward(fctx, grad_out: torch.Tensor):
        (g,) = fctx.saved_tensors
        return (grad_out.to(g.dtype) * g), None, None, None, None


def neg_log_posterior(s: torch.Tensor, ctx: Context, N: torch.Tensor,
                      w: Optional[torch.Tensor] = None, nbar: float = 1.0) -> torch.Tensor:
    return NegLogPosterior.apply(s, ctx, N, w, nbar)


class MapField(torch.autograd.Function):
    """s* = MapField.apply(N, ln_amp, ctx, k, P, mu, inv_lambda_dc, w, nbar, opts).

    N: float64 counts (whole numbers; cast to int32 for the solve);
    ln_amp: 0-d float64 tensor, the prior is P(k) e^{ln_amp} (the DC inverse
    eigenvalue inv_lambda_dc is not scaled: the amplitude multiplies the
    non-DC eigenvalues);
    opts: dict of plc_opts fields for both the solve and the adjoint CG.
    """

    @staticmethod
    def forward(fctx, N: torch.Tensor, ln_amp: torch.Tensor, ctx: Context, k, P, mu: float,
                inv_lambda_dc: float, w: Optional[torch.Tensor], nbar: float, opts: dict):
        amp = float(torch.exp(ln_amp.detach().double()).item())
        prior = (np.array(k, dtype=np.float64), np.asarray(P, dtype=np.float64) * amp,
                 float(mu), float(inv_lambda_dc))
        ctx.set_prior(*prior)
        Ni = N.detach().round().to(torch.int32)
        res = ctx.newton_krylov_map(Ni, w, nbar, **opts)
        fctx.ctx, fctx.w, fctx.nbar, fctx.opts, fctx.prior = ctx, w, nbar, opts, prior
        fctx.save_for_backward(res.s)
        return res.s.clone()

    @staticmethod
    def backward(fctx, u: torch.Tensor):
        (s,) = fctx.saved_tensors
        if not fctx.ctx.prior_is(*fctx.prior):
            fctx.ctx.set_prior(*fctx.prior)
        vjp_N, vjp_lnA, _ = fctx.ctx.map_vjp(s, fctx.w, fctx.nbar,
                                             u.detach().double().contiguous(), **fctx.opts)
        g_lnA = torch.tensor(vjp_lnA, dtype=torch.float64, device=s.device)
        return vjp_N, g_lnA, None, None, None, None, None, None, None, None


def map_field(N: torch.Tensor, ln_amp: torch.Tensor, ctx: Context, k, P, mu: float,
              w: Optional[torch.Tensor] = None, nbar: float = 1.0, inv_lambda_dc: float = 0.0,
              **opts) -> torch.Tensor:
    return MapField.apply(N, ln_amp, ctx, k, P, mu, inv_lambda_dc, w, nbar, opts)
