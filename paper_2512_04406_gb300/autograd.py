"""torch.autograd wrappers over the C ABI (argument marshalling only).

SubproblemValue: Psi_k(Y) of the factorised ALM subproblem (Section 4, Eq. (Sub-k)).
  forward   manidsdp_subproblem_eval        -> Psi
  backward  its Riemannian gradient kernel  -> grad Psi = 2 X Y          (Proposition 4.2)
  backward of the backward: the Hessian-vector kernel -> Hess Psi[V]     (Eq. (4.7))
The derivatives are the manifold ones: for tangent perturbations V of Y on the
oblique manifold, <grad, V> is the first derivative of Psi along any curve
through Y with velocity V, and Hess[V] the covariant derivative of the gradient.

SDPValue: the optimal value V(b, C) of (DSDP) computed by Algorithm 1.  By the
envelope theorem applied to (PSDP), whose objective is <C, X + Diag z> + sum(z)
subject to A(X + Diag z) = b, the sensitivities at a unique optimum are
  dV/db = y*        and        dV/dC = X* + Diag(z*) = Xt* + D,
the converged multiplier plus D (Algorithm 1, steps 5-8).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Context, PREC_FP64, manidsdp_default_params, manidsdp_destroy,
               manidsdp_get_dual_matrix, manidsdp_hessvec, manidsdp_setup, manidsdp_solve,
               manidsdp_subproblem_eval)


class _Handle:
    """Holds a context and the Y at which its G was last evaluated."""

    def __init__(self, ctx: Context, N: int, m: int, precision: int = PREC_FP64):
        self.ctx, self.N, self.m, self.precision = ctx, N, m, precision
        self.Y = None


class _Grad(torch.autograd.Function):
    @staticmethod
    def forward(fctx, Y, handle: _Handle):
        p = Y.shape[1]
        g = torch.empty_like(Y)
        manidsdp_subproblem_eval(handle.ctx, Y, p, rgrad=g)
        handle.Y = Y
        fctx.handle = handle
        fctx.save_for_backward(Y)
        return g

    @staticmethod
    def backward(fctx, V):
        (Y,) = fctx.saved_tensors
        h = fctx.handle
        p = Y.shape[1]
        if h.Y is not Y:
            manidsdp_subproblem_eval(h.ctx, Y, p)
            h.Y = Y
        HV = torch.empty_like(Y)
        manidsdp_hessvec(h.ctx, Y, V.contiguous(), p, HV, h.precision)
        return HV, None


class SubproblemValue(torch.autograd.Function):
    @staticmethod
    def forward(fctx, Y, handle: _Handle):
        p = Y.shape[1]
        psi, _ = manidsdp_subproblem_eval(handle.ctx, Y, p)
        handle.Y = Y
        fctx.handle = handle
        fctx.save_for_backward(Y)
        return torch.tensor(psi, dtype=Y.dtype, device=Y.device)

    @staticmethod
    def backward(fctx, gout):
        (Y,) = fctx.saved_tensors
        return gout * _Grad.apply(Y, fctx.handle), None


class Subproblem:
    """Psi_k as a differentiable function of a CUDA FP64 tensor Y (N x p, unit rows)."""

    def __init__(self, N, m, idx, b, Xt=None, sigma=1.0, precision=PREC_FP64):
        from . import manidsdp_set_state
        prm = manidsdp_default_params()
        prm.precision_mode = precision
        self.handle = _Handle(manidsdp_setup(N, m, idx, b, params=prm), N, m, precision)
        manidsdp_set_state(self.handle.ctx, Xt, sigma)

    def __call__(self, Y):
        return SubproblemValue.apply(Y, self.handle)

    def close(self):
        manidsdp_destroy(self.handle.ctx)


class SDPValue(torch.autograd.Function):
    """V = value of (DSDP) for the right-hand side b and a dense symmetric cost C
    (None: C = 0): forward solves with Algorithm 1; backward returns gout * y*
    for b and gout * (Xt* + D) for C (envelope theorem on (PSDP))."""

    @staticmethod
    def forward(fctx, b, C, N, m, idx, Y0, params):
        from . import C_DENSE, C_ZERO
        bh = b.detach().cpu().numpy().astype(np.float64)
        ch = None if C is None else np.ascontiguousarray(C.detach().cpu().numpy(), dtype=np.float64)
        ctx = manidsdp_setup(N, m, idx, bh, C_DENSE if ch is not None else C_ZERO, ch,
                             params=params)
        try:
            y = np.empty(m)
            rep, _ = manidsdp_solve(ctx, Y0, Y0.shape[1], y_out=y)
            XD = np.empty((N, N))
            manidsdp_get_dual_matrix(ctx, XD)
        finally:
            manidsdp_destroy(ctx)
        fctx.save_for_backward(torch.tensor(y, dtype=b.dtype, device=b.device),
                               torch.tensor(XD, dtype=b.dtype, device=b.device))
        fctx.has_C = C is not None
        fctx.report = rep
        return torch.tensor(rep.value, dtype=b.dtype, device=b.device)

    @staticmethod
    def backward(fctx, gout):
        y, XD = fctx.saved_tensors
        return gout * y, (gout * XD if fctx.has_C else None), None, None, None, None, None


def value_and_sensitivities(N, m, idx, b, Y0, params=None):
    """Solve once; return (report, y* = dV/db, Xt* + D = dV/dC) as NumPy arrays."""
    ctx = manidsdp_setup(N, m, idx, b, params=params)
    try:
        y = np.empty(m)
        rep, _ = manidsdp_solve(ctx, Y0, Y0.shape[1], y_out=y)
        XD = np.empty((N, N))
        manidsdp_get_dual_matrix(ctx, XD)
    finally:
        manidsdp_destroy(ctx)
    return rep, y, XD
