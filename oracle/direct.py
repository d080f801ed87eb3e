"""The direct formulation: two-block ADMM applied to (DSDP) itself rather than to
the variable-projected (DSDP') (Section 3, the comparison of the reduced
subproblem with the direct one; Eq. (direct-augmented-lagrangian),
(direct-ALM-subproblem), (penalty-decomposition), (hessian-comparison)).

After its first multiplier update the direct scheme keeps A(Xbar) = b, so
Xbar = D + W with A(W) = 0, and its y-update gives A*(y^k) = P(Z^k) with
Z^k = S^k + C.  Its S-subproblem, up to terms independent of S, is

    Psi_dir(Y) = <D + W, Z> + sigma/2 ||A*(y^k) - Z||^2,   Z = Y Y' + C,

the reduced subproblem plus sigma/2 ||P(Z - Z^k)||^2: the same function with
y frozen at the stale y^k instead of the best response y(S).  Hence

    grad_S Phi_dir = W + D - sigma (A*(y^k) - Z)            (G with the stale y)
    Hess Psi_dir(Y)[U] = H - Diag(H Y') Y - 2 Diag(z) U,
        H = 2 G U + 2 sigma (Y U' + U Y') Y,  z = diag(G Y Y')  (Eq. (4.7) with Q -> I)

Test infrastructure: only tests/ use this module.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops
from . import subproblem as sp


def stale_residual(Y, prob, y_prev):
    """A*(y^k) - Z at the current Y."""
    return ops.Astar_prob(y_prev, prob) - sp.Zmat(Y, prob)


def cost(Y, prob, W, sigma, y_prev) -> float:
    Z = sp.Zmat(Y, prob)
    R = ops.Astar_prob(y_prev, prob) - Z
    return float(np.sum((prob["D"] + W) * Z) + 0.5 * sigma * np.sum(R * R))


def lagrangian(Y, prob, Xbar, sigma, y) -> float:
    """The direct augmented Lagrangian L^_sigma(S, y, Xbar) of Eq.
    (direct-augmented-lagrangian), at S = Y Y'."""
    R = ops.Astar_prob(y, prob) - sp.Zmat(Y, prob)
    return float(prob["b"] @ y - np.sum(Xbar * R) + 0.5 * sigma * np.sum(R * R))


def egrad_S(Y, prob, W, sigma, y_prev) -> np.ndarray:
    return W + prob["D"] - sigma * stale_residual(Y, prob, y_prev)


def rgrad(Y, prob, W, sigma, y_prev) -> np.ndarray:
    return sp.proj_tangent(Y, 2.0 * egrad_S(Y, prob, W, sigma, y_prev) @ Y)


def rhess(Y, U, prob, W, sigma, y_prev, G=None) -> np.ndarray:
    if G is None:
        G = egrad_S(Y, prob, W, sigma, y_prev)
    U = sp.proj_tangent(Y, U)
    H = 2.0 * G @ U + 2.0 * sigma * (Y @ U.T + U @ Y.T) @ Y
    z = sp.rowdot(G @ Y, Y)
    return H - sp.rowdot(H, Y)[:, None] * Y - 2.0 * z[:, None] * U
