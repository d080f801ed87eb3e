"""First-order relaxation of the unit-modulus complex quadratic program
min z^H Q z over |z_i| = 1 (Q Hermitian): min <Q, X> over Hermitian X >= 0 with
diag X = 1 -- the complex counterpart of the BQP relaxations of Section 3.1,
solved in the factorised form of Section 4 with a complex factor.

In ManiDSDP's terms every off-diagonal entry of this relaxation is a class of
its own, so the projector residual R vanishes on the manifold, the multiplier
stays 0, and one ALM step is the whole solve: a rank-adaptive Riemannian trust
region on the complex oblique manifold

    { Y in C^{n x p} : |Y_i| = 1 for every row i },   f(Y) = Re tr(Y^H Q Y),

certified by the dual matrix X = Q - Diag(mu), mu_i = Re (Q Y Y^H)_ii
(Lemma 4.1 and Proposition 4.2 with G = Q; Theorem 4.5 for the escape
direction [0, v] when lambda_min(X) < 0).

Test infrastructure: only tests/, the smoke check and bench.py's CPU baseline
use this module.

Representation: the generic trust region (oracle/rtr.py) works with real
arrays and the inner product sum(a * b).  A complex factor Y = A + iB is held
as the real n x 2p array [A, B]; then sum(a * b) over such arrays equals
Re <a, b> of the complex factors, the row norms agree, and the complex oblique
manifold is exactly the real oblique manifold of the stacked rows.
"""
from __future__ import annotations

import math

import numpy as np

from . import rtr as rtr_mod


def to_complex(Yr: np.ndarray) -> np.ndarray:
    p = Yr.shape[1] // 2
    return Yr[:, :p] + 1j * Yr[:, p:]


def to_real(Y: np.ndarray) -> np.ndarray:
    return np.concatenate([Y.real, Y.imag], axis=1)


def rowdot(A_: np.ndarray, B_: np.ndarray) -> np.ndarray:
    """Re <A_i, B_i> for each row i (complex rows)."""
    return np.real(np.sum(np.conj(A_) * B_, axis=1))


def proj_tangent(Y: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Tangent space of the complex oblique manifold at Y: Re <Y_i, U_i> = 0."""
    return U - rowdot(Y, U)[:, None] * Y


def retract(Y: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Row normalisation of Y + U."""
    Z = Y + U
    return Z / np.linalg.norm(Z, axis=1)[:, None]


def cost(Y: np.ndarray, Q: np.ndarray) -> float:
    """f(Y) = Re tr(Y^H Q Y) = <Q, Y Y^H> for Hermitian Q."""
    return float(np.real(np.sum(np.conj(Y) * (Q @ Y))))


def multipliers(Y: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """mu_i = Re (Q Y Y^H)_ii = Re <Y_i, (Q Y)_i>."""
    return rowdot(Y, Q @ Y)


def certificate(Y: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """X = Q - Diag(mu): the dual slack of the relaxation at Y."""
    return Q - np.diag(multipliers(Y, Q))


def rgrad(Y: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Riemannian gradient: P_Y(2 Q Y) = 2 X Y."""
    return proj_tangent(Y, 2.0 * (Q @ Y))


def rhess(Y: np.ndarray, U: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """Riemannian Hessian on the product of spheres: P_Y(2 Q U) - 2 Diag(mu) U,
    applied to P_Y(U)."""
    U = proj_tangent(Y, U)
    return proj_tangent(Y, 2.0 * (Q @ U)) - 2.0 * multipliers(Y, Q)[:, None] * U


def kkt(Y: np.ndarray, Q: np.ndarray):
    """(eta_d, eta_g, lambda_min, lambda_max, primal f, dual sum(mu)); eta_p = 0
    because diag(Y Y^H) = 1 holds exactly on the manifold."""
    mu = multipliers(Y, Q)
    w = np.linalg.eigvalsh(Q - np.diag(mu))
    f = cost(Y, Q)
    d = float(np.sum(mu))
    eta_d = max(0.0, -w[0]) / (1.0 + abs(w[-1]))
    eta_g = abs(f - d) / (1.0 + abs(f) + abs(d))
    return eta_d, eta_g, float(w[0]), float(w[-1]), f, d


def solve(Q: np.ndarray, Y0: np.ndarray, tol: float = 1e-10, p_max: int = 64,
          max_outer: int = 50, tol_grad: float = 1e-11, neg_tol: float = 1e-12):
    """Rank-adaptive trust region to KKT residual <= tol.  Each round: RTR on f
    at the current rank; if lambda_min(X) < -neg_tol (1 + |lambda_max|), append a
    zero column and move along [0, v] (v the eigenvector of lambda_min, which is
    a descent direction of second order: its curvature is 2 v^H X v < 0, the
    complex form of Theorem 4.5) by backtracking on f."""
    n = Q.shape[0]
    Y = Y0 / np.linalg.norm(Y0, axis=1)[:, None]
    Delta_bar = math.pi * math.sqrt(n)
    hist = []
    for k in range(max_outer):
        Yr, info = rtr_mod.rtr(
            to_real(Y),
            lambda x: cost(to_complex(x), Q),
            lambda x: to_real(rgrad(to_complex(x), Q)),
            lambda x, u: to_real(rhess(to_complex(x), to_complex(u), Q)),
            lambda x, u: to_real(retract(to_complex(x), to_complex(u))),
            Delta_bar, tol_grad, max_iter=500)
        Y = to_complex(Yr)
        eta_d, eta_g, lmin, lmax, f, d = kkt(Y, Q)
        hist.append(dict(p=Y.shape[1], f=f, eta_d=eta_d, eta_g=eta_g, lmin=lmin,
                         hessvecs=info["hessvecs"]))
        if max(eta_d, eta_g) <= tol:
            break
        if lmin >= -neg_tol * (1.0 + abs(lmax)) or Y.shape[1] >= p_max:
            continue
        w, V = np.linalg.eigh(certificate(Y, Q))
        v = V[:, 0]
        Ya = np.concatenate([Y, np.zeros((n, 1), dtype=Y.dtype)], axis=1)
        U = np.zeros_like(Ya)
        U[:, -1] = v
        f0 = cost(Ya, Q)
        curv = 2.0 * float(np.real(np.vdot(v, certificate(Y, Q) @ v)))
        t = math.sqrt(n)
        for _ in range(40):
            Yt = retract(Ya, t * U)
            if cost(Yt, Q) <= f0 - 1e-4 * 0.5 * t * t * abs(curv):
                Ya = Yt
                break
            t *= 0.5
        Y = Ya
    eta_d, eta_g, lmin, lmax, f, d = kkt(Y, Q)
    return dict(Y=Y, value=f, dual=d, eta_d=eta_d, eta_g=eta_g, eta_max=max(eta_d, eta_g),
                lambda_min=lmin, lambda_max=lmax, p=Y.shape[1], history=hist)
