"""The factorised ALM subproblem on the oblique manifold (Section 4).

Psi_k(Y) = <D + Xt, Y Y' + C> + sigma/2 ||Q(Y Y' + C)||^2   (Eq. (reduced-ALM-subproblem))
grad Phi_k(S) = Xt + D - sigma (A*(y(S)) - S - C)            (Lemma 3.1)
Tangent space  T_Y = {U : diag(U Y') = 0}, projector P_Y(U) = U - Diag(U Y') Y (Lemma 4.1)
grad Psi_k(Y) = 2 X Y,  X = G - Diag(G S)                    (Proposition 4.2)
Hess Psi_k(Y)[U] = H - Diag(H Y') Y - 2 Diag(G S) U,
    H = 2 G U + 2 sigma Q(Y U' + U Y') Y                     (Proposition 4.2)

Retraction (a reading: the paper names none; the oblique manifold's usual
choice): Retr_Y(U) normalises each row of Y + U to unit length.

Every function takes the data as a dict ``prob`` with keys b, C (None for
C = 0), D and the constraint operator (idx, mult for 0/1 classes, or Amat and
the factor Mfac of A A* for a general A), and the ALM state Xt, sigma.
"""
from __future__ import annotations

import numpy as np

from . import operators as ops


def rowdot(A_: np.ndarray, B_: np.ndarray) -> np.ndarray:
    return np.einsum("ij,ij->i", A_, B_)


def proj_tangent(Y: np.ndarray, U: np.ndarray) -> np.ndarray:
    """P_Y(U) = U - Diag(U Y') Y  (Lemma 4.1)."""
    return U - rowdot(U, Y)[:, None] * Y


def retract(Y: np.ndarray, U: np.ndarray) -> np.ndarray:
    W = Y + U
    return W / np.linalg.norm(W, axis=1)[:, None]


def Zmat(Y, prob):
    S = Y @ Y.T
    return S if prob["C"] is None else S + prob["C"]


def residual(Y, prob):
    """R = A*(y(S)) - S - C = -Q(S + C)  (Eq. (projected-y)) and y(S)."""
    Z = Zmat(Y, prob)
    y = ops.y_prob(Z, prob)
    R = ops.Astar_prob(y, prob) - Z
    return R, y


def cost(Y, prob, Xt, sigma) -> float:
    """Psi_k(Y) written as <D + Xt, Z> + sigma/2 ||Q(Z)||^2."""
    Z = Zmat(Y, prob)
    QZ = ops.Q_prob(Z, prob)
    return float(np.sum((prob["D"] + Xt) * Z) + 0.5 * sigma * np.sum(QZ * QZ))


def cost_lagrangian(Y, prob, Xt, sigma) -> float:
    """Psi_k(Y) as L_sigma(S, y(S), Xt) of Section 3 (a second, independent
    statement of the same function, used as a pin)."""
    S = Y @ Y.T
    C = 0.0 if prob["C"] is None else prob["C"]
    y = ops.y_prob(S if prob["C"] is None else S + prob["C"], prob)
    Ay = ops.Astar_prob(y, prob)
    Rr = Ay - S - C
    return float(prob["b"] @ y - np.sum(Xt * Rr) + 0.5 * sigma * np.sum(Rr * Rr))


def egrad_S(Y, prob, Xt, sigma) -> np.ndarray:
    """G = grad Phi_k(S) = Xt + D - sigma R  (Lemma 3.1)."""
    R, _ = residual(Y, prob)
    return Xt + prob["D"] - sigma * R


def certificate(G: np.ndarray, S: np.ndarray):
    """X = G - Diag(diag(G S)) and z = diag(G S)  (Lemma 3.1)."""
    z = np.einsum("ij,ji->i", G, S)
    return G - np.diag(z), z


def rgrad(Y, prob, Xt, sigma) -> np.ndarray:
    """grad Psi_k(Y) = P_Y(2 G Y)  (first line of the proof of Prop. 4.2)."""
    G = egrad_S(Y, prob, Xt, sigma)
    return proj_tangent(Y, 2.0 * G @ Y)


def rgrad_certificate(Y, prob, Xt, sigma) -> np.ndarray:
    """grad Psi_k(Y) = 2 X Y  (Eq. (4.6)), the certificate form."""
    G = egrad_S(Y, prob, Xt, sigma)
    X, _ = certificate(G, Y @ Y.T)
    return 2.0 * X @ Y


def ehess(Y, U, prob, Xt, sigma, G=None) -> np.ndarray:
    """Euclidean Hessian H = 2 G U + 2 sigma Q(Y U' + U Y') Y  (Prop. 4.2)."""
    if G is None:
        G = egrad_S(Y, prob, Xt, sigma)
    W = Y @ U.T + U @ Y.T
    return 2.0 * G @ U + 2.0 * sigma * ops.Q_prob(W, prob) @ Y


def rhess(Y, U, prob, Xt, sigma, G=None) -> np.ndarray:
    """Hess Psi_k(Y)[U] = H - Diag(H Y') Y - 2 Diag(G S) U  (Eq. (4.7)).

    Eq. (4.7) defines the Hessian on T_Y.  It is applied here to P_Y(U), which
    equals U on T_Y and keeps the output tangent when rounding has left U a
    little outside T_Y (the -2 Diag(z) U term would otherwise carry a normal
    component along and amplify it across CG iterations)."""
    if G is None:
        G = egrad_S(Y, prob, Xt, sigma)
    U = proj_tangent(Y, U)
    H = ehess(Y, U, prob, Xt, sigma, G)
    z = rowdot(G @ Y, Y)
    return H - rowdot(H, Y)[:, None] * Y - 2.0 * z[:, None] * U
