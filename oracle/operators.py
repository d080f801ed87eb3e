"""Linear operators of the dual formulation (Section 2, Section 3, Eq.
(projection-operators) and Eq. (projected-y)).

With A_alpha the 0/1 indicator of the entries mapped to monomial alpha:
  A(Z)_alpha      = sum of Z over the entries of alpha
  A*(v)[b, g]     = v[idx[b, g]]
  A A*            = Diag(mult)                     (orthogonal indicators)
  y(S)            = (A A*)^{-1} A(S + C)           (variable projection)
  P               = A* (A A*)^{-1} A,  Q = I - P   (orthogonal projectors)
  D               = A* (A A*)^{-1} b
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cho_solve


def A(Z: np.ndarray, idx: np.ndarray, m: int) -> np.ndarray:
    return np.bincount(idx.ravel(), weights=Z.ravel(), minlength=m)


def Astar(v: np.ndarray, idx: np.ndarray) -> np.ndarray:
    return v[idx]


def AAstar(v: np.ndarray, idx: np.ndarray, m: int) -> np.ndarray:
    """A(A*(v)), used to pin that A A* is the diagonal of multiplicities."""
    return A(Astar(v, idx), idx, m)


def y_of(S: np.ndarray, C: np.ndarray | None, idx, mult) -> np.ndarray:
    Z = S if C is None else S + C
    return A(Z, idx, len(mult)) / mult


def P(Z: np.ndarray, idx, mult) -> np.ndarray:
    return Astar(A(Z, idx, len(mult)) / mult, idx)


def Q(Z: np.ndarray, idx, mult) -> np.ndarray:
    return Z - P(Z, idx, mult)


def D_matrix(b: np.ndarray, idx, mult) -> np.ndarray:
    return Astar(b / mult, idx)


# ---- the operators of a problem dict: 0/1 classes (idx, mult) or a general A ----
# A general operator is held as the m x N^2 matrix Amat of the vectorised
# constraint matrices, with the Cholesky factor Mfac of A A* computed once (the
# remark after Algorithm 1: A A* is factored once and reused).

def y_prob(Z: np.ndarray, prob) -> np.ndarray:
    """(A A*)^{-1} A(Z)."""
    if prob.get("Amat") is not None:
        return cho_solve(prob["Mfac"], prob["Amat"] @ Z.ravel())
    return A(Z, prob["idx"], len(prob["mult"])) / prob["mult"]


def Astar_prob(v: np.ndarray, prob) -> np.ndarray:
    if prob.get("Amat") is not None:
        N = prob["N"]
        return (prob["Amat"].T @ v).reshape(N, N)
    return Astar(v, prob["idx"])


def Q_prob(Z: np.ndarray, prob) -> np.ndarray:
    return Z - Astar_prob(y_prob(Z, prob), prob)

