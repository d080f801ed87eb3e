"""Moment data of the real second-order relaxation of a unit-modulus complex
quadratic program min x*Qx + Re(c'x), |x_i| = 1, with real Q, c (Section 3.1,
UCQP paragraph).

On |x_i| = 1 the conjugate is the inverse, so every monomial in x and conj(x) is
a Laurent monomial x^delta, delta in Z^q.  The reduced basis keeps the exponents
with ||delta||_1 <= 2 (x_i conj(x_i) = 1 is dropped): 2q^2 + 2q + 1 of them.  The
Hermitian moment matrix v v* has entry x^(beta - gamma); for real data the real
part is used, cos(theta . (beta - gamma)) with x = exp(i theta), so delta and
-delta fall in one class.  A class is represented by the exponent whose first
nonzero entry is positive.

Orders (readings: the paper fixes none):
  basis  by ||delta||_1, then by the list of (index, value) pairs of the nonzero
         entries in increasing index, compared lexicographically;
  class  the same key applied to the representative.
"""
from __future__ import annotations

import itertools

import numpy as np


def basis(q: int):
    """Exponent vectors (tuples of (index, value) pairs) of the reduced basis."""
    out = [()]
    for i in range(q):
        for v in (1, -1, 2, -2):
            out.append(((i, v),))
    for i, j in itertools.combinations(range(q), 2):
        for a in (1, -1):
            for b in (1, -1):
                out.append(((i, a), (j, b)))
    return sorted(out, key=_key)


def _key(d):
    return (sum(abs(v) for _, v in d), d)


def _sub(beta, gamma):
    acc = {}
    for i, v in beta:
        acc[i] = acc.get(i, 0) + v
    for i, v in gamma:
        acc[i] = acc.get(i, 0) - v
    return tuple(sorted((i, v) for i, v in acc.items() if v != 0))


def _canon(d):
    if d and d[0][1] < 0:
        return tuple((i, -v) for i, v in d)
    return d


def index_map(q: int):
    """idx[b, g] = rank of the class {beta - gamma, gamma - beta}; returns (idx, classes)."""
    B = basis(q)
    N = len(B)
    reps = {}
    cls = np.empty((N, N), dtype=object)
    for a, beta in enumerate(B):
        for g, gamma in enumerate(B):
            r = _canon(_sub(beta, gamma))
            cls[a, g] = r
            reps[r] = None
    classes = sorted(reps, key=_key)
    rank = {r: k for k, r in enumerate(classes)}
    idx = np.vectorize(lambda r: rank[r], otypes=[np.int32])(cls)
    return idx, classes


def num_classes(q: int) -> int:
    """m = (|Delta_4| + 1) / 2 = (q^4 + 2q^3 + 5q^2 + 4q + 3) / 3 (the count of real coefficient classes, Section 3.1)."""
    return (q**4 + 2 * q**3 + 5 * q**2 + 4 * q + 3) // 3


def rhs(q: int, Q: np.ndarray, c: np.ndarray, classes):
    """b = coefficients of x*Qx + Re(c'x) on the classes: on |x_i| = 1,
    x*Qx = trace(Q) + sum_{i != j} Q_ij x^(e_j - e_i), Re(c'x) = sum_i c_i (x^{e_i} + x^{-e_i})/2,
    and a class collects the coefficients of delta and -delta."""
    rank = {r: k for k, r in enumerate(classes)}
    b = np.zeros(len(classes))
    tr = 0.0
    for i in range(q):
        tr += float(Q[i, i])
    b[rank[()]] = tr
    for i in range(q):
        b[rank[((i, 1),)]] += float(c[i])
    for i in range(q):
        for j in range(q):
            if i != j:
                b[rank[_canon(_sub(((j, 1),), ((i, 1),)))]] += float(Q[i, j])
    return b


def objective(theta: np.ndarray, Q: np.ndarray, c: np.ndarray) -> float:
    x = np.exp(1j * theta)
    return float(np.real(np.conj(x) @ Q @ x + c @ x))


def class_values(theta: np.ndarray, classes) -> np.ndarray:
    """cos(theta . delta) for each class representative: the moments of the point
    x = exp(i theta) in the real relaxation."""
    return np.array([np.cos(sum(theta[i] * v for i, v in d)) for d in classes])
