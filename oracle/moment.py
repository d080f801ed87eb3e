"""Moment-relaxation data for binary quadratic programs.

Section 3.1 (Eq. (BQP) and the second-order SOS relaxation): the basis is
v(x) = [1, x_1..x_q, x_1x_2, x_1x_3, ..., x_{q-1}x_q]; modulo the ideal
x_i^2 = 1 a product of two basis monomials x^beta x^gamma reduces to the
square-free monomial of the symmetric difference beta (xor) gamma.  Each
constraint of the dual SOS problem is indexed by one such monomial.  A_alpha
is the 0/1 matrix marking the moment-matrix entries whose product reduces to
alpha, so A A* is diagonal with the multiplicities on its diagonal (remark on
A A* after Algorithm 1).

Canonical monomial order (a reading: the paper fixes none): by degree, then
lexicographically on the sorted variable tuple.

The order-1 relaxation (basis [1, x]) follows the same rules.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np


def basis(q: int, order: int = 2):
    """Basis monomials as tuples of 0-based variable indices, in the order of
    v(x) printed in Section 3.1."""
    out = [()]
    out += [(i,) for i in range(q)]
    if order >= 2:
        out += list(itertools.combinations(range(q), 2))
    return out


def monomials(q: int, order: int = 2):
    """All square-free monomials of degree <= 2*order, in canonical order."""
    out = []
    for d in range(0, 2 * order + 1):
        out += list(itertools.combinations(range(q), d))
    return out


def num_monomials(q: int, order: int = 2) -> int:
    """m = sum_{d <= 2 order} C(q, d)."""
    return sum(comb(q, d) for d in range(0, 2 * order + 1))


def index_map_enumerated(q: int, order: int = 2):
    """idx[beta, gamma] = rank of the monomial beta xor gamma, built by a
    dictionary over explicitly enumerated monomials (small q only)."""
    B = basis(q, order)
    rank = {mono: r for r, mono in enumerate(monomials(q, order))}
    N = len(B)
    idx = np.empty((N, N), dtype=np.int32)
    for a, beta in enumerate(B):
        for g, gamma in enumerate(B):
            prod = tuple(sorted(set(beta) ^ set(gamma)))
            idx[a, g] = rank[prod]
    return idx


def _comb_rank(sets: np.ndarray, q: int) -> np.ndarray:
    """Lexicographic rank of each sorted d-subset (rows of ``sets``) among all
    d-subsets of {0..q-1}: the number of d-subsets that precede it.  A subset
    (c_1 < ... < c_d) is preceded by every subset sharing its first i-1
    elements and having a smaller i-th element j (c_{i-1} < j < c_i); there are
    C(q-1-j, d-i) of those for each such j."""
    n, d = sets.shape
    r = np.zeros(n, dtype=np.int64)
    prev = np.full(n, -1, dtype=np.int64)
    table = np.array([[comb(a, b) for b in range(d + 1)] for a in range(q + 1)], dtype=np.int64)
    for i in range(d):
        ci = sets[:, i].astype(np.int64)
        for j in range(q):
            mask = (j > prev) & (j < ci)
            if mask.any():
                r[mask] += table[q - 1 - j, d - i - 1]
        prev = ci
    return r


def index_map(q: int, order: int = 2) -> np.ndarray:
    """Vectorised idx map, identical to ``index_map_enumerated``.  Each basis
    monomial is a bit set; the product monomial is the xor of two bit sets; its
    rank is the degree offset plus the lexicographic rank of its sorted index
    tuple."""
    B = basis(q, order)
    N = len(B)
    # basis monomials padded to two slots with -1 for missing variables
    el = np.full((N, 2), -1, dtype=np.int64)
    for a, beta in enumerate(B):
        for s, v in enumerate(beta):
            el[a, s] = v
    # symmetric difference via a q-wide indicator (q <= 200 in practice)
    ind = np.zeros((N, q), dtype=np.int8)
    for s in range(2):
        ok = el[:, s] >= 0
        ind[np.nonzero(ok)[0], el[ok, s]] = 1
    offsets = np.cumsum([0] + [comb(q, d) for d in range(0, 2 * order + 1)])
    idx = np.empty((N, N), dtype=np.int64)
    for a in range(N):
        x = ind[a][None, :] ^ ind  # (N, q)
        deg = x.sum(axis=1)
        out = np.empty(N, dtype=np.int64)
        for d in np.unique(deg):
            rows = np.nonzero(deg == d)[0]
            if d == 0:
                out[rows] = 0
                continue
            sets = np.nonzero(x[rows])[1].reshape(len(rows), d)
            out[rows] = offsets[d] + _comb_rank(sets, q)
        idx[a] = out
    return idx.astype(np.int32)


def multiplicities(idx: np.ndarray, m: int) -> np.ndarray:
    """mult[alpha] = number of entries with idx == alpha = diag(A A*)."""
    return np.bincount(idx.ravel(), minlength=m).astype(np.float64)


def rhs(q: int, Q: np.ndarray, c: np.ndarray, order: int = 2) -> np.ndarray:
    """Right-hand side b of the SOS constraints: the coefficients of
    f(x) = x'Qx + c'x reduced modulo x_i^2 = 1 (Section 3.1).  So
    b[1] = trace(Q), b[x_i] = c_i, b[x_i x_j] = 2 Q_ij (i < j), 0 above degree 2.
    The constant term enters through monomial 1, since the dual (PSDP) places
    sum(z) against it."""
    m = num_monomials(q, order)
    b = np.zeros(m)
    tr = 0.0
    for i in range(q):  # left to right, so that the rounding order is fixed
        tr += float(Q[i, i])
    b[0] = tr
    b[1:1 + q] = c
    k = 1 + q
    for i in range(q):
        for j in range(i + 1, q):
            b[k] = 2.0 * Q[i, j]
            k += 1
    return b


def bqp_objective(x: np.ndarray, Q: np.ndarray, c: np.ndarray) -> float:
    return float(x @ Q @ x + c @ x)
