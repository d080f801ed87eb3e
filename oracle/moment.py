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


def _lex_rank(sets: np.ndarray, q: int, d: int, table: np.ndarray) -> np.ndarray:
    """Lexicographic rank of each sorted d-subset (the first d columns of
    ``sets``) among all d-subsets of {0..q-1}: the number of d-subsets that
    precede it.  A subset (c_1 < ... < c_d) is preceded by every subset that
    shares its first i-1 elements and has a smaller i-th element j
    (c_{i-1} < j < c_i), C(q-1-j, d-i) of them for each such j; summed over j
    (hockey-stick identity) that is C(q-1-c_{i-1}, d-i+1) - C(q-c_i, d-i+1),
    with c_0 = -1.  ``table[n, k]`` = C(n, k)."""
    r = np.zeros(sets.shape[0], dtype=np.int64)
    prev = np.full(sets.shape[0], -1, dtype=np.int64)
    for i in range(1, d + 1):
        ci = sets[:, i - 1]
        r += table[q - 1 - prev, d - i + 1] - table[q - ci, d - i + 1]
        prev = ci
    return r


def index_map(q: int, order: int = 2, block: int = 256) -> np.ndarray:
    """Vectorised idx map, identical to ``index_map_enumerated``.  For a block
    of rows at a time: the variables of the two basis monomials of each entry
    (padded with q), sorted; a variable present twice cancels (x_i^2 = 1), which
    leaves the sorted symmetric difference; its rank is the degree offset plus
    its lexicographic rank among the monomials of that degree."""
    B = basis(q, order)
    N = len(B)
    el = np.full((N, order), q, dtype=np.int64)
    for a, beta in enumerate(B):
        for s_, v in enumerate(beta):
            el[a, s_] = v
    offsets = np.cumsum([0] + [comb(q, d) for d in range(0, 2 * order + 1)])
    table = np.array([[comb(n, k) for k in range(2 * order + 2)] for n in range(q + 2)],
                     dtype=np.int64)
    idx = np.empty((N, N), dtype=np.int32)
    for r0 in range(0, N, block):
        rows = el[r0:r0 + block]
        nb = rows.shape[0]
        v = np.concatenate([np.broadcast_to(rows[:, None, :], (nb, N, order)),
                            np.broadcast_to(el[None, :, :], (nb, N, order))], axis=2)
        v = np.sort(v, axis=2)
        same = (v[..., 1:] == v[..., :-1]) & (v[..., 1:] < q)
        gone = np.zeros(v.shape, dtype=bool)
        gone[..., 1:] |= same
        gone[..., :-1] |= same
        v = np.sort(np.where(gone, q, v), axis=2).reshape(nb * N, 2 * order)
        deg = (v < q).sum(axis=1)
        out = np.zeros(nb * N, dtype=np.int64)
        for d in range(1, 2 * order + 1):
            sel = np.nonzero(deg == d)[0]
            if len(sel):
                out[sel] = offsets[d] + _lex_rank(v[sel], q, d, table)
        idx[r0:r0 + nb] = out.reshape(nb, N)
    return idx


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
