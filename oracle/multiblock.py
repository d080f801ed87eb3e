"""Sparse BQPs with overlapping variable blocks and their multi-block second-order
relaxation (Section 6, sparse BQPs: Eq. (BQP-sparse), (DSDP-sparse)).

Block k (k = 1..t) holds the q variables x_{(q-2)(k-1)+1} .. x_{(q-2)k+2}; the
problem is min sum_k x_k' Q_k x_k + c_k' x_k over x in {-1,1}^{(q-2)t+2}.  The
relaxation has one moment block per k, of order n_b = 1 + q + q(q-1)/2, with the
basis [1, x_k, products of two block variables]; a constraint class is a
square-free monomial of degree <= 4 in one block's variables, and a monomial
shared by two blocks (through their two common variables) has entries in both.

Exact single-matrix embedding (a reading used to solve the relaxation with the
dense path): stack the blocks into one matrix of order t n_b and give every
entry outside the diagonal blocks a class of its own (the pair {(r, c), (c, r)})
with b = 0.  The embedded problem has the same optimal value: a block-diagonal
S >= 0 extended by zeros is feasible for it, and the diagonal blocks of any
feasible S of the embedded problem are feasible for the block problem with the
same objective (only in-block classes carry b).

Orders (readings: the paper fixes none): classes of monomials first, by degree
and then lexicographically on the sorted global variable tuple (the dense BQP
order; with t = 1 the maps coincide); then the off-block pairs (r < c) in
row-major order.

Test infrastructure: only tests/ use this module.
"""
from __future__ import annotations

import itertools

import numpy as np


def num_variables(q: int, t: int) -> int:
    return (q - 2) * t + 2


def block_variables(q: int, t: int):
    """0-based global indices of the q variables of each block."""
    return [list(range((q - 2) * k, (q - 2) * k + q)) for k in range(t)]


def block_basis(vars_k):
    """[1, x_i, x_i x_j (i < j)] over the block's variables, in the order of v(x)."""
    return [()] + [(i,) for i in vars_k] + list(itertools.combinations(vars_k, 2))


def monomials(q: int, t: int):
    """The monomial classes: every subset of at most 4 variables of some block, in
    canonical order."""
    seen = set()
    for vars_k in block_variables(q, t):
        for d in range(5):
            seen.update(itertools.combinations(vars_k, d))
    return sorted(seen, key=lambda mono: (len(mono), mono))


def index_map(q: int, t: int):
    """Embedded class map (t n_b x t n_b int32) and the number of monomial classes."""
    blocks = block_variables(q, t)
    nb = 1 + q + q * (q - 1) // 2
    mons = monomials(q, t)
    rank = {mono: r for r, mono in enumerate(mons)}
    Nt = t * nb
    idx = np.full((Nt, Nt), -1, dtype=np.int64)
    for k, vars_k in enumerate(blocks):
        B = block_basis(vars_k)
        o = k * nb
        for a, beta in enumerate(B):
            for g, gamma in enumerate(B):
                idx[o + a, o + g] = rank[tuple(sorted(set(beta) ^ set(gamma)))]
    nxt = len(mons)
    for r in range(Nt):
        for c in range(r + 1, Nt):
            if idx[r, c] < 0:
                idx[r, c] = idx[c, r] = nxt
                nxt += 1
    assert (idx >= 0).all()
    return idx.astype(np.int32), len(mons)


def num_classes(q: int, t: int) -> int:
    nb = 1 + q + q * (q - 1) // 2
    off = (t * nb) * (t * nb - nb) // 2  # unordered off-block pairs
    return len(monomials(q, t)) + off


def rhs(q: int, t: int, Qs, cs) -> np.ndarray:
    """b: the coefficients of sum_k x_k' Q_k x_k + c_k' x_k modulo x_i^2 = 1 on the
    monomial classes (constant: the traces, summed block by block left to right;
    x_i: c_k; x_i x_j: Q_k[i, j] + Q_k[j, i]), zero on the off-block classes."""
    mons = monomials(q, t)
    rank = {mono: r for r, mono in enumerate(mons)}
    b = np.zeros(num_classes(q, t))
    tr = 0.0
    for k, vars_k in enumerate(block_variables(q, t)):
        Q, c = Qs[k], cs[k]
        for i in range(q):
            tr += float(Q[i, i])
        for i in range(q):
            b[rank[(vars_k[i],)]] += float(c[i])
        for i in range(q):
            for j in range(i + 1, q):
                b[rank[(vars_k[i], vars_k[j])]] += float(Q[i, j]) + float(Q[j, i])
    b[rank[()]] = tr
    return b


def objective(x: np.ndarray, q: int, t: int, Qs, cs) -> float:
    f = 0.0
    for k, vars_k in enumerate(block_variables(q, t)):
        xk = x[vars_k]
        f += float(xk @ Qs[k] @ xk + cs[k] @ xk)
    return f


def brute_min(q: int, t: int, Qs, cs):
    """Minimum of the sparse BQP over all 2^((q-2)t+2) sign vectors (small sizes)."""
    n = num_variables(q, t)
    best, arg = np.inf, None
    for bits in range(1 << n):
        x = np.array([1.0 if (bits >> i) & 1 else -1.0 for i in range(n)])
        f = objective(x, q, t, Qs, cs)
        if f < best:
            best, arg = f, x
    return best, arg
