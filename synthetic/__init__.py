"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module draws random numbers only; it holds none of the solver's arithmetic
(no index maps, no right-hand sides, no normalisation).  Both the CPU oracle and
the CUDA path receive exactly the arrays produced here.

Instance recipes follow the random instances of the paper's experiments
(Section 6): for the dense BQP of Section 6.1, Q is symmetric with standard
normal free entries and c is standard normal; the sparse-Q variant keeps each
upper-triangular entry with probability `density`; the Hermitian UCQP matrix
has standard normal real and imaginary parts.  Draw order is fixed so that any consumer reproduces the
same arrays from the same seed.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "bqp_instance",
    "ucqp_instance",
    "gaussian_factor",
    "batched_bqp_sizes",
]


def bqp_instance(q: int, seed: int, density: float | None = None):
    """Return (Q, c) for min x'Qx + c'x over x in {-1,1}^q.

    Draw order with ``numpy.random.default_rng(seed)``: the upper triangle of Q
    including the diagonal, row-major, iid N(0,1); then c, iid N(0,1); then, if
    ``density`` is given, one uniform per upper-triangular entry (row-major)
    keeping the entry when it is below ``density``.  Q is mirrored to be
    symmetric.
    """
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(q)
    vals = rng.standard_normal(len(iu[0]))
    c = rng.standard_normal(q)
    if density is not None:
        keep = rng.random(len(iu[0])) < density
        vals = np.where(keep, vals, 0.0)
    Q = np.zeros((q, q))
    Q[iu] = vals
    Q = Q + np.triu(Q, 1).T
    return Q, c


def sparse_bqp_instance(q: int, t: int, seed: int):
    """Return (Qs, cs) for the t blocks of a sparse BQP with overlapping variable
    blocks: for each block in order, with one ``default_rng(seed)`` stream, the
    upper triangle of Q_k including the diagonal, row-major, iid N(0,1) (mirrored),
    then c_k, iid N(0,1)."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(q)
    Qs, cs = [], []
    for _ in range(t):
        Q = np.zeros((q, q))
        Q[iu] = rng.standard_normal(len(iu[0]))
        Qs.append(Q + np.triu(Q, 1).T)
        cs.append(rng.standard_normal(q))
    return Qs, cs


def ucqp_instance(n: int, seed: int):
    """Return a Hermitian complex Q (n x n): real and imaginary parts of the
    strict upper triangle iid N(0,1) (real parts drawn first, row-major), a real
    N(0,1) diagonal drawn last."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    re = rng.standard_normal(len(iu[0]))
    im = rng.standard_normal(len(iu[0]))
    d = rng.standard_normal(n)
    Q = np.zeros((n, n), dtype=np.complex128)
    Q[iu] = re + 1j * im
    Q = Q + Q.conj().T
    Q[np.diag_indices(n)] = d
    return Q


def gaussian_factor(n: int, p: int, seed: int) -> np.ndarray:
    """An n x p matrix of iid N(0,1) draws (row-major), used as the unnormalised
    starting factor.  ``default_rng(seed + 7919)`` keeps it independent of the
    instance stream drawn with the same seed."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((n, p))


def batched_bqp_sizes(n_order1: int, n_order2: int, lo1: int, hi1: int, lo2: int, hi2: int,
                      seed: int = 0):
    """Sizes for a batch of independent BQP instances: ``n_order1`` sizes uniform
    on [lo1, hi1] and then ``n_order2`` sizes uniform on [lo2, hi2], both inclusive,
    drawn from ``default_rng(seed)``.  Instance i uses seed 1000 + i."""
    rng = np.random.default_rng(seed)
    s1 = rng.integers(lo1, hi1 + 1, size=n_order1)
    s2 = rng.integers(lo2, hi2 + 1, size=n_order2)
    return s1, s2
