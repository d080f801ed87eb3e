"""Exhaustive minimum of f(x) = x'Qx + c'x over x in {-1,1}^q.

The relaxation value V of Algorithm 1 is a lower bound on this minimum (weak
duality between (PSDP) and (DSDP) for the moment relaxation of Section 3.1);
when the relaxation is tight the two coincide.  Enumerates all 2^q sign vectors
in blocks; fine up to q = 22.
"""
from __future__ import annotations

import numpy as np


def bqp_min(Q: np.ndarray, c: np.ndarray, block_bits: int = 16):
    q = len(c)
    best = np.inf
    best_x = None
    lo_bits = min(q, block_bits)
    hi_bits = q - lo_bits
    codes = np.arange(1 << lo_bits, dtype=np.int64)
    lo = 1.0 - 2.0 * ((codes[:, None] >> np.arange(lo_bits)) & 1)
    for h in range(1 << hi_bits):
        hi = 1.0 - 2.0 * ((h >> np.arange(hi_bits)) & 1)
        X = np.hstack([lo, np.broadcast_to(hi, (lo.shape[0], hi_bits))])
        vals = np.einsum("ij,ij->i", X @ Q, X) + X @ c
        i = int(np.argmin(vals))
        if vals[i] < best:
            best = float(vals[i])
            best_x = X[i].copy()
    return best, best_x
