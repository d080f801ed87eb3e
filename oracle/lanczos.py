"""Lanczos with full reorthogonalisation for the extreme eigenpairs of the
certificate X (Algorithm 1, step 9; the remark after Algorithm 1 that a partial
eigendecomposition may replace the full one; lambda_max enters eta_d of
Section 6).

Textbook Lanczos: beta_{j} v_{j+1} = X v_j - alpha_j v_j - beta_{j-1} v_{j-1},
each new vector re-orthogonalised (twice) against all previous ones in FP64;
Ritz pairs from the tridiagonal matrix T_k.  ``matvec`` is any symmetric
operator; ``v0`` the start vector.
"""
from __future__ import annotations

import numpy as np


def lanczos(matvec, n: int, k: int, v0: np.ndarray, which: str = "min", n_pairs: int = 1):
    k = min(k, n)
    V = np.zeros((k + 1, n))
    alpha = np.zeros(k)
    beta = np.zeros(k)
    V[0] = v0 / np.linalg.norm(v0)
    steps = k
    for j in range(k):
        w = matvec(V[j])
        alpha[j] = V[j] @ w
        for _ in range(2):
            w = w - V[: j + 1].T @ (V[: j + 1] @ w)
        beta[j] = np.linalg.norm(w)
        if beta[j] <= 1e-14 * max(1.0, abs(alpha[j])):
            steps = j + 1
            break
        V[j + 1] = w / beta[j]
    T = np.diag(alpha[:steps]) + np.diag(beta[: steps - 1], 1) + np.diag(beta[: steps - 1], -1)
    theta, s = np.linalg.eigh(T)
    if which == "max":
        theta, s = theta[::-1], s[:, ::-1]
    theta = theta[:n_pairs]
    vecs = (V[:steps].T @ s[:, :n_pairs]).T
    return theta, vecs, steps
