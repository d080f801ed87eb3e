"""Pins for the generic pieces: tCG reduces to the Newton step on a convex
quadratic with a large radius; RTR on the sphere minimises a Rayleigh quotient
(the textbook special case, compared with LAPACK's eigh); Lanczos against eigh."""
import math

import numpy as np
import pytest

from oracle.lanczos import lanczos
from oracle.rtr import rtr, tcg


def test_tcg_newton_step_on_spd():
    rng = np.random.default_rng(0)
    n = 30
    M = rng.standard_normal((n, n)); H = M @ M.T + n * np.eye(n)
    g = rng.standard_normal(n)
    eta, Heta, it, stop = tcg(None, g, lambda x, d: H @ d, Delta=1e6, kappa=1e-12, theta=1.0,
                              max_iter=200, floor=1e-14)
    assert stop == "converged"
    assert np.allclose(eta, -np.linalg.solve(H, g), rtol=1e-10, atol=1e-12)
    assert np.allclose(Heta, H @ eta, rtol=1e-10, atol=1e-10)


def test_tcg_stops_at_boundary_and_on_negative_curvature():
    n = 5
    H = np.diag([1.0, 2.0, 3.0, -1.0, 4.0])
    g = np.ones(n)
    eta, _, _, stop = tcg(None, g, lambda x, d: H @ d, Delta=0.5)
    assert stop in ("negcurv", "boundary")
    assert np.linalg.norm(eta) == pytest.approx(0.5, rel=1e-12)


def test_rtr_rayleigh_quotient_on_sphere():
    rng = np.random.default_rng(1)
    n = 40
    A = rng.standard_normal((n, n)); A = A + A.T
    proj = lambda x, u: u - (x @ u) * x
    f = lambda x: float(x @ A @ x)
    grad = lambda x: proj(x, 2 * A @ x)
    hess = lambda x, u: proj(x, 2 * A @ proj(x, u)) - 2 * (x @ A @ x) * proj(x, u)
    retr = lambda x, u: (x + u) / np.linalg.norm(x + u)
    x0 = rng.standard_normal(n); x0 /= np.linalg.norm(x0)
    x, info = rtr(x0, f, grad, hess, retr, Delta_bar=math.pi, tol_grad=1e-10, max_iter=500)
    w = np.linalg.eigvalsh(A)
    assert f(x) == pytest.approx(w[0], rel=1e-10, abs=1e-10)


def test_lanczos_extreme_pairs():
    rng = np.random.default_rng(2)
    n = 120
    A = rng.standard_normal((n, n)); A = A + A.T
    w, V = np.linalg.eigh(A)
    v0 = rng.standard_normal(n)
    lo, vecs, _ = lanczos(lambda v: A @ v, n, 120, v0, "min", 2)
    hi, _, _ = lanczos(lambda v: A @ v, n, 120, v0, "max", 1)
    assert lo == pytest.approx(w[:2], rel=1e-10)
    assert hi[0] == pytest.approx(w[-1], rel=1e-10)
    for j in range(2):
        r = A @ vecs[j] - lo[j] * vecs[j]
        assert np.linalg.norm(r) < 1e-8 * np.abs(w).max()
