"""Pins for the factorised subproblem (Section 4): two independent statements of
Psi_k, two of grad (P_Y(2GY) vs 2XY, Prop. 4.2), finite differences along the
retraction for grad and Hess, Hessian symmetry, the closed form of Theorem 4.5,
the delayed-curvature identity and bound of Proposition 5.1, and the ALM
invariants of Lemmas 3.2 and 3.3."""
import math

import numpy as np
import pytest

from oracle import moment, operators as ops, subproblem as sp
from oracle.manidsdp import make_problem


def setup(q=5, p=3, seed=0, with_C=False):
    rng = np.random.default_rng(seed)
    idx = moment.index_map(q); m = moment.num_monomials(q)
    mult = moment.multiplicities(idx, m)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    b = moment.rhs(q, Q, rng.standard_normal(q))
    N = idx.shape[0]
    C = None
    if with_C:
        C = rng.standard_normal((N, N)); C = 0.1 * (C + C.T)
    prob = make_problem(idx, mult, b, C)
    # a multiplier in ker A, as Lemma 3.2 guarantees for every iterate
    W = rng.standard_normal((N, N)); W = W + W.T
    Xt = 0.3 * ops.Q(W, idx, mult)
    Y = rng.standard_normal((N, p)); Y /= np.linalg.norm(Y, axis=1)[:, None]
    return prob, Xt, Y, rng


def tangent(rng, Y):
    return sp.proj_tangent(Y, rng.standard_normal(Y.shape))


@pytest.mark.parametrize("with_C", [False, True])
def test_cost_two_forms(with_C):
    prob, Xt, Y, _ = setup(with_C=with_C)
    for sigma in (0.5, 3.0):
        assert sp.cost(Y, prob, Xt, sigma) == pytest.approx(sp.cost_lagrangian(Y, prob, Xt, sigma), rel=1e-12)


@pytest.mark.parametrize("with_C", [False, True])
def test_grad_two_forms(with_C):
    prob, Xt, Y, _ = setup(with_C=with_C)
    g1 = sp.rgrad(Y, prob, Xt, 2.0)
    g2 = sp.rgrad_certificate(Y, prob, Xt, 2.0)
    assert np.allclose(g1, g2, rtol=0, atol=1e-11 * np.abs(g1).max())
    assert np.abs(sp.rowdot(g1, Y)).max() < 1e-12 * np.abs(g1).max()


@pytest.mark.parametrize("with_C", [False, True])
def test_grad_finite_difference(with_C):
    prob, Xt, Y, rng = setup(with_C=with_C)
    sigma = 1.7
    U = tangent(rng, Y)
    g = sp.rgrad(Y, prob, Xt, sigma)
    f = lambda t: sp.cost(sp.retract(Y, t * U), prob, Xt, sigma)
    errs = []
    for t in (1e-3, 5e-4):
        fd = (f(t) - f(-t)) / (2 * t)
        errs.append(abs(fd - np.sum(g * U)))
    assert errs[1] < 0.3 * errs[0] + 1e-9  # O(t^2) decay
    assert errs[1] < 1e-4 * abs(np.sum(g * U)) + 1e-8


@pytest.mark.parametrize("with_C", [False, True])
def test_hess_finite_difference_of_gradient(with_C):
    """Riemannian submanifold: Hess f(Y)[U] = P_Y(d/dt grad f(c(t))|_0) for any
    curve with c(0) = Y, c'(0) = U; here c(t) = Retr(Y + tU)."""
    prob, Xt, Y, rng = setup(with_C=with_C)
    sigma = 0.8
    U = tangent(rng, Y)
    H = sp.rhess(Y, U, prob, Xt, sigma)
    t = 1e-5
    gp = sp.rgrad(sp.retract(Y, t * U), prob, Xt, sigma)
    gm = sp.rgrad(sp.retract(Y, -t * U), prob, Xt, sigma)
    fd = sp.proj_tangent(Y, (gp - gm) / (2 * t))
    assert np.abs(fd - H).max() < 1e-6 * np.abs(H).max()


def test_hess_symmetric_and_tangent():
    prob, Xt, Y, rng = setup(q=6, p=4)
    U, V = tangent(rng, Y), tangent(rng, Y)
    HU = sp.rhess(Y, U, prob, Xt, 1.3)
    HV = sp.rhess(Y, V, prob, Xt, 1.3)
    assert np.sum(V * HU) == pytest.approx(np.sum(U * HV), rel=1e-11)
    assert np.abs(sp.rowdot(HU, Y)).max() < 1e-12 * np.abs(HU).max()


def test_theorem_4_5_closed_form():
    """At Yhat = [Y, 0] and U = [0, V]: <U, grad> = 0 and <U, Hess U> = 2 tr(V'XV),
    with X the certificate at S = Y Y'."""
    prob, Xt, Y, rng = setup(q=6, p=3)
    sigma = 2.0
    N = Y.shape[0]
    G = sp.egrad_S(Y, prob, Xt, sigma)
    X, _ = sp.certificate(G, Y @ Y.T)
    w, Vx = np.linalg.eigh(X)
    V = Vx[:, :2]
    Yh = np.hstack([Y, np.zeros((N, 2))])
    U = np.hstack([np.zeros((N, 3)), V])
    assert abs(np.sum(U * sp.rgrad(Yh, prob, Xt, sigma))) < 1e-12
    lhs = np.sum(U * sp.rhess(Yh, U, prob, Xt, sigma))
    assert lhs == pytest.approx(2.0 * np.trace(V.T @ X @ V), rel=1e-11)
    assert lhs == pytest.approx(2.0 * (w[0] + w[1]), rel=1e-11)


def test_proposition_5_1_delayed_curvature():
    """After one ALM update with sigma_k, the curvature of Psi_{k+1} (penalty
    sigma_{k+1}) along [0, v] at [Y, 0] equals -2 nu - 2 sigma_{k+1} v'C_S(R)v and
    is at most -2 nu + 2 (1 + sqrt n) sigma_{k+1} ||R||."""
    prob, Xt, Y, rng = setup(q=6, p=3, seed=4)
    idx, mult, D = prob["idx"], prob["mult"], prob["D"]
    N = Y.shape[0]
    sig_k, sig_k1 = 1.5, 3.0
    S = Y @ Y.T
    y = ops.y_of(S, None, idx, mult)
    R = ops.Astar(y, idx) - S
    Xt1 = Xt - sig_k * R
    z = sp.rowdot((Xt1 + D) @ Y, Y)
    X = Xt1 + D - np.diag(z)
    w, Vx = np.linalg.eigh(X)
    assert w[0] < 0
    nu, v = -w[0], Vx[:, 0]
    Yh = np.hstack([Y, np.zeros((N, 1))])
    U = np.zeros((N, 4)); U[:, 3] = v
    curv = np.sum(U * sp.rhess(Yh, U, prob, Xt1, sig_k1))
    CR = R - np.diag(np.diag(R @ S))
    assert curv == pytest.approx(-2 * nu - 2 * sig_k1 * v @ CR @ v, rel=1e-10, abs=1e-12)
    assert curv <= -2 * nu + 2 * (1 + math.sqrt(N)) * sig_k1 * np.linalg.norm(R) + 1e-12
    assert abs(np.sum(U * sp.rgrad(Yh, prob, Xt1, sig_k1))) < 1e-12


def test_alm_invariants_lemmas_3_2_3_3():
    """A(Xt^k) = 0, A(X^k + Diag z^k) = b and <X^k, S^k> = 0 after an update."""
    prob, Xt, Y, rng = setup(q=5, p=2, seed=2)
    idx, mult, D, b = prob["idx"], prob["mult"], prob["D"], prob["b"]
    m = len(mult)
    for sigma in (0.7, 4.0):
        S = Y @ Y.T
        y = ops.y_of(S, None, idx, mult)
        Xt = Xt - sigma * (ops.Astar(y, idx) - S)
        z = sp.rowdot((Xt + D) @ Y, Y)
        X = Xt + D - np.diag(z)
        assert np.abs(ops.A(Xt, idx, m)).max() < 1e-11
        assert np.allclose(ops.A(X + np.diag(z), idx, m), b, atol=1e-11)
        assert abs(np.sum(X * S)) < 1e-10
        Y = sp.retract(Y, 0.1 * tangent(rng, Y))


def test_retraction_and_projector():
    _, _, Y, rng = setup(q=4, p=3)
    U = rng.standard_normal(Y.shape)
    PU = sp.proj_tangent(Y, U)
    assert np.abs(sp.rowdot(PU, Y)).max() < 1e-14
    assert np.allclose(sp.proj_tangent(Y, PU), PU, atol=1e-15)
    Z = sp.retract(Y, PU)
    assert np.allclose(np.linalg.norm(Z, axis=1), 1.0, atol=1e-15)
