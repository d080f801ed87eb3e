"""Pins of the complex first-order UCQP oracle (oracle/ucqp_complex.py).

- derivatives: central differences of f and of the Riemannian gradient along
  the retraction; Hessian symmetry;
- n = 2 closed form: min <Q, X> over [[1, x], [conj x, 1]] >= 0 is
  Q11 + Q22 - 2 |Q12|;
- a planted rank-one optimum: Q = -v v^H with |v_i| = 1 gives -n^2;
- real symmetric Q: the complex relaxation has the value of the real one (for
  real Q, <Q, X> = <Q, Re X> and Re X is feasible for the real relaxation), so
  it must equal the value of the real-path oracle (order-1 BQP relaxation with
  c = 0), which is pinned independently;
- weak duality against random unit-modulus points, and the KKT certificate.
"""
import math

import numpy as np
import pytest

from oracle import manidsdp as om, moment, ucqp_complex as uc
from synthetic import gaussian_factor, ucqp_instance


def random_point(n, p, seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p))
    return Y / np.linalg.norm(Y, axis=1)[:, None]


def random_tangent(Y, seed):
    rng = np.random.default_rng(seed)
    U = rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape)
    return uc.proj_tangent(Y, U)


def real_inner(a, b):
    return float(np.real(np.vdot(a, b)))


@pytest.mark.parametrize("n,p", [(5, 2), (12, 3)])
def test_gradient_and_hessian_by_central_differences(n, p):
    Q = ucqp_instance(n, 3)
    Y = random_point(n, p, 1)
    U = random_tangent(Y, 2)
    h = 1e-5
    fd = (uc.cost(uc.retract(Y, h * U), Q) - uc.cost(uc.retract(Y, -h * U), Q)) / (2 * h)
    assert abs(fd - real_inner(uc.rgrad(Y, Q), U)) <= 1e-7 * max(1.0, abs(fd))
    gd = (uc.rgrad(uc.retract(Y, h * U), Q) - uc.rgrad(uc.retract(Y, -h * U), Q)) / (2 * h)
    H = uc.rhess(Y, U, Q)
    assert np.abs(uc.proj_tangent(Y, gd) - H).max() <= 1e-6 * max(1.0, np.abs(H).max())


def test_hessian_is_symmetric():
    Q = ucqp_instance(9, 4)
    Y = random_point(9, 3, 5)
    U, V = random_tangent(Y, 6), random_tangent(Y, 7)
    a = real_inner(V, uc.rhess(Y, U, Q))
    b = real_inner(U, uc.rhess(Y, V, Q))
    assert abs(a - b) <= 1e-12 * max(1.0, abs(a))


def test_two_by_two_closed_form():
    Q = np.array([[0.7, 1.2 - 0.5j], [1.2 + 0.5j, -0.3]])
    res = uc.solve(Q, random_point(2, 2, 0))
    assert res["eta_max"] <= 1e-10
    assert abs(res["value"] - (0.7 - 0.3 - 2 * abs(1.2 - 0.5j))) <= 1e-10


def test_planted_rank_one_optimum():
    n = 10
    rng = np.random.default_rng(4)
    v = np.exp(1j * rng.uniform(0, 2 * math.pi, n))
    Q = -np.outer(v, v.conj())
    res = uc.solve(Q, random_point(n, 2, 1))
    assert res["eta_max"] <= 1e-10
    assert abs(res["value"] + n * n) <= 1e-9 * n * n
    # the optimum is rank one: Y Y^H = v v^H
    S = res["Y"] @ res["Y"].conj().T
    assert np.abs(S - np.outer(v, v.conj())).max() <= 1e-6


@pytest.mark.parametrize("n,seed", [(6, 0), (9, 2)])
def test_real_symmetric_q_matches_the_real_relaxation(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    Q = (A + A.T) / 2
    res = uc.solve(Q.astype(complex), random_point(n, 2, seed))
    assert res["eta_max"] <= 1e-10
    idx = moment.index_map(n, 1)
    b = moment.rhs(n, Q, np.zeros(n), 1)
    prob = om.make_problem(idx, moment.multiplicities(idx, len(b)), b)
    ref = om.solve(prob, gaussian_factor(idx.shape[0], 2, seed))
    assert max(ref["eta"]) <= 1e-8
    assert abs(res["value"] - ref["value"]) <= 1e-8 * max(1.0, abs(ref["value"]))


@pytest.mark.parametrize("n,seed", [(8, 1), (16, 2)])
def test_certificate_and_weak_duality(n, seed):
    Q = ucqp_instance(n, seed)
    res = uc.solve(Q, random_point(n, 2, seed))
    assert res["eta_max"] <= 1e-10
    assert res["lambda_min"] >= -1e-10 * (1 + abs(res["lambda_max"]))
    rng = np.random.default_rng(seed + 100)
    for _ in range(200):
        z = np.exp(1j * rng.uniform(0, 2 * math.pi, n))
        assert float(np.real(np.vdot(z, Q @ z))) >= res["value"] - 1e-9
