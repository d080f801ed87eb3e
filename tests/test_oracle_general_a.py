"""Pins of the general-A operators (a non-diagonal A A*, factored once by
Cholesky; next to the remark after Algorithm 1 on factoring A A* once).

- with A the 0/1 class matrix of a BQP relaxation the general operators equal
  the class operators (y(S), P, Q, D);
- P is idempotent and self-adjoint, ||Q(Z)||^2 is the least-squares distance
  from Z to range(A*), A(D) = b;
- recombining the constraints, A' = T A and b' = T b with T invertible, leaves
  the SDP unchanged while A' A'* is no longer diagonal: the solve on (A', b')
  reaches eta_max <= 1e-8 and the class-based solve's value.
"""
import numpy as np
import pytest

from oracle import manidsdp as om, moment, operators as ops
from synthetic import bqp_instance, gaussian_factor


def class_matrix(idx, m):
    N = idx.shape[0]
    A = np.zeros((m, N * N))
    A[idx.ravel(), np.arange(N * N)] = 1.0
    return A


def bqp(q, seed):
    Q, c = bqp_instance(q, seed)
    idx = moment.index_map(q)
    b = moment.rhs(q, Q, c)
    return idx, b, om.make_problem(idx, moment.multiplicities(idx, len(b)), b)


def test_general_operators_reduce_to_the_class_operators():
    idx, b, prob = bqp(4, 1)
    gen = om.make_problem_general(class_matrix(idx, len(b)), b)
    rng = np.random.default_rng(0)
    Z = rng.standard_normal(idx.shape); Z = Z + Z.T
    assert np.allclose(ops.y_prob(Z, gen), ops.y_prob(Z, prob), rtol=1e-13, atol=1e-13)
    assert np.allclose(ops.Q_prob(Z, gen), ops.Q_prob(Z, prob), rtol=1e-13, atol=1e-13)
    assert np.allclose(gen["D"], prob["D"], rtol=1e-13, atol=1e-13)


def recombined(q, seed):
    idx, b, prob = bqp(q, seed)
    m = len(b)
    rng = np.random.default_rng(seed + 50)
    T = np.eye(m) + 0.3 * rng.standard_normal((m, m)) / np.sqrt(m)
    A2 = T @ class_matrix(idx, m)
    return prob, om.make_problem_general(A2, T @ b)


def test_projector_properties_with_a_non_diagonal_gram_matrix():
    prob, gen = recombined(4, 2)
    M = gen["Amat"] @ gen["Amat"].T
    assert np.abs(M - np.diag(np.diag(M))).max() > 0.1  # A A* not diagonal
    rng = np.random.default_rng(3)
    N = gen["N"]
    Z = rng.standard_normal((N, N)); Z = Z + Z.T
    W = rng.standard_normal((N, N)); W = W + W.T
    PZ = Z - ops.Q_prob(Z, gen)
    assert np.allclose(PZ - ops.Q_prob(PZ, gen), PZ, atol=1e-12)          # P P = P
    PW = W - ops.Q_prob(W, gen)
    assert abs(np.sum(PZ * W) - np.sum(Z * PW)) <= 1e-10 * np.abs(Z).sum()  # self-adjoint
    coef, *_ = np.linalg.lstsq(gen["Amat"].T, Z.ravel(), rcond=None)
    dist2 = np.sum((gen["Amat"].T @ coef - Z.ravel()) ** 2)
    assert abs(np.sum(ops.Q_prob(Z, gen) ** 2) - dist2) <= 1e-10 * max(1.0, dist2)
    assert np.allclose(gen["Amat"] @ gen["D"].ravel(), gen["b"], atol=1e-10)


@pytest.mark.parametrize("q,seed", [(4, 2), (6, 0)])
def test_recombined_constraints_solve_to_the_same_value(q, seed):
    prob, gen = recombined(q, seed)
    Y0 = gaussian_factor(prob["N"], 2, seed)
    ref = om.solve(prob, Y0)
    res = om.solve(gen, Y0)
    assert max(ref["eta"]) <= 1e-8 and max(res["eta"]) <= 1e-8
    assert abs(res["value"] - ref["value"]) <= 1e-8 * abs(ref["value"])
