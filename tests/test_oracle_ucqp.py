"""Pins for the real second-order UCQP relaxation (Section 3.1, UCQP paragraph):
the basis size 2q^2 + 2q + 1 and class count (q^4 + 2q^3 + 5q^2 + 4q + 3)/3 printed
there; the defining property of the index map (Re(v v*) at a point of the unit
torus has entry cos(theta . (beta - gamma)), equal on each class); b reproducing
the objective on the torus; a solve whose value bounds the objective at random
feasible points from below and reaches the KKT tolerance."""
import numpy as np
import pytest

from oracle import manidsdp as om, ucqp
from oracle.moment import multiplicities
from synthetic import gaussian_factor


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 7])
def test_counts(q):
    idx, classes = ucqp.index_map(q)
    assert idx.shape[0] == 2 * q * q + 2 * q + 1
    assert len(classes) == ucqp.num_classes(q)
    assert idx.max() == len(classes) - 1 and np.array_equal(idx, idx.T)


@pytest.mark.parametrize("q", [2, 4, 5])
def test_index_map_reproduces_real_moment_matrix(q):
    rng = np.random.default_rng(q)
    idx, classes = ucqp.index_map(q)
    B = ucqp.basis(q)
    for _ in range(3):
        theta = rng.uniform(-np.pi, np.pi, q)
        x = np.exp(1j * theta)
        v = np.array([np.prod([x[i] ** val for i, val in d]) for d in B])
        S = np.real(np.outer(v, np.conj(v)))
        assert np.allclose(S, ucqp.class_values(theta, classes)[idx], atol=1e-13)


@pytest.mark.parametrize("q", [3, 6])
def test_rhs_reproduces_objective_on_torus(q):
    rng = np.random.default_rng(10 + q)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    idx, classes = ucqp.index_map(q)
    b = ucqp.rhs(q, Q, c, classes)
    for _ in range(5):
        theta = rng.uniform(-np.pi, np.pi, q)
        assert b @ ucqp.class_values(theta, classes) == pytest.approx(
            ucqp.objective(theta, Q, c), rel=1e-12, abs=1e-12)


def test_solve_bounds_objective():
    q = 4
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    idx, classes = ucqp.index_map(q)
    m = len(classes)
    prob = om.make_problem(idx, multiplicities(idx, m), ucqp.rhs(q, Q, c, classes))
    res = om.solve(prob, gaussian_factor(idx.shape[0], 2, 0))
    assert max(res["eta"]) <= 1e-8
    best = min(ucqp.objective(rng.uniform(-np.pi, np.pi, q), Q, c) for _ in range(2000))
    assert res["value"] <= best + 1e-8
