"""Pins for the BQP moment data (Section 3.1): closed-form counts, the defining
property of the index map (x^beta x^gamma = x^(beta xor gamma) on {-1,1}^q),
the defining property of b (f(x) = sum_alpha b_alpha x^alpha on {-1,1}^q), and
A A* = Diag(mult) (remark on A A* after Algorithm 1)."""
from math import comb

import numpy as np
import pytest

from oracle import moment, operators as ops


def m_sos_closed_form(q):
    # Section 3.1, BQP constraint count: m_sos^B = (q^4 - 2q^3 + 11q^2 + 14q + 24) / 24
    return (q**4 - 2 * q**3 + 11 * q**2 + 14 * q + 24) // 24


@pytest.mark.parametrize("q", list(range(1, 31)) + [80, 120])
def test_monomial_count_matches_paper(q):
    assert moment.num_monomials(q, 2) == m_sos_closed_form(q)
    assert (q**4 - 2 * q**3 + 11 * q**2 + 14 * q + 24) % 24 == 0


def test_named_sizes():
    assert moment.num_monomials(20) == 6196
    assert moment.num_monomials(80) == 1666981
    assert moment.num_monomials(120) == 8502671
    assert len(moment.basis(20)) == 211
    assert len(moment.basis(80)) == 3241
    assert len(moment.basis(120)) == 7261


@pytest.mark.parametrize("q,order", [(3, 2), (4, 2), (5, 2), (7, 2), (3, 1), (9, 1)])
def test_vectorised_index_map_equals_enumeration(q, order):
    assert np.array_equal(moment.index_map(q, order), moment.index_map_enumerated(q, order))


@pytest.mark.parametrize("q,order", [(4, 2), (6, 2), (9, 2), (12, 1)])
def test_index_map_reproduces_products_on_hypercube(q, order):
    """For x in {-1,1}^q: v(x)v(x)' has entry x^beta x^gamma, which must equal
    the value at x of the monomial the map assigns to (beta, gamma)."""
    rng = np.random.default_rng(5)
    idx = moment.index_map(q, order)
    B = moment.basis(q, order)
    monos = moment.monomials(q, order)
    for _ in range(5):
        x = rng.choice([-1.0, 1.0], size=q)
        v = np.array([np.prod(x[list(s)]) for s in B])
        mv = np.array([np.prod(x[list(s)]) for s in monos])
        assert np.array_equal(np.outer(v, v), mv[idx])


@pytest.mark.parametrize("q", [3, 5, 6, 8, 11])
def test_multiplicities_by_degree(q):
    """mult = (N, 2q, 2q, 6, 6) for degrees 0..4 (order 2); all >= 1 so that
    A A* is invertible (Assumption 2); they sum to N^2."""
    idx = moment.index_map(q)
    m = moment.num_monomials(q)
    mult = moment.multiplicities(idx, m)
    N = 1 + q + comb(q, 2)
    deg = np.array([len(s) for s in moment.monomials(q)])
    expect = {0: N, 1: 2 * q, 2: 2 * q, 3: 6, 4: 6}
    for d, e in expect.items():
        if (deg == d).any():
            assert np.all(mult[deg == d] == e)
    assert mult.sum() == N * N and mult.min() >= 1


def test_order1_multiplicities():
    q = 10
    idx = moment.index_map(q, 1)
    mult = moment.multiplicities(idx, moment.num_monomials(q, 1))
    assert mult[0] == q + 1 and np.all(mult[1:] == 2)


@pytest.mark.parametrize("q,order", [(5, 2), (8, 2), (7, 1)])
def test_rhs_reproduces_objective_on_hypercube(q, order):
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    b = moment.rhs(q, Q, c, order)
    monos = moment.monomials(q, order)
    for _ in range(10):
        x = rng.choice([-1.0, 1.0], size=q)
        mv = np.array([np.prod(x[list(s)]) for s in monos])
        assert b @ mv == pytest.approx(moment.bqp_objective(x, Q, c), rel=1e-13, abs=1e-12)


def test_AAstar_is_diagonal_of_multiplicities():
    q = 6
    idx = moment.index_map(q); m = moment.num_monomials(q)
    mult = moment.multiplicities(idx, m)
    v = np.random.default_rng(0).standard_normal(m)
    assert np.allclose(ops.AAstar(v, idx, m), mult * v, rtol=0, atol=1e-12)
