"""Pins of the sparse (multi-block) BQP relaxation (oracle/multiblock.py).

- with one block the class map and b are the dense BQP ones (oracle/moment.py);
- b reproduces the objective: sum over monomial classes of b_alpha x^alpha = f(x)
  on random sign vectors; off-block classes carry b = 0 and multiplicity 2;
  A A* is the diagonal of multiplicities;
- solves of the embedded problem (the dense oracle on the embedded map) reach
  eta_max <= 1e-8, stay below the brute-force minimum over all sign vectors
  (weak duality), and certify the block problem: every diagonal block of the
  certificate is PSD and complementary to its block of S; when the solution is
  rank one the rounded point attains the brute-force minimum.
"""
import math

import numpy as np
import pytest

from oracle import manidsdp as om, moment, multiblock as mb, operators as ops
from synthetic import gaussian_factor, sparse_bqp_instance


@pytest.mark.parametrize("q", [3, 5, 8])
def test_one_block_is_the_dense_relaxation(q):
    idx, nm = mb.index_map(q, 1)
    assert np.array_equal(idx, moment.index_map(q))
    assert nm == moment.num_monomials(q)
    Qs, cs = sparse_bqp_instance(q, 1, 4)
    assert np.array_equal(mb.rhs(q, 1, Qs, cs), moment.rhs(q, Qs[0], cs[0]))


@pytest.mark.parametrize("q,t", [(4, 2), (5, 3), (6, 2)])
def test_rhs_reproduces_the_objective_and_classes_are_orthogonal(q, t):
    idx, nm = mb.index_map(q, t)
    m = mb.num_classes(q, t)
    assert idx.max() + 1 == m
    assert np.array_equal(idx, idx.T)
    Qs, cs = sparse_bqp_instance(q, t, 1)
    b = mb.rhs(q, t, Qs, cs)
    mons = mb.monomials(q, t)
    rng = np.random.default_rng(2)
    for _ in range(20):
        x = rng.choice([-1.0, 1.0], mb.num_variables(q, t))
        val = sum(b[a] * math.prod(x[i] for i in mono) for a, mono in enumerate(mons))
        assert abs(val - mb.objective(x, q, t, Qs, cs)) <= 1e-12 * (1 + abs(val))
    mult = moment.multiplicities(idx, m)
    assert (mult[nm:] == 2).all() and (b[nm:] == 0).all()
    nb = 1 + q + q * (q - 1) // 2
    assert mult[0] == t * nb  # the constant: every diagonal entry of every block
    v = rng.standard_normal(m)
    assert np.allclose(ops.AAstar(v, idx, m), mult * v)


@pytest.mark.parametrize("q,t,seed", [(4, 2, 0), (5, 3, 1), (6, 3, 2)])
def test_embedded_solve_certifies_the_block_relaxation(q, t, seed):
    idx, nm = mb.index_map(q, t)
    m = mb.num_classes(q, t)
    Qs, cs = sparse_bqp_instance(q, t, seed)
    b = mb.rhs(q, t, Qs, cs)
    prob = om.make_problem(idx, moment.multiplicities(idx, m), b)
    res = om.solve(prob, gaussian_factor(idx.shape[0], 2, seed))
    assert max(res["eta"]) <= 1e-8
    fmin, xmin = mb.brute_min(q, t, Qs, cs)
    assert res["value"] <= fmin + 1e-8 * (1 + abs(fmin))
    nb = 1 + q + q * (q - 1) // 2
    X, S = res["X"], res["S"]
    scale = 1 + np.abs(X).max()
    for k in range(t):
        sl = slice(k * nb, (k + 1) * nb)
        assert np.linalg.eigvalsh(X[sl, sl])[0] >= -1e-8 * scale
        assert abs(np.sum(X[sl, sl] * S[sl, sl])) <= 1e-7 * scale * nb
    if res["p"] == 1 or np.linalg.matrix_rank(S, tol=1e-6) == 1:
        # rank one: the block-0 row of the constant monomial carries the point
        xr = np.zeros(mb.num_variables(q, t))
        for k, vars_k in enumerate(mb.block_variables(q, t)):
            xr[vars_k] = np.sign(S[k * nb, k * nb + 1:k * nb + 1 + q])
        assert abs(mb.objective(xr, q, t, Qs, cs) - res["value"]) <= 1e-7 * (1 + abs(fmin))
        assert abs(res["value"] - fmin) <= 1e-7 * (1 + abs(fmin))
