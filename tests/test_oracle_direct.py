"""Pins of the direct-formulation subproblem (oracle/direct.py) against what
Section 3 fixes about it, and of the direct solve against the projected one.

- Eq. (penalty-decomposition): ||P(Z^k) - Z||^2 = ||P(Z - Z^k)||^2 + ||Q(Z)||^2;
- the direct subproblem is the reduced one plus sigma/2 ||P(Z - Z^k)||^2
  (Eq. (additional-proximal-term)), and it is the direct augmented Lagrangian at
  the stale y^k up to a constant (Eq. (direct-ALM-subproblem));
- Eq. (hessian-comparison): in S the direct gradient has derivative sigma I, the
  projected one sigma Q;
- gradient and Hessian by central differences along the retraction;
- the direct scheme solves the same SDP: its value equals the projected one's,
  in at least as many outer iterations.  It runs with a fixed penalty (the
  standard two-block ADMM): under the sigma rule (5.1) sigma grows while R is
  large, which strengthens the damping term of Eq. (additional-proximal-term),
  and the scheme stalls with a negative certificate eigenvalue.
"""
import numpy as np
import pytest

from oracle import direct, manidsdp as om, moment, operators as ops, subproblem as sp
from synthetic import bqp_instance, gaussian_factor
from tests.test_oracle_subproblem import setup, tangent


def unit_rows(rng, N, p):
    Y = rng.standard_normal((N, p))
    return Y / np.linalg.norm(Y, axis=1)[:, None]


def test_penalty_decomposition_and_extra_proximal_term():
    prob, Xt, Y, rng = setup(seed=11)
    sigma = 1.3
    idx, mult = prob["idx"], prob["mult"]
    Yk = unit_rows(rng, *Y.shape)
    Z, Zk = Y @ Y.T, Yk @ Yk.T
    yk = ops.y_of(Zk, None, idx, mult)
    lhs = np.sum((ops.P(Zk, idx, mult) - Z) ** 2)
    PZ = ops.P(Z - Zk, idx, mult)
    QZ = ops.Q(Z, idx, mult)
    assert abs(lhs - (np.sum(PZ ** 2) + np.sum(QZ ** 2))) <= 1e-12 * lhs
    extra = direct.cost(Y, prob, Xt, sigma, yk) - sp.cost(Y, prob, Xt, sigma)
    assert abs(extra - 0.5 * sigma * np.sum(PZ ** 2)) <= 1e-10 * max(1.0, abs(extra))


def test_direct_subproblem_is_the_direct_lagrangian_at_the_stale_y():
    prob, Xt, Y, rng = setup(seed=12)
    sigma = 0.8
    yk = ops.y_of(unit_rows(rng, *Y.shape) @ unit_rows(rng, *Y.shape).T, None, prob["idx"],
                  prob["mult"])
    Xbar = prob["D"] + Xt
    offsets = []
    for s in range(3):
        Ys = unit_rows(np.random.default_rng(40 + s), *Y.shape)
        offsets.append(direct.lagrangian(Ys, prob, Xbar, sigma, yk)
                       - direct.cost(Ys, prob, Xt, sigma, yk))
    assert max(offsets) - min(offsets) <= 1e-10 * max(1.0, abs(offsets[0]))


def test_hessian_comparison_in_s():
    prob, Xt, Y, rng = setup(seed=13)
    sigma, h = 2.0, 1e-3
    idx, mult = prob["idx"], prob["mult"]
    yk = ops.y_of(Y @ Y.T, None, idx, mult)
    E = rng.standard_normal((Y.shape[0], Y.shape[0]))
    E = E + E.T
    S = Y @ Y.T

    def g_direct(Sv):  # W + D - sigma (A*(y^k) - S)
        return Xt + prob["D"] - sigma * (ops.Astar(yk, idx) - Sv)

    def g_proj(Sv):  # W + D - sigma (A*(y(S)) - S)
        return Xt + prob["D"] - sigma * (ops.Astar(ops.y_of(Sv, None, idx, mult), idx) - Sv)

    dd = (g_direct(S + h * E) - g_direct(S)) / h
    dp = (g_proj(S + h * E) - g_proj(S)) / h
    assert np.abs(dd - sigma * E).max() <= 1e-9 * np.abs(E).max() * sigma
    assert np.abs(dp - sigma * ops.Q(E, idx, mult)).max() <= 1e-9 * np.abs(E).max() * sigma


def test_direct_gradient_and_hessian_by_central_differences():
    prob, Xt, Y, rng = setup(seed=14)
    sigma = 0.9
    yk = ops.y_of(unit_rows(rng, *Y.shape) @ unit_rows(rng, *Y.shape).T, None, prob["idx"],
                  prob["mult"])
    U = tangent(rng, Y)
    t = 1e-5
    fd = (direct.cost(sp.retract(Y, t * U), prob, Xt, sigma, yk)
          - direct.cost(sp.retract(Y, -t * U), prob, Xt, sigma, yk)) / (2 * t)
    g = direct.rgrad(Y, prob, Xt, sigma, yk)
    assert abs(fd - np.sum(g * U)) <= 1e-7 * max(1.0, abs(fd))
    gp = direct.rgrad(sp.retract(Y, t * U), prob, Xt, sigma, yk)
    gm = direct.rgrad(sp.retract(Y, -t * U), prob, Xt, sigma, yk)
    H = direct.rhess(Y, U, prob, Xt, sigma, yk)
    fdh = sp.proj_tangent(Y, (gp - gm) / (2 * t))
    assert np.abs(fdh - H).max() <= 1e-6 * np.abs(H).max()


@pytest.mark.parametrize("q,seed", [(5, 0), (8, 2)])
def test_direct_scheme_reaches_the_projected_value(q, seed):
    Q, c = bqp_instance(q, seed)
    idx = moment.index_map(q)
    b = moment.rhs(q, Q, c)
    prob = om.make_problem(idx, moment.multiplicities(idx, len(b)), b)
    Y0 = gaussian_factor(idx.shape[0], 2, seed)
    ref = om.solve(prob, Y0)
    fixed = dict(sigma0=0.25, kappa1=-1.0, kappa2=1e300, sigma_stall=0.0, max_outer=1000)
    res = om.solve(prob, Y0, direct=True, params=fixed)
    assert max(ref["eta"]) <= 1e-8 and max(res["eta"]) <= 1e-8
    assert abs(res["value"] - ref["value"]) <= 1e-8 * abs(ref["value"])
    assert res["outer"] >= ref["outer"]
