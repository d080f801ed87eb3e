"""End-to-end pins for Algorithm 1 on the dense BQP relaxation: the KKT
residuals of Section 6 reach 1e-8; the relaxation value never exceeds the
brute-force BQP minimum (weak duality); when the solution has rank one the
rounded point x = sign(S[0, 1:q+1]) attains V (tightness, Section 6.1 reports
rank(S) = 1 on dense BQPs); unit diagonal; X S = 0 and X PSD to tolerance."""
import numpy as np
import pytest

from oracle import brute, manidsdp, moment
from synthetic import bqp_instance, gaussian_factor


def run(q, seed, order=2, p0=2, **params):
    Q, c = bqp_instance(q, seed)
    idx = moment.index_map(q, order); m = moment.num_monomials(q, order)
    mult = moment.multiplicities(idx, m)
    b = moment.rhs(q, Q, c, order)
    prob = manidsdp.make_problem(idx, mult, b)
    Y0 = gaussian_factor(idx.shape[0], p0, seed)
    res = manidsdp.solve(prob, Y0, params=params)
    return Q, c, prob, res


def check_certificates(res, tol=1e-8):
    assert max(res["eta"]) <= tol
    S = res["Y"] @ res["Y"].T
    assert np.allclose(np.diag(S), 1.0, atol=1e-13)
    X = res["X"]
    assert np.linalg.eigvalsh(X)[0] >= -tol * (1 + np.abs(np.linalg.eigvalsh(X)).max())
    assert np.linalg.norm(X @ S) <= 1e-5 * (1 + np.linalg.norm(X))


@pytest.mark.parametrize("q,seed", [(4, 0), (6, 1), (8, 2), (10, 0), (12, 3)])
def test_order2_bounds_brute_force(q, seed):
    Q, c, prob, res = run(q, seed)
    check_certificates(res)
    fmin, _ = brute.bqp_min(Q, c)
    V = res["value"]
    assert V <= fmin + 1e-8 * (1 + abs(fmin))
    S = res["Y"] @ res["Y"].T
    sv = np.linalg.svd(S, compute_uv=False)
    if sv[1] < 1e-6 * sv[0]:
        # rank one: tight relaxation, rounding recovers the optimum
        x = np.sign(S[0, 1:q + 1])
        assert moment.bqp_objective(x, Q, c) == pytest.approx(V, rel=1e-8, abs=1e-8)
        assert fmin == pytest.approx(V, rel=1e-8, abs=1e-8)


@pytest.mark.parametrize("q,seed", [(16, 0), (40, 3)])
def test_order1_relaxation_bounds(q, seed):
    """Order-1 (Shor) relaxation: R vanishes on the manifold, so the ALM is plain
    rank-adaptive RTR; the value still bounds the BQP minimum from below."""
    Q, c, prob, res = run(q, seed, order=1)
    check_certificates(res)
    if q <= 16:
        fmin, _ = brute.bqp_min(Q, c)
        assert res["value"] <= fmin + 1e-8 * (1 + abs(fmin))


@pytest.mark.slow
def test_q20_dense_bqp_brute_force_2_pow_20():
    """The 211 x 211 workload (q = 20, seed 0): solve, then brute force all 2^20
    sign vectors."""
    Q, c, prob, res = run(20, 0)
    check_certificates(res)
    fmin, xmin = brute.bqp_min(Q, c)
    assert res["value"] <= fmin + 1e-8 * (1 + abs(fmin))
    assert res["value"] == pytest.approx(fmin, rel=1e-9)
