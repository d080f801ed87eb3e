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


def _problem(q, seed):
    Q, c = bqp_instance(q, seed)
    idx = moment.index_map(q)
    b = moment.rhs(q, Q, c)
    return manidsdp.make_problem(idx, moment.multiplicities(idx, len(b)), b), b


@pytest.mark.parametrize("q,seed", [(6, 0), (8, 1), (10, 2)])
def test_sigma_sequence_follows_rule_5_1_and_the_stall_safeguard(q, seed):
    """The penalty sequence of a solve obeys Eq. (5.1) with kappa_1 = 0.1, kappa_2 = 10,
    gamma = 2 and, when neither branch fires, the stall safeguard: sigma doubles after
    a subproblem solved to eps_k = clamp(||R_prev|| / (1 + ||b||), 1e-11, 1e-2) whose
    scaled residual exceeds half the previous one.  Reconstructed from the history
    (eta_p = ||R|| with C = 0, the RTR's final gradient norm), for the safeguard on
    and off; both settings reach the same value."""
    prob, b = _problem(q, seed)
    Y0 = gaussian_factor(prob["N"], 2, seed)
    nb = 1.0 + float(np.linalg.norm(b))
    values = []
    for stall in (0.0, 0.5):
        hist = []
        res = manidsdp.solve(prob, Y0, dict(sigma_stall=stall), history=hist)
        assert max(res["eta"]) <= 1e-8
        values.append(res["value"])
        steps = [h for h in hist if not h.get("rounded")]
        prev = None
        for h, nxt in zip(steps, steps[1:]):
            lhs, g, s = h["eta_p"] / nb, h["gnorm"], h["sigma"]
            tol_k = 1e-2 if prev is None else max(1e-11, min(1e-2, prev))
            if lhs < 0.1 * g:
                want = max(s / 2.0, 1e-3)
            elif lhs > 10.0 * g:
                want = min(2.0 * s, 1e6)
            elif stall > 0 and prev is not None and g <= tol_k and lhs > stall * prev:
                want = min(2.0 * s, 1e6)
            else:
                want = s
            assert nxt["sigma"] == want, (h["k"], s, nxt["sigma"], want)
            prev = lhs
    assert abs(values[0] - values[1]) <= 1e-9 * abs(values[0])
