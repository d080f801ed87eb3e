"""The pins must fail on a plausible mistake.  Each case plants one mistake in a
copy of an oracle function (on the CPU) and checks that the corresponding pin
detects it: a dropped penalty term in the Hessian, a wrong sign on the
curvature term, a transposed operand in the gradient, a missing factor 2 in b."""
import numpy as np

from oracle import moment, operators as ops, subproblem as sp
from tests.test_oracle_subproblem import setup, tangent


def fd_hess_error(hess_fn):
    prob, Xt, Y, rng = setup(seed=7)
    sigma = 0.9
    U = tangent(rng, Y)
    H = hess_fn(Y, U, prob, Xt, sigma)
    t = 1e-5
    gp = sp.rgrad(sp.retract(Y, t * U), prob, Xt, sigma)
    gm = sp.rgrad(sp.retract(Y, -t * U), prob, Xt, sigma)
    fd = sp.proj_tangent(Y, (gp - gm) / (2 * t))
    return np.abs(fd - H).max() / np.abs(H).max()


def test_correct_hessian_passes():
    assert fd_hess_error(sp.rhess) < 1e-6


def test_dropped_penalty_term_caught():
    def bad(Y, U, prob, Xt, sigma):
        G = sp.egrad_S(Y, prob, Xt, sigma)
        U = sp.proj_tangent(Y, U)
        H = 2.0 * G @ U
        z = sp.rowdot(G @ Y, Y)
        return H - sp.rowdot(H, Y)[:, None] * Y - 2.0 * z[:, None] * U
    assert fd_hess_error(bad) > 1e-3


def test_wrong_curvature_sign_caught():
    def bad(Y, U, prob, Xt, sigma):
        G = sp.egrad_S(Y, prob, Xt, sigma)
        U = sp.proj_tangent(Y, U)
        H = sp.ehess(Y, U, prob, Xt, sigma, G)
        z = sp.rowdot(G @ Y, Y)
        return H - sp.rowdot(H, Y)[:, None] * Y + 2.0 * z[:, None] * U
    assert fd_hess_error(bad) > 1e-3


def test_transposed_gradient_operand_caught():
    prob, Xt, Y, rng = setup(seed=8)
    G = sp.egrad_S(Y, prob, Xt, 1.0)
    G_bad = G + np.triu(np.ones_like(G), 1) * 0.1  # loses symmetry, as a mixed-up operand would
    g_ok = sp.rgrad(Y, prob, Xt, 1.0)
    g_bad = sp.proj_tangent(Y, 2.0 * G_bad.T @ Y)
    U = tangent(rng, Y)
    f = lambda t: sp.cost(sp.retract(Y, t * U), prob, Xt, 1.0)
    fd = (f(1e-4) - f(-1e-4)) / 2e-4
    assert abs(fd - np.sum(g_ok * U)) < 1e-6 * abs(fd)
    assert abs(fd - np.sum(g_bad * U)) > 1e-3 * abs(fd)


def test_missing_factor_two_in_rhs_caught():
    q = 5
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    b = moment.rhs(q, Q, c).copy()
    b[1 + q:1 + q + q * (q - 1) // 2] *= 0.5
    monos = moment.monomials(q)
    x = np.array([1.0, -1.0, 1.0, 1.0, -1.0])
    mv = np.array([np.prod(x[list(s)]) for s in monos])
    assert abs(b @ mv - moment.bqp_objective(x, Q, c)) > 1e-3


def complex_hess_fd_error(hess_fn):
    from oracle import ucqp_complex as uc
    from synthetic import ucqp_instance
    Q = ucqp_instance(8, 2)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    Y /= np.linalg.norm(Y, axis=1)[:, None]
    U = uc.proj_tangent(Y, rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3)))
    t = 1e-5
    fd = uc.proj_tangent(Y, (uc.rgrad(uc.retract(Y, t * U), Q)
                             - uc.rgrad(uc.retract(Y, -t * U), Q)) / (2 * t))
    H = hess_fn(Y, U, Q)
    return np.abs(fd - H).max() / np.abs(H).max()


def test_complex_hessian_pins_catch_a_dropped_weingarten_term_and_a_conjugation():
    from oracle import ucqp_complex as uc
    assert complex_hess_fd_error(uc.rhess) < 1e-6

    def no_weingarten(Y, U, Q):
        return uc.proj_tangent(Y, 2.0 * (Q @ U))
    assert complex_hess_fd_error(no_weingarten) > 1e-3

    def conjugated(Y, U, Q):  # Q^T in place of the Hermitian Q
        return uc.proj_tangent(Y, 2.0 * (Q.T @ U)) - 2.0 * uc.multipliers(Y, Q)[:, None] * U
    assert complex_hess_fd_error(conjugated) > 1e-3


def test_multiblock_rhs_pin_catches_an_overwritten_shared_monomial():
    """Blocks share two variables, so the monomials of those variables collect terms
    from both blocks; overwriting instead of accumulating must break the pin that b
    reproduces the objective."""
    import math
    from oracle import multiblock as mb
    from synthetic import sparse_bqp_instance
    q, t = 4, 3
    Qs, cs = sparse_bqp_instance(q, t, 5)
    mons = mb.monomials(q, t)
    rank = {mono: r for r, mono in enumerate(mons)}

    def bad_rhs():
        b = np.array(mb.rhs(q, t, Qs, cs))
        for k, vars_k in enumerate(mb.block_variables(q, t)):  # overwrite: last block wins
            for i in range(q):
                b[rank[(vars_k[i],)]] = cs[k][i]
        return b

    def max_error(b):
        rng = np.random.default_rng(0)
        err = 0.0
        for _ in range(20):
            x = rng.choice([-1.0, 1.0], mb.num_variables(q, t))
            val = sum(b[a] * math.prod(x[i] for i in mono) for a, mono in enumerate(mons))
            err = max(err, abs(val - mb.objective(x, q, t, Qs, cs)))
        return err

    assert max_error(mb.rhs(q, t, Qs, cs)) < 1e-10
    assert max_error(bad_rhs()) > 1e-3
