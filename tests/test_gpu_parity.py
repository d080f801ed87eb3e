"""GPU parity through the C ABI against the FP64 oracle.

Tolerances (normwise: max |gpu - oracle| / max |oracle|):
  FP64 primitives (Psi, grad, z, y, Hess-vec): 1e-12.
  Mixed-precision Hess-vec (FP32 products, FP32 accumulation over N terms):
  5e-5 (unit roundoff 6e-8 times a sqrt(N)-sized accumulation with headroom).
  Lanczos lambda_min: 1e-10 (1 + ||X||_2).
  Solves: both reach eta_max <= 1e-8; values agree to 1e-9 relative.
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import brute, manidsdp as om, subproblem as sp
from synthetic import gaussian_factor
from tests.gpu_util import instance, random_state, relerr, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [(1, 1), (3, 2), (6, 3), (10, 5), (20, 7), (20, 33)]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def make_ctx(inst, params=None):
    return mds.manidsdp_setup(inst["N"], inst["m"], inst["idx"], inst["b"], params=params)


@pytest.mark.parametrize("ctx_prec", [mds.PREC_FP64, mds.PREC_MIXED])
@pytest.mark.parametrize("q,p", CASES)
def test_subproblem_eval_and_hessvec_fp64(torch, q, p, ctx_prec):
    """ctx_prec FP64: native FP64 evaluation; MIXED: the evaluation runs as
    compensated float pairs (df64) on the FP32 pipe and must meet the same 1e-12."""
    inst = instance(q, seed=q)
    prob = inst["prob"]
    Y, Xt, U = random_state(inst, p, seed=q + p)
    sigma = 1.7
    prm = mds.manidsdp_default_params()
    prm.precision_mode = ctx_prec
    ctx = make_ctx(inst, prm)
    try:
        mds.manidsdp_set_state(ctx, Xt, sigma)
        N, m = inst["N"], inst["m"]
        Yd = torch.tensor(Y, device="cuda")
        Ud = torch.tensor(U, device="cuda")
        g = torch.empty_like(Yd); z = torch.empty(N, dtype=torch.float64, device="cuda")
        y = torch.empty(m, dtype=torch.float64, device="cuda")
        psi, rn = mds.manidsdp_subproblem_eval(ctx, Yd, p, g, z, y)
        psi_ref = sp.cost(Y, prob, Xt, sigma)
        g_ref = sp.rgrad(Y, prob, Xt, sigma)
        G = sp.egrad_S(Y, prob, Xt, sigma)
        z_ref = sp.rowdot(G @ Y, Y)
        R_ref, y_ref = sp.residual(Y, prob)
        assert abs(psi - psi_ref) <= 1e-12 * max(1.0, abs(psi_ref))
        assert abs(rn - np.linalg.norm(R_ref)) <= 1e-12 * max(1.0, np.linalg.norm(R_ref))
        assert relerr(g.cpu().numpy(), g_ref) <= 1e-12
        assert relerr(z.cpu().numpy(), z_ref) <= 1e-12
        assert relerr(y.cpu().numpy(), y_ref) <= 1e-12
        HU = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, mds.PREC_FP64)
        H_ref = sp.rhess(Y, U, prob, Xt, sigma)
        assert relerr(HU.cpu().numpy(), H_ref) <= 1e-12
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, mds.PREC_MIXED)
        assert relerr(HU.cpu().numpy(), H_ref) <= 5e-5
    finally:
        mds.manidsdp_destroy(ctx)


@pytest.mark.parametrize("q,p", [(6, 3), (10, 5), (20, 4)])
def test_lanczos_lambda_min_and_max(torch, q, p):
    inst = instance(q, seed=q)
    prob = inst["prob"]
    Y, Xt, _ = random_state(inst, p, seed=3)
    ctx = make_ctx(inst)
    try:
        mds.manidsdp_set_state(ctx, Xt, 1.0)
        Yd = torch.tensor(Y, device="cuda")
        v = torch.empty(inst["N"], dtype=torch.float64, device="cuda")
        lam, steps = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MIN, inst["N"], v)
        lmax, _ = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MAX, inst["N"])
        XD = Xt + prob["D"]
        z = sp.rowdot(XD @ Y, Y)
        X = XD - np.diag(z)
        w, V = np.linalg.eigh(X)
        scale = 1 + np.abs(w).max()
        assert abs(lam - w[0]) <= 1e-10 * scale
        assert abs(lmax - w[-1]) <= 1e-8 * scale
        vv = v.cpu().numpy()
        assert abs(np.linalg.norm(vv) - 1) < 1e-10
        assert np.linalg.norm(X @ vv - lam * vv) <= 1e-6 * scale
    finally:
        mds.manidsdp_destroy(ctx)


def gpu_solve(torch, inst, p0, seed, precision=mds.PREC_FP64, **kw):
    prm = mds.manidsdp_default_params()
    prm.precision_mode = precision
    for k, v in kw.items():
        setattr(prm, k, v)
    ctx = make_ctx(inst, prm)
    try:
        Y0 = gaussian_factor(inst["N"], p0, seed)
        y = np.empty(inst["m"])
        Yout = np.empty(inst["N"] * prm.p_max)
        rep, p = mds.manidsdp_solve(ctx, Y0, p0, Y_out=Yout, y_out=y)
        return rep, y, Yout[: inst["N"] * p].reshape(inst["N"], p)
    finally:
        mds.manidsdp_destroy(ctx)


@pytest.mark.parametrize("q,seed,tcg_device", [(4, 0, 1), (6, 1, 1), (10, 0, 1), (10, 0, 0),
                                               (14, 2, 1), (20, 0, 1)])
def test_solve_matches_oracle_fp64(torch, q, seed, tcg_device):
    """tcg_device = 1: each tCG run is one CUDA-graph launch looping on the
    device; 0: the host-driven loop."""
    inst = instance(q, seed)
    rep, y, Y = gpu_solve(torch, inst, 2, seed, tcg_device=tcg_device)
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, seed))
    assert rep.status == mds.OK and rep.eta_max <= 1e-8
    assert max(ref["eta"]) <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])
    assert np.allclose(np.linalg.norm(Y, axis=1), 1.0, atol=1e-13)
    if q <= 20:
        fmin, _ = brute.bqp_min(inst["Q"], inst["c"])
        assert rep.value <= fmin + 1e-8 * (1 + abs(fmin))


@pytest.mark.parametrize("q,seed", [(10, 0), (20, 0)])
def test_solve_mixed_precision_matches_oracle(torch, q, seed):
    inst = instance(q, seed)
    rep, y, _ = gpu_solve(torch, inst, 2, seed, precision=mds.PREC_MIXED)
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, seed))
    assert rep.status == mds.OK and rep.eta_max <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])


def test_order1_relaxation_solve(torch):
    inst = instance(24, seed=5, order=1)
    rep, _, _ = gpu_solve(torch, inst, 2, 5)
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, 5))
    assert rep.status == mds.OK and rep.eta_max <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])


@pytest.mark.parametrize("q,seed", [(3, 0), (4, 1)])
def test_ucqp_order2_solve_matches_oracle(torch, q, seed):
    """Real second-order UCQP relaxation (Section 3.1): the same hot path on a
    Laurent-exponent index map."""
    from oracle import ucqp
    from oracle.moment import multiplicities
    rng = np.random.default_rng(100 + seed)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    N, m, idx = mds.manidsdp_ucqp_index_map(q)
    b = mds.manidsdp_ucqp_rhs(q, Q, c)
    ref_idx, classes = ucqp.index_map(q)
    prob = om.make_problem(ref_idx, multiplicities(ref_idx, m), ucqp.rhs(q, Q, c, classes))
    ctx = mds.manidsdp_setup(N, m, idx, b)
    try:
        Y0 = gaussian_factor(N, 2, seed)
        rep, _ = mds.manidsdp_solve(ctx, Y0, 2)
    finally:
        mds.manidsdp_destroy(ctx)
    ref = om.solve(prob, Y0)
    assert rep.status == mds.OK and rep.eta_max <= 1e-8 and max(ref["eta"]) <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])
    best = min(ucqp.objective(rng.uniform(-np.pi, np.pi, q), Q, c) for _ in range(2000))
    assert rep.value <= best + 1e-8


@pytest.mark.parametrize("order,q,seed", [(1, 16, 1000), (1, 41, 1001), (1, 64, 1002),
                                          (2, 6, 1003), (2, 10, 1004), (2, 14, 1005)])
def test_small_instances_of_the_batched_mix(torch, order, q, seed):
    """Instances shaped like the many-small-instances workload (order-1 relaxations
    with n in [16, 64], order-2 with n in [6, 14], per-instance seeds), solved one by
    one through the same path; value against the oracle and, for n <= 16, brute force."""
    inst = instance(q, seed, order=order)
    rep, _, _ = gpu_solve(torch, inst, 2, seed)
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, seed))
    assert rep.status == mds.OK and rep.eta_max <= 1e-8 and max(ref["eta"]) <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])
    if q <= 16:
        fmin, _ = brute.bqp_min(inst["Q"], inst["c"])
        assert rep.value <= fmin + 1e-8 * (1 + abs(fmin))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_resumes_from_context_state(torch, prec):
    """A solve stopped after two outer iterations and resumed with warm_start
    (factor with its current column count, multiplier, sigma, inner-tolerance
    scale and carried direction kept in the context) follows the uninterrupted
    solve's trajectory exactly, and the resumed solve reaches the oracle's value."""
    inst = instance(12, 3)
    pm = mds.PREC_FP64 if prec == "fp64" else mds.PREC_MIXED
    Y0 = gaussian_factor(inst["N"], 2, 3)

    def params(max_outer, warm):
        prm = mds.manidsdp_default_params()
        prm.precision_mode = pm
        prm.max_outer = max_outer
        prm.warm_start = warm
        return prm

    ctx = make_ctx(inst, params(5, 0))
    try:
        whole, p_whole = mds.manidsdp_solve(ctx, Y0, 2)
    finally:
        mds.manidsdp_destroy(ctx)
    ctx = make_ctx(inst, params(2, 0))
    try:
        rep1, p1 = mds.manidsdp_solve(ctx, Y0, 2)
        assert rep1.outer == 2
        mds.manidsdp_set_params(ctx, params(3, 1))
        rep2, p2 = mds.manidsdp_solve(ctx, Y0, 2)
        mds.manidsdp_set_params(ctx, params(300, 1))
        rep3, _ = mds.manidsdp_solve(ctx, Y0, 2)
    finally:
        mds.manidsdp_destroy(ctx)
    if whole.outer == 5:  # not converged inside the first five iterations
        assert rep2.outer == 3 and p2 == p_whole
        assert rep2.value == whole.value and rep2.eta_p == whole.eta_p
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, 3))
    assert rep3.status == mds.OK and rep3.eta_max <= 1e-8
    assert abs(rep3.value - ref["value"]) <= 1e-9 * abs(ref["value"])
