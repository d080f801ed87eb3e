"""Parity at the benchmark's size: dense BQP order-2 relaxation, q = 80
(N = 3241, m = 1,666,981), through the C ABI against the FP64 oracle.
Index map and right-hand side bit-exact; Psi, grad, z, y and the Hessian-vector
product at p = 15 (p_0 = ceil(ln m)) and p = 100 (the large-p kernel paths),
with the same tolerances as the small cases (see test_gpu_parity)."""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import subproblem as sp
from tests.gpu_util import instance, random_state, relerr, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    inst = instance(80, seed=0)
    assert np.array_equal(inst["idx"], inst["prob"]["idx"])
    assert np.array_equal(inst["b"], inst["prob"]["b"])
    return inst


@pytest.mark.parametrize("ctx_prec", [mds.PREC_FP64, mds.PREC_MIXED])
@pytest.mark.parametrize("p", [15, 100])
def test_q80_eval_and_hessvec(big, p, ctx_prec):
    torch = torch_cuda()
    prob = big["prob"]
    Y, Xt, U = random_state(big, p, seed=p, xt_scale=0.05)
    sigma = 2.5
    prm = mds.manidsdp_default_params()
    prm.precision_mode = ctx_prec
    ctx = mds.manidsdp_setup(big["N"], big["m"], big["idx"], big["b"], params=prm)
    try:
        mds.manidsdp_set_state(ctx, Xt, sigma)
        Yd = torch.tensor(Y, device="cuda"); Ud = torch.tensor(U, device="cuda")
        g = torch.empty_like(Yd)
        z = torch.empty(big["N"], dtype=torch.float64, device="cuda")
        psi, rn = mds.manidsdp_subproblem_eval(ctx, Yd, p, g, z)
        G = sp.egrad_S(Y, prob, Xt, sigma)
        assert abs(psi - sp.cost(Y, prob, Xt, sigma)) <= 1e-12 * abs(sp.cost(Y, prob, Xt, sigma))
        assert relerr(g.cpu().numpy(), sp.proj_tangent(Y, 2 * G @ Y)) <= 1e-12
        assert relerr(z.cpu().numpy(), sp.rowdot(G @ Y, Y)) <= 1e-12
        H_ref = sp.rhess(Y, U, prob, Xt, sigma, G)
        HU = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, mds.PREC_FP64)
        assert relerr(HU.cpu().numpy(), H_ref) <= 1e-12
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, mds.PREC_MIXED)
        assert relerr(HU.cpu().numpy(), H_ref) <= 5e-5
    finally:
        mds.manidsdp_destroy(ctx)


@pytest.fixture(scope="module")
def sparse120():
    """The sparse-Q workload: q = 120, 5% Bernoulli support on the upper triangle
    (N = 7261, m = 8,502,671); index map and b bit-exact against the oracle."""
    inst = instance(120, seed=0, density=0.05)
    assert inst["N"] == 7261 and inst["m"] == 8502671
    assert np.array_equal(inst["idx"], inst["prob"]["idx"])
    assert np.array_equal(inst["b"], inst["prob"]["b"])
    return inst


@pytest.mark.parametrize("engine", [0, 1])
def test_q120_sparse_eval_and_hessvec(sparse120, engine):
    """Psi, grad, z (df64, 1e-12) and the mixed Hess-vec (5e-5) with both gather-GEMM
    engines at N = 7261: the largest index map of the workloads (211 MB)."""
    torch = torch_cuda()
    inst = sparse120
    prob = inst["prob"]
    p = 16
    Y, Xt, U = random_state(inst, p, seed=7, xt_scale=0.02)
    sigma = 2.0
    prm = mds.manidsdp_default_params()
    prm.precision_mode = mds.PREC_MIXED
    prm.tensor_cores = engine
    ctx = mds.manidsdp_setup(inst["N"], inst["m"], inst["idx"], inst["b"], params=prm)
    try:
        mds.manidsdp_set_state(ctx, Xt, sigma)
        Yd = torch.tensor(Y, device="cuda"); Ud = torch.tensor(U, device="cuda")
        g = torch.empty_like(Yd)
        z = torch.empty(inst["N"], dtype=torch.float64, device="cuda")
        psi, rn = mds.manidsdp_subproblem_eval(ctx, Yd, p, g, z)
        G = sp.egrad_S(Y, prob, Xt, sigma)
        psi_ref = sp.cost(Y, prob, Xt, sigma)
        assert abs(psi - psi_ref) <= 1e-12 * abs(psi_ref)
        assert relerr(g.cpu().numpy(), sp.proj_tangent(Y, 2 * G @ Y)) <= 1e-12
        assert relerr(z.cpu().numpy(), sp.rowdot(G @ Y, Y)) <= 1e-12
        HU = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, HU, mds.PREC_MIXED)
        err = relerr(HU.cpu().numpy(), sp.rhess(Y, U, prob, Xt, sigma, G))
        print(f"q=120 engine={engine}: Hess-vec relative error {err:.2e}")
        assert err <= 5e-5
    finally:
        mds.manidsdp_destroy(ctx)
