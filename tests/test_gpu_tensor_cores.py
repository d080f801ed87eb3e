"""The tensor-core engine of the FP32 Hessian-vector product (params.tensor_cores
= 1: TMA-fed tcgen05 kind::tf32 SDDMM and gather GEMM on TF32 operand pairs,
three products per step) against the FP64 oracle (Proposition 4.2, Eq. (4.7))
and against the FP32 FMA kernels, through the C ABI.

Tolerances: the mixed-form Hessian-vector product's 5e-5 relative against the
oracle, for both FP32 engines and between them (the pairs represent each
operand to 2^-23, about FP32's own accuracy; the tensor core's FP32 accumulation
over chains of up to 640 K-values costs ~1e-5 at N = 3241).  A solve with the
tensor-core engine meets the solver bar: eta_max <= 1e-8, value within 1e-9 of
the oracle, also under the precision schedule (single TF32 products while
eta_max > tc_lowprec_eta).
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import manidsdp as om, subproblem as sp
from synthetic import gaussian_factor
from tests.gpu_util import instance, random_state, relerr, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def hessvec_both_engines(torch, inst, p, seed, sigma=1.3, xt_scale=0.3):
    Y, Xt, U = random_state(inst, p, seed=seed, xt_scale=xt_scale)
    prm = mds.manidsdp_default_params()
    prm.precision_mode = mds.PREC_MIXED
    prm.tensor_cores = 1
    ctx = mds.manidsdp_setup(inst["N"], inst["m"], inst["idx"], inst["b"], params=prm)
    try:
        mds.manidsdp_set_state(ctx, Xt, sigma)
        Yd = torch.tensor(Y, device="cuda")
        Ud = torch.tensor(U, device="cuda")
        mds.manidsdp_subproblem_eval(ctx, Yd, p)
        H_tc = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, H_tc, mds.PREC_MIXED)
        H_tc2 = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, H_tc2, mds.PREC_MIXED)
        prm.tensor_cores = 0
        mds.manidsdp_set_params(ctx, prm)
        H_fma = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, Ud, p, H_fma, mds.PREC_MIXED)
    finally:
        mds.manidsdp_destroy(ctx)
    H_ref = sp.rhess(Y, U, inst["prob"], Xt, sigma)
    return H_tc.cpu().numpy(), H_tc2.cpu().numpy(), H_fma.cpu().numpy(), H_ref


@pytest.mark.parametrize("q,p", [(1, 1), (3, 2), (6, 3), (10, 5), (20, 7), (20, 16), (20, 33),
                                 (20, 130), (20, 256), (20, 300), (20, 512)])
def test_tensor_core_hessvec_small(torch, q, p):
    inst = instance(q, seed=q)
    H_tc, H_tc2, H_fma, H_ref = hessvec_both_engines(torch, inst, p, seed=q + p)
    assert np.array_equal(H_tc, H_tc2)  # deterministic: no atomics in the reduction
    assert relerr(H_tc, H_ref) <= 5e-5
    assert relerr(H_fma, H_ref) <= 5e-5
    assert relerr(H_tc, H_fma) <= 5e-5


@pytest.mark.parametrize("p", [15, 100, 256, 330, 512])
def test_tensor_core_hessvec_q80(torch, p):
    inst = instance(80, seed=0)
    H_tc, _, H_fma, H_ref = hessvec_both_engines(torch, inst, p, seed=p, sigma=2.5, xt_scale=0.05)
    print(f"q=80 p={p}: tc {relerr(H_tc, H_ref):.2e}, fma {relerr(H_fma, H_ref):.2e} vs oracle")
    assert relerr(H_tc, H_ref) <= 5e-5
    assert relerr(H_fma, H_ref) <= 5e-5
    assert relerr(H_tc, H_fma) <= 5e-5


@pytest.mark.parametrize("q,seed,tcg_device,lowprec", [(8, 1, 1, 0.0), (12, 3, 1, 0.0),
                                                       (12, 3, 0, 0.0), (12, 3, 1, 1e-3)])
def test_tensor_core_solve(torch, q, seed, tcg_device, lowprec):
    inst = instance(q, seed)
    prm = mds.manidsdp_default_params()
    prm.precision_mode = mds.PREC_MIXED
    prm.tensor_cores = 1
    prm.tcg_device = tcg_device
    prm.tc_lowprec_eta = lowprec
    ctx = mds.manidsdp_setup(inst["N"], inst["m"], inst["idx"], inst["b"], params=prm)
    try:
        rep, _ = mds.manidsdp_solve(ctx, gaussian_factor(inst["N"], 2, seed), 2)
    finally:
        mds.manidsdp_destroy(ctx)
    ref = om.solve(inst["prob"], gaussian_factor(inst["N"], 2, seed))
    assert rep.status == mds.OK and rep.eta_max <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])
