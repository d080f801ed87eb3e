"""The direct formulation (params.direct = 1): the two-block ADMM on (DSDP) itself
(Section 3, the comparison with the direct subproblem), through the C ABI against
oracle/direct.py.

- subproblem value, Riemannian gradient and Hessian-vector product at a frozen y_k
  (Eq. (direct-ALM-subproblem); Eq. (hessian-comparison): sigma I in place of
  sigma Q) at 1e-12 in the FP64 form and 5e-5 with both FP32 engines;
- solves with a fixed penalty (sigma = 0.25, the reading for the direct scheme)
  reach the projected method's value (and the oracle's direct solve) to 1e-8 with
  eta_max <= 1e-8, in no fewer outer iterations than the projected method;
- the first outer iterations of the direct scheme follow the oracle's (eta_p after
  five iterations at q = 8).  The direct scheme converges linearly and slowly; its
  small instances finish through the rank-one rounding once eta_max <= 1e-2, so
  where that happens depends on the exact trajectory and later iterates are not
  compared.
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import direct, manidsdp as om, moment
from synthetic import bqp_instance, gaussian_factor
from tests.gpu_util import instance, random_state, relerr, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tc", [(mds.PREC_FP64, 0), (mds.PREC_MIXED, 0), (mds.PREC_MIXED, 1)])
def test_direct_subproblem_eval_and_hessvec(prec, tc):
    torch = torch_cuda()
    inst = instance(6, seed=4)
    prob, N, m = inst["prob"], inst["N"], inst["m"]
    p = 5
    Y, Xt, U = random_state(inst, p, seed=9)
    yk = np.random.default_rng(2).standard_normal(m)
    sigma = 0.7
    prm = mds.manidsdp_default_params()
    prm.precision_mode = prec
    prm.tensor_cores = tc
    prm.direct = 1
    ctx = mds.manidsdp_setup(N, m, inst["idx"], inst["b"], params=prm)
    try:
        mds.manidsdp_set_state(ctx, Xt, sigma)
        mds.manidsdp_set_direct_y(ctx, yk)
        Yd = torch.tensor(Y, device="cuda")
        g = torch.empty_like(Yd)
        psi, _ = mds.manidsdp_subproblem_eval(ctx, Yd, p, g)
        f_ref = direct.cost(Y, prob, Xt, sigma, yk)
        assert abs(psi - f_ref) <= 1e-12 * max(1.0, abs(f_ref))
        assert relerr(g.cpu().numpy(), direct.rgrad(Y, prob, Xt, sigma, yk)) <= 1e-12
        HU = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, torch.tensor(U, device="cuda"), p, HU, prec)
        err = relerr(HU.cpu().numpy(), direct.rhess(Y, U, prob, Xt, sigma, yk))
        assert err <= (1e-12 if prec == mds.PREC_FP64 else 5e-5), err
    finally:
        mds.manidsdp_destroy(ctx)


@pytest.mark.parametrize("q,seed,prec,tc", [(5, 0, mds.PREC_FP64, 0), (5, 0, mds.PREC_MIXED, 1),
                                            (10, 0, mds.PREC_FP64, 0), (10, 0, mds.PREC_MIXED, 1)])
def test_direct_solve_reaches_the_projected_value(q, seed, prec, tc):
    torch_cuda()
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    Y0 = gaussian_factor(N, 2, seed)
    out = {}
    for name, dflag in (("projected", 0), ("direct", 1)):
        prm = mds.manidsdp_default_params()
        prm.precision_mode, prm.tensor_cores = prec, tc
        prm.direct = dflag
        if dflag:
            prm.sigma0, prm.kappa1, prm.kappa2, prm.max_outer = 0.25, -1.0, 1e300, 1000
            prm.sigma_stall = 0.0
        ctx = mds.manidsdp_setup(N, m, idx, b, params=prm)
        try:
            out[name], _ = mds.manidsdp_solve(ctx, Y0, 2)
        finally:
            mds.manidsdp_destroy(ctx)
    ref_idx = moment.index_map(q)
    prob = om.make_problem(ref_idx, moment.multiplicities(ref_idx, m), moment.rhs(q, Q, c))
    ref = om.solve(prob, Y0, direct=True,
                   params=dict(sigma0=0.25, kappa1=-1.0, kappa2=1e300, sigma_stall=0.0,
                               max_outer=1000))
    pr, dr = out["projected"], out["direct"]
    print(f"q={q}: projected {pr.outer} outer, direct {dr.outer} outer (oracle {ref['outer']})")
    assert pr.status == mds.OK and dr.status == mds.OK and dr.eta_max <= 1e-8
    assert abs(dr.value - pr.value) <= 1e-8 * abs(pr.value)
    assert abs(dr.value - ref["value"]) <= 1e-8 * abs(ref["value"])
    assert dr.outer >= pr.outer


def test_direct_first_outer_iterations_follow_the_oracle():
    torch_cuda()
    q, seed, k = 8, 2, 5
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    Y0 = gaussian_factor(N, 2, seed)
    prm = mds.manidsdp_default_params()
    prm.direct = 1
    prm.sigma0, prm.kappa1, prm.kappa2, prm.max_outer = 0.25, -1.0, 1e300, k
    prm.sigma_stall = 0.0
    ctx = mds.manidsdp_setup(N, m, idx, b, params=prm)
    try:
        rep, _ = mds.manidsdp_solve(ctx, Y0, 2)
    finally:
        mds.manidsdp_destroy(ctx)
    ref_idx = moment.index_map(q)
    prob = om.make_problem(ref_idx, moment.multiplicities(ref_idx, m), moment.rhs(q, Q, c))
    hist = []
    om.solve(prob, Y0, direct=True, history=hist,
             params=dict(sigma0=0.25, kappa1=-1.0, kappa2=1e300, sigma_stall=0.0, max_outer=k))
    h = hist[-1]
    print(f"after {k} outer iterations: eta_p {rep.eta_p:.6e} (oracle {h['eta_p']:.6e}), "
          f"value {rep.value:.10f} (oracle {h['dobj']:.10f})")
    assert rep.outer == k
    assert abs(rep.eta_p - h["eta_p"]) <= 1e-3 * h["eta_p"]
    assert abs(rep.value - h["dobj"]) <= 1e-4 * abs(h["dobj"])
