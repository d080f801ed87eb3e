"""Differentiation through the C ABI (torch.autograd), checked against the
oracle and finite differences:
  * backward of Psi_k is the Riemannian gradient kernel (Prop. 4.2), double
    backward the Hessian-vector kernel (Eq. (4.7)) — equal to the oracle's to 1e-12;
  * the gradient matches a central difference of Psi along the retraction;
  * dV/db = y* and dV/dC = Xt* + D (envelope theorem on (PSDP)) match central
    differences of re-solved values; for a tight instance also the closed form
    dV/dQ_ij = 2 x_i x_j of the optimal vertex.
Also covers the dense-C path of the evaluation kernels."""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import manidsdp as om, subproblem as sp
from synthetic import bqp_instance, gaussian_factor
from tests.gpu_util import instance, random_state, relerr, torch_cuda

pytestmark = pytest.mark.gpu


def test_autograd_grad_and_double_backward():
    torch = torch_cuda()
    from paper_2512_04406_gb300.autograd import Subproblem
    inst = instance(10, seed=3)
    prob = inst["prob"]
    Y, Xt, U = random_state(inst, 5, seed=4)
    sigma = 1.3
    f = Subproblem(inst["N"], inst["m"], inst["idx"], inst["b"], Xt=Xt, sigma=sigma)
    try:
        Yd = torch.tensor(Y, device="cuda", requires_grad=True)
        psi = f(Yd)
        assert abs(psi.item() - sp.cost(Y, prob, Xt, sigma)) <= 1e-12 * abs(psi.item())
        (g,) = torch.autograd.grad(psi, Yd, create_graph=True)
        assert relerr(g.detach().cpu().numpy(), sp.rgrad(Y, prob, Xt, sigma)) <= 1e-12
        V = torch.tensor(U, device="cuda")
        (HV,) = torch.autograd.grad((g * V).sum(), Yd)
        assert relerr(HV.cpu().numpy(), sp.rhess(Y, U, prob, Xt, sigma)) <= 1e-12
        # first derivative along the retraction curve
        t = 1e-5
        fp = sp.cost(sp.retract(Y, t * U), prob, Xt, sigma)
        fm = sp.cost(sp.retract(Y, -t * U), prob, Xt, sigma)
        fd = (fp - fm) / (2 * t)
        assert abs(fd - float((g.detach() * V).sum())) <= 1e-6 * abs(fd)
    finally:
        f.close()


def test_dense_C_evaluation_parity():
    torch = torch_cuda()
    inst = instance(6, seed=2)
    rng = np.random.default_rng(9)
    N = inst["N"]
    C = rng.standard_normal((N, N)); C = 0.2 * (C + C.T)
    prob = om.make_problem(inst["prob"]["idx"], inst["prob"]["mult"], inst["prob"]["b"], C)
    Y, Xt, U = random_state(inst, 4, seed=5)
    ctx = mds.manidsdp_setup(N, inst["m"], inst["idx"], inst["b"], c_kind=mds.C_DENSE, c_dense=C)
    try:
        mds.manidsdp_set_state(ctx, Xt, 0.9)
        Yd = torch.tensor(Y, device="cuda")
        g = torch.empty_like(Yd)
        psi, rn = mds.manidsdp_subproblem_eval(ctx, Yd, 4, g)
        assert abs(psi - sp.cost(Y, prob, Xt, 0.9)) <= 1e-12 * max(1, abs(psi))
        assert relerr(g.cpu().numpy(), sp.rgrad(Y, prob, Xt, 0.9)) <= 1e-12
        HU = torch.empty_like(Yd)
        mds.manidsdp_hessvec(ctx, Yd, torch.tensor(U, device="cuda"), 4, HU)
        assert relerr(HU.cpu().numpy(), sp.rhess(Y, U, prob, Xt, 0.9)) <= 1e-12
    finally:
        mds.manidsdp_destroy(ctx)


def solve_value(q, Q, c, seed, tol=1e-11, order=2):
    N, m, idx = mds.manidsdp_bqp_index_map(q, order)
    b = mds.manidsdp_bqp_rhs(q, Q, c, order)
    prm = mds.manidsdp_default_params()
    prm.tol = tol
    prm.max_outer = 80
    from paper_2512_04406_gb300.autograd import value_and_sensitivities
    rep, y, XD = value_and_sensitivities(N, m, idx, b, gaussian_factor(N, 2, seed), prm)
    assert rep.status == mds.OK, rep.as_dict()
    return rep.value, y, XD, idx


def test_value_sensitivity_dV_dQ_finite_differences():
    torch_cuda()
    q, seed = 8, 1
    Q, c = bqp_instance(q, seed)
    V, y, XD, idx = solve_value(q, Q, c, seed)
    rng = np.random.default_rng(7)
    pairs = [tuple(sorted(rng.choice(q, 2, replace=False))) for _ in range(6)]
    h = 1e-6
    for i, j in pairs:
        Qp = Q.copy(); Qp[i, j] += h; Qp[j, i] += h
        Qm = Q.copy(); Qm[i, j] -= h; Qm[j, i] -= h
        fd = (solve_value(q, Qp, c, seed)[0] - solve_value(q, Qm, c, seed)[0]) / (2 * h)
        # b[x_i x_j] = Q_ij + Q_ji, so dV/dQ_ij (symmetric perturbation) = 2 y[x_i x_j]
        k = 1 + q + sum(q - 1 - t for t in range(i)) + (j - i - 1)
        assert abs(fd - 2 * y[k]) <= 1e-5 * max(1.0, abs(fd)), (i, j, fd, 2 * y[k])


def test_value_sensitivity_dV_dC_matches_dual_matrix():
    """dV/dC = Xt* + D.  Checked against the oracle's converged Xt + D, and exactly
    along range(A*): for E = A*(e) the substitution y -> y - e gives
    V(C + hE) = V(C) + h b'e, so <Xt* + D, E> must equal b'e, and re-solving with
    C = hE must move the value by h b'e.  (Difference quotients along ker A are
    ill-posed here: the perturbed problems leave the exact vertex, lose the
    residue dive and stall near 1e-9, in the oracle as well.)"""
    torch_cuda()
    from paper_2512_04406_gb300.autograd import value_and_sensitivities
    from oracle import moment
    q, seed = 6, 2
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    prm = mds.manidsdp_default_params(); prm.tol = 1e-10; prm.max_outer = 60
    rep, y, XD = value_and_sensitivities(N, m, idx, b, gaussian_factor(N, 2, seed), prm)
    ref_idx = moment.index_map(q)
    prob = om.make_problem(ref_idx, moment.multiplicities(ref_idx, m), moment.rhs(q, Q, c))
    ref = om.solve(prob, gaussian_factor(N, 2, seed), params=dict(tol=1e-10))
    assert np.abs(XD - (ref["Xt"] + prob["D"])).max() <= 1e-6 * (1 + np.abs(XD).max())
    assert np.abs(y - ref["y"]).max() <= 1e-6
    rng = np.random.default_rng(3)
    e = rng.standard_normal(m)
    E = e[idx]  # A*(e)
    assert float(np.sum(XD * E)) == pytest.approx(float(b @ e), rel=1e-9, abs=1e-9)
    h = 1e-3
    ctx = mds.manidsdp_setup(N, m, idx, b, c_kind=mds.C_DENSE, c_dense=h * E, params=prm)
    try:
        r, _ = mds.manidsdp_solve(ctx, gaussian_factor(N, 2, seed), 2)
    finally:
        mds.manidsdp_destroy(ctx)
    assert r.eta_max <= 1e-8
    assert (r.value - rep.value) / h == pytest.approx(float(b @ e), rel=1e-5, abs=1e-5)


def test_sdp_value_backward_gives_y_and_dual_matrix():
    """SDPValue's backward through torch.autograd: b.grad = y* and C.grad = Xt* + D
    (the same solve's multiplier and dual matrix), and <C.grad, A*(e)> = b'e for
    any e (the range(A*) identity of the dV/dC test above)."""
    torch = torch_cuda()
    from paper_2512_04406_gb300.autograd import SDPValue, value_and_sensitivities
    q, seed = 6, 2
    Q, c = bqp_instance(q, seed)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    b = mds.manidsdp_bqp_rhs(q, Q, c, 2)
    prm = mds.manidsdp_default_params(); prm.tol = 1e-10; prm.max_outer = 60
    Y0 = gaussian_factor(N, 2, seed)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    Ct = torch.zeros((N, N), dtype=torch.float64, device="cuda", requires_grad=True)
    V = SDPValue.apply(bt, Ct, N, m, idx, Y0, prm)
    V.backward()
    rep, y, XD = value_and_sensitivities(N, m, idx, b, Y0, prm)
    # (a zero dense C takes the dense-C kernels: the same solve up to rounding)
    assert abs(V.item() - rep.value) <= 1e-10 * abs(rep.value)
    assert np.abs(bt.grad.cpu().numpy() - y).max() <= 1e-9
    assert np.abs(Ct.grad.cpu().numpy() - XD).max() <= 1e-9 * (1 + np.abs(XD).max())
    e = np.random.default_rng(4).standard_normal(m)
    assert float(np.sum(Ct.grad.cpu().numpy() * e[idx])) == pytest.approx(float(b @ e), rel=1e-9,
                                                                          abs=1e-9)
    # C = None: only b gets a gradient
    bt2 = torch.tensor(b, device="cuda", requires_grad=True)
    SDPValue.apply(bt2, None, N, m, idx, Y0, prm).backward()
    assert np.abs(bt2.grad.cpu().numpy() - y).max() <= 1e-12  # the same path as value_and_sensitivities
