"""The benchmark's solve at full size: the dense BQP order-2 relaxation at q = 80
(N = 3241, m = 1,666,981) solved by the library in the mixed form with the
tensor-core Hess-vec, its final result checked on the host.

- KKT residuals of Section 6 recomputed from the returned y, Xt and Y with the
  oracle's operators and LAPACK eigenvalues of the certificate X: each <= 1e-8,
  and the library's own residuals reproduced to 1e-10.
- Tightness (Section 6.1 reports rank(S) = 1 on dense BQPs): the degree-1
  moments S[0, 1..q] round to x in {-1,1}^q with x'Qx + c'x = V to 1e-8 relative.
- Lanczos on the certificate at an intermediate iterate of the same solve (five
  outer iterations, p > 2): the smallest and largest Ritz values against LAPACK
  eigh of the same X, and the smallest pair's residual ||X v - lambda v||.
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import manidsdp as om, operators as ops, subproblem as sp
from synthetic import gaussian_factor
from tests.gpu_util import instance, torch_cuda

pytestmark = pytest.mark.gpu

Q80 = 80


@pytest.fixture(scope="module")
def big():
    return instance(Q80, seed=0)


def _solve(big, max_outer, lanczos_k=None):
    torch = torch_cuda()
    N, m = big["N"], big["m"]
    p0 = int(np.ceil(np.log(m)))
    prm = mds.manidsdp_default_params()
    prm.precision_mode = mds.PREC_MIXED
    prm.tensor_cores = 1
    prm.max_outer = max_outer
    if lanczos_k is not None:
        prm.lanczos_k = lanczos_k
    ctx = mds.manidsdp_setup(N, m, big["idx"], big["b"], params=prm)
    Y0 = gaussian_factor(N, p0, 0)
    Yout = np.empty(N * prm.p_max)
    y = np.empty(m)
    z = np.empty(N)
    Xt = np.empty((N, N))
    rep, p = mds.manidsdp_solve(ctx, Y0, p0, Y_out=Yout, y_out=y, z_out=z, Xt_out=Xt)
    return torch, ctx, rep, Yout[:N * p].reshape(N, p), p, y, z, Xt


def test_q80_solve_kkt_recomputed_on_host_and_tight(big):
    _, ctx, rep, Y, p, y, z, Xt = _solve(big, 300)
    try:
        assert rep.status == mds.OK and rep.eta_max <= 1e-8
        prob = big["prob"]
        S = Y @ Y.T
        assert np.abs(np.diag(S) - 1.0).max() <= 1e-13
        X = Xt + prob["D"] - np.diag(z)
        w = np.linalg.eigvalsh(X)
        eta_p, eta_d, eta_g, pobj, dobj = om.kkt_residuals(prob, y, S, X, z, w[0], w[-1])
        assert max(eta_p, eta_d, eta_g) <= 1e-8
        for mine, lib in ((eta_p, rep.eta_p), (eta_d, rep.eta_d), (eta_g, rep.eta_g)):
            assert abs(mine - lib) <= 1e-10
        assert abs(dobj - rep.value) <= 1e-12 * abs(rep.value)
        # z = diag((Xt + D) S) at the returned factor, and the multiplier in ker A (Lemma 3.2)
        assert np.abs(z - sp.rowdot((Xt + prob["D"]) @ Y, Y)).max() <= 1e-9 * np.abs(z).max()
        assert np.abs(ops.A(Xt, prob["idx"], len(y))).max() <= 1e-9 * (1 + np.abs(Xt).max())
        # tightness: the rounded degree-1 moments attain V
        x = np.where(S[0, 1:Q80 + 1] >= 0, 1.0, -1.0)
        f = float(x @ big["Q"] @ x + big["c"] @ x)
        assert abs(f - rep.value) <= 1e-8 * (1 + abs(rep.value))
    finally:
        mds.manidsdp_destroy(ctx)


def test_q80_lanczos_against_lapack_at_an_intermediate_iterate(big):
    torch, ctx, rep, Y, p, y, z, Xt = _solve(big, 5, lanczos_k=1200)
    try:
        assert p > 2
        prob = big["prob"]
        Yd = torch.tensor(Y, device="cuda")
        v = torch.empty(big["N"], dtype=torch.float64, device="cuda")
        lam_min, steps = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MIN, 1200, v)
        lam_max, _ = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MAX, 1200)
        XD = Xt + prob["D"]
        zz = sp.rowdot(XD @ Y, Y)
        X = XD - np.diag(zz)
        w = np.linalg.eigvalsh(X)
        scale = 1.0 + max(abs(w[0]), abs(w[-1]))
        vv = v.cpu().numpy()
        res = np.linalg.norm(X @ vv - lam_min * vv)
        print(f"q=80 p={p}: lambda_min {lam_min:.6e} (LAPACK {w[0]:.6e}), lambda_max "
              f"{lam_max:.6e} (LAPACK {w[-1]:.6e}), {steps} steps, residual {res:.2e}")
        assert abs(np.linalg.norm(vv) - 1.0) <= 1e-12
        assert res <= 1e-8 * scale
        # a Ritz value with residual r lies within r of an eigenvalue; the extreme one
        assert abs(lam_min - w[0]) <= max(1e-9 * scale, 2 * res)
        assert abs(lam_max - w[-1]) <= 1e-6 * scale
    finally:
        mds.manidsdp_destroy(ctx)
