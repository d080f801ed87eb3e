"""manidsdp_lanczos_dense_noalloc against manidsdp_lanczos (the context's
certificate check) and against LAPACK on the same matrix.

The no-alloc entry point keeps its Krylov basis in a static device array, so
the file is collected last: it must give the context path's answer both when it
runs alone and after every other GPU test, and twice in a row (nothing left in
the scratch by one call may change the next).
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from tests.gpu_util import instance, random_state, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("q,p,k", [(4, 3, 0), (8, 3, 37), (16, 5, 60), (24, 7, 64)])
def test_noalloc_lanczos_matches_context_lanczos(torch, q, p, k):
    inst = instance(q, seed=q)
    N = inst["N"]
    if k == 0:
        k = N  # a full Krylov space: the Ritz values are eigenvalues of X
    Y, Xt, _ = random_state(inst, p, seed=5)
    ctx = mds.manidsdp_setup(N, inst["m"], inst["idx"], inst["b"])
    try:
        mds.manidsdp_set_state(ctx, Xt, 1.0)
        Yd = torch.tensor(Y, device="cuda")
        v_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        lam_ref, steps_ref = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MIN, k, v_ref)
        lmax_ref, steps_max_ref = mds.manidsdp_lanczos(ctx, Yd, p, mds.EIG_MAX, k)
        XD = torch.empty((N, N), dtype=torch.float64, device="cuda")
        mds.manidsdp_get_dual_matrix(ctx, XD)
    finally:
        mds.manidsdp_destroy(ctx)
    z = ((XD @ Yd) * Yd).sum(dim=1).contiguous()
    scale = 1.0 + max(abs(lam_ref), abs(lmax_ref))
    vr = v_ref.cpu().numpy()
    # the certificate's spectrum itself, independent of both CUDA paths
    X = (XD - torch.diag(z)).cpu().numpy()
    w, V = np.linalg.eigh(X)
    for _ in range(2):  # two calls in a row on the shared scratch
        v = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        lam, steps = mds.manidsdp_lanczos_dense_noalloc(XD, z, mds.EIG_MIN, k, v)
        vmax = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        lmax, steps_max = mds.manidsdp_lanczos_dense_noalloc(XD, z, mds.EIG_MAX, k, vmax)
        torch.cuda.synchronize()
        assert steps == steps_ref
        assert abs(lam - lam_ref) <= 1e-12 * scale
        vv = v.cpu().numpy()
        assert np.all(np.isfinite(vv))
        assert np.linalg.norm(vv - vr) <= 1e-8
        # both ends against LAPACK, and each Ritz pair's residual
        assert abs(lam - w[0]) <= 1e-9 * scale
        assert abs(lmax - w[-1]) <= 1e-9 * scale
        assert np.linalg.norm(X @ vv - lam * vv) <= 1e-8 * scale
        vm = vmax.cpu().numpy()
        assert np.linalg.norm(X @ vm - lmax * vm) <= 1e-8 * scale


def test_noalloc_lanczos_plain_matrix_and_host_vector(torch):
    """d = NULL (no diagonal shift) and a host output vector; both ends of the
    spectrum, each with its vector, against LAPACK."""
    rng = np.random.default_rng(7)
    N = 300
    A = rng.standard_normal((N, N))
    A = (A + A.T) / 2
    A[0, 0] -= 40.0  # one well-separated smallest eigenvalue
    A[1, 1] += 40.0  # and one well-separated largest
    Ad = torch.tensor(A, device="cuda")
    w, V = np.linalg.eigh(A)

    def signed(u):
        return u * np.sign(u[np.argmax(np.abs(u) > 1e-14)])

    for _ in range(2):
        vh = np.empty(N)
        lam, steps = mds.manidsdp_lanczos_dense_noalloc(Ad, None, mds.EIG_MIN, 80, vh)
        assert abs(lam - w[0]) <= 1e-10 * (1 + abs(w).max())
        assert np.linalg.norm(vh - signed(V[:, 0])) <= 1e-8
        vh = np.empty(N)
        lam, steps = mds.manidsdp_lanczos_dense_noalloc(Ad, None, mds.EIG_MAX, 80, vh)
        assert abs(lam - w[-1]) <= 1e-10 * (1 + abs(w).max())
        assert np.linalg.norm(vh - signed(V[:, -1])) <= 1e-8


def test_noalloc_lanczos_rejects_oversized_and_bad_inputs(torch):
    """Size limits through the raw C entry point (explicit N, a small buffer that is
    never read), argument errors through the binding."""
    import ctypes
    small = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    lam = ctypes.c_double()

    def raw(N, k, which=mds.EIG_MIN):
        return mds._lib.manidsdp_lanczos_dense_noalloc(
            N, ctypes.c_void_p(small.data_ptr()), None, which, k, ctypes.byref(lam), None, None,
            None)

    assert raw(16385, 4) == mds.E_TOOLARGE
    assert raw(8192, 65) == mds.E_TOOLARGE  # 65 x 8192 > 524288
    assert raw(4, 4, which=7) == mds.E_ARG
    with pytest.raises(mds.ManidsdpError) as e:  # pageable host memory is not device-readable
        mds.manidsdp_lanczos_dense_noalloc(np.zeros((4, 4)), None, mds.EIG_MIN, 4)
    assert e.value.status == mds.E_ARG
