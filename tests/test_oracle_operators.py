"""Pins for the projectors of Section 3 (Eq. (projection-operators),
Eq. (projected-y), Eq. (projection-distance)) and D = A*(AA*)^{-1} b."""
import numpy as np
import pytest

from oracle import moment, operators as ops


@pytest.fixture(scope="module")
def data():
    q = 5
    idx = moment.index_map(q); m = moment.num_monomials(q)
    mult = moment.multiplicities(idx, m)
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    b = moment.rhs(q, Q, rng.standard_normal(q))
    return idx, mult, m, b


def sym(rng, N):
    Z = rng.standard_normal((N, N)); return Z + Z.T


def test_projector_idempotent_selfadjoint(data):
    idx, mult, m, _ = data
    rng = np.random.default_rng(0)
    N = idx.shape[0]
    Z1, Z2 = sym(rng, N), sym(rng, N)
    PZ = ops.P(Z1, idx, mult)
    assert np.allclose(ops.P(PZ, idx, mult), PZ, atol=1e-13)
    assert np.sum(PZ * Z2) == pytest.approx(np.sum(Z1 * ops.P(Z2, idx, mult)), rel=1e-12)
    # A(Q(Z)) = 0: Q projects onto ker A
    assert np.abs(ops.A(ops.Q(Z1, idx, mult), idx, m)).max() < 1e-12


def test_distance_to_range_is_norm_of_Q(data):
    """Eq. (projection-distance): min_y ||A*(y) - Z||^2 = ||Q(Z)||^2, with the
    least-squares problem solved by LAPACK on the explicit m x N^2 matrix."""
    idx, mult, m, _ = data
    rng = np.random.default_rng(1)
    N = idx.shape[0]
    Z = sym(rng, N)
    Amat = np.zeros((N * N, m))
    Amat[np.arange(N * N), idx.ravel()] = 1.0
    ybest, *_ = np.linalg.lstsq(Amat, Z.ravel(), rcond=None)
    dist2 = np.sum((Amat @ ybest - Z.ravel()) ** 2)
    QZ = ops.Q(Z, idx, mult)
    assert np.sum(QZ * QZ) == pytest.approx(dist2, rel=1e-10)
    # and y(S) is that least-squares solution (footnote to the variable projection)
    assert np.allclose(ops.y_of(Z, None, idx, mult), ybest, atol=1e-10)


def test_D_reproduces_b(data):
    """A(D) = b (Lemma 3.2's last line) and D is in range(A*)."""
    idx, mult, m, b = data
    D = ops.D_matrix(b, idx, mult)
    assert np.allclose(ops.A(D, idx, m), b, atol=1e-12)
    assert np.allclose(ops.Q(D, idx, mult), 0.0, atol=1e-13)
    assert np.array_equal(D, D.T)
