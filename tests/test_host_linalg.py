"""Host linear algebra of the rank update (the eigenvalues of the p x p Gram
Y'Y and the eigenvectors of the directions it keeps) against LAPACK: the
Householder tridiagonal form, Sturm bisection and inverse iteration compiled on
their own from ``csrc/host_linalg.h`` with the host C++ compiler."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_04406_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("hostla") / "eig_driver")
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CSRC}",
                    os.path.join(ROOT, "tests", "host", "eig_driver.cpp"), "-o", exe], check=True)
    return exe


def run(exe, A, r):
    n = A.shape[0]
    inp = f"{n} {r}\n" + "\n".join(" ".join(repr(float(x)) for x in row) for row in A) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    lines = out.strip().split("\n")
    w = np.array([float(x) for x in lines[:n]])
    V = np.array([[float(x) for x in ln.split()] for ln in lines[n:n + r]]).reshape(r, n).T
    return w, V


def gram(rng, N, p, decay):
    """Y'Y of an N x p factor with unit rows whose column scales decay
    geometrically: the spread of the spectra the rank update sees."""
    Y = rng.standard_normal((N, p)) * (decay ** np.arange(p))[None, :]
    Y /= np.linalg.norm(Y, axis=1)[:, None]
    return Y.T @ Y


@pytest.mark.parametrize("n,decay,seed", [(1, 1.0, 0), (2, 0.5, 1), (7, 0.9, 2), (40, 0.7, 3),
                                          (128, 0.95, 4), (300, 0.97, 5)])
def test_eigenvalues_match_lapack(driver, n, decay, seed):
    rng = np.random.default_rng(seed)
    A = gram(rng, max(3 * n, 8), n, decay)
    w, _ = run(driver, A, 0)
    ref = np.linalg.eigvalsh(A)
    assert np.abs(w - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n,r,seed", [(5, 2, 0), (60, 20, 1), (200, 150, 2)])
def test_kept_eigenvectors_span_the_top_eigenspace(driver, n, r, seed):
    """The r returned vectors are orthonormal and span the eigenspace of the r
    largest eigenvalues (checked through the projector, independent of the basis
    chosen within clusters)."""
    rng = np.random.default_rng(seed)
    A = gram(rng, 4 * n, n, 0.9)
    w, U = np.linalg.eigh(A)
    # the rank update keeps only directions well above rounding level
    r = min(r, int(np.sum(w > 1e-8 * w[-1])))
    _, V = run(driver, A, r)
    assert np.abs(V.T @ V - np.eye(r)).max() <= 1e-10
    P = U[:, -r:] @ U[:, -r:].T
    gap = (w[-r] - w[-r - 1]) / w[-1]
    assert np.abs(V @ V.T - P).max() <= 1e-9 / max(gap, 1e-6)
    assert np.linalg.norm(A @ V - V @ (V.T @ A @ V)) <= 1e-10 * w[-1] / max(gap, 1e-6)


def test_repeated_eigenvalues_and_zero_reflectors(driver):
    """A diagonal block (every reflector zero) plus a rank-two update: repeated
    eigenvalues; the top-two eigenspace is still recovered."""
    n = 12
    D = np.diag(np.r_[np.full(n - 2, 1.0), 5.0, 5.0])
    w, V = run(driver, D, 2)
    assert np.abs(w - np.sort(np.diag(D))).max() <= 1e-14 * 5
    P = np.zeros((n, n)); P[-2:, -2:] = np.eye(2)
    assert np.abs(V @ V.T - P).max() <= 1e-12
