"""C ABI checks that need no GPU: the shared library loads and exports every
function declared in include/manidsdp.h; the host helpers that build the BQP
moment data agree bit for bit with the oracle (Section 3.1); argument checks
reject malformed index maps before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import moment

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(manidsdp_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(mds.lib_path())
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_match_documented_readings():
    p = mds.manidsdp_default_params()
    assert (p.sigma0, p.sigma_min, p.sigma_max, p.gamma, p.kappa1, p.kappa2) == (1.0, 1e-3, 1e6, 2.0, 0.1, 10.0)
    assert p.tol == 1e-8 and p.p0 == 2 and p.p_min == 2 and p.delta_max == 16
    assert mds.manidsdp_strerror(-1) == "invalid argument"
    # the library and the oracle implement the same readings with the same constants
    from oracle.manidsdp import DEFAULTS
    for k, v in DEFAULTS.items():
        if hasattr(p, k):
            assert getattr(p, k) == v, k


@pytest.mark.parametrize("q,order", [(1, 2), (2, 2), (3, 2), (5, 2), (9, 2), (20, 2), (4, 1), (17, 1)])
def test_bqp_index_map_bit_exact_vs_oracle(q, order):
    N, m, idx = mds.manidsdp_bqp_index_map(q, order)
    ref = moment.index_map(q, order)
    assert (N, m) == (ref.shape[0], moment.num_monomials(q, order))
    assert np.array_equal(idx, ref)


@pytest.mark.parametrize("q,order", [(6, 2), (11, 2), (8, 1)])
def test_bqp_rhs_bit_exact_vs_oracle(q, order):
    rng = np.random.default_rng(q)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    b = mds.manidsdp_bqp_rhs(q, Q, c, order)
    ref = moment.rhs(q, Q, c, order)
    assert np.array_equal(b, ref)


@pytest.mark.parametrize("q,density", [(80, None), (120, 0.05)])
def test_workload_index_maps_and_rhs_bit_exact_vs_oracle(q, density):
    """The benchmark's dense q = 80 map (N = 3241) and the sparse-Q q = 120 map
    (N = 7261), with their right-hand sides, on the host."""
    from synthetic import bqp_instance
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    assert (N, m) == (1 + q + q * (q - 1) // 2, moment.num_monomials(q, 2))
    assert np.array_equal(idx, moment.index_map(q, 2))
    Q, c = bqp_instance(q, 0, density)
    assert np.array_equal(mds.manidsdp_bqp_rhs(q, Q, c, 2), moment.rhs(q, Q, c, 2))


def test_setup_rejects_bad_index_maps_before_touching_the_gpu():
    N, m, idx = mds.manidsdp_bqp_index_map(3, 2)
    b = np.zeros(m)
    bad = idx.copy(); bad[0, 1] = (bad[0, 1] + 1) % m  # breaks symmetry
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_setup(N, m, bad, b)
    assert e.value.status == mds.E_ARG
    bad = idx.copy(); bad[0, 0] = m  # out of range
    with pytest.raises(mds.ManidsdpError):
        mds.manidsdp_setup(N, m, bad, b)
    with pytest.raises(mds.ManidsdpError):  # a class with no entry: A A* singular
        mds.manidsdp_setup(N, m + 1, idx, np.zeros(m + 1))


@pytest.mark.parametrize("field,value", [("tensor_cores", 2), ("precision_mode", 5),
                                         ("tcg_device", -1), ("warm_start", 3), ("gamma", 1.0),
                                         ("p_max", 513), ("max_tcg", 0), ("sigma0", 0.0),
                                         ("direct", 2), ("sigma_stall", 1.0),
                                         ("sigma_stall", -0.5)])
def test_setup_rejects_out_of_range_params_before_touching_the_gpu(field, value):
    N, m, idx = mds.manidsdp_bqp_index_map(3, 2)
    prm = mds.manidsdp_default_params()
    setattr(prm, field, value)
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_setup(N, m, idx, np.zeros(m), params=prm)
    assert e.value.status == mds.E_ARG


@pytest.mark.parametrize("q", [1, 2, 3, 5, 8])
def test_ucqp_index_map_and_rhs_bit_exact_vs_oracle(q):
    from oracle import ucqp
    N, m, idx = mds.manidsdp_ucqp_index_map(q)
    ref, classes = ucqp.index_map(q)
    assert (N, m) == (ref.shape[0], len(classes))
    assert np.array_equal(idx, ref)
    rng = np.random.default_rng(q)
    Q = rng.standard_normal((q, q)); Q = Q + Q.T
    c = rng.standard_normal(q)
    assert np.array_equal(mds.manidsdp_ucqp_rhs(q, Q, c), ucqp.rhs(q, Q, c, classes))


def _noalloc_raw(N, which, k):
    """The C entry point itself with an explicit N and 1-element dummies: the size
    checks come before any pointer is read."""
    import ctypes
    dummy = np.zeros(1)
    lam = ctypes.c_double()
    return mds._lib.manidsdp_lanczos_dense_noalloc(
        N, dummy.ctypes.data_as(ctypes.c_void_p), None, which, k, ctypes.byref(lam), None,
        None, None)


def test_noalloc_lanczos_rejects_sizes_and_arguments_before_touching_the_gpu():
    """The no-alloc certificate check validates its sizes against the static
    scratch (N <= 16384, k <= 256, k N <= 524288) and its arguments before any
    CUDA call, so these return on a machine without a GPU."""
    assert _noalloc_raw(16385, mds.EIG_MIN, 4) == mds.E_TOOLARGE
    assert _noalloc_raw(4096, mds.EIG_MIN, 129) == mds.E_TOOLARGE
    assert _noalloc_raw(4, 7, 4) == mds.E_ARG
    assert _noalloc_raw(0, mds.EIG_MIN, 4) == mds.E_ARG
    assert "scratch" in mds.manidsdp_strerror(mds.E_TOOLARGE)


def test_noalloc_wrapper_checks_shapes_before_the_call():
    """The binding refuses arrays whose shapes disagree with N (the C entry point
    reads N x N doubles of X and N of d and v whatever was allocated)."""
    with pytest.raises(ValueError):
        mds.manidsdp_lanczos_dense_noalloc(np.zeros((16385, 1)), None, mds.EIG_MIN, 4)
    with pytest.raises(ValueError):
        mds.manidsdp_lanczos_dense_noalloc(np.zeros((4, 4)), np.zeros(3), mds.EIG_MIN, 4)
    with pytest.raises(ValueError):
        mds.manidsdp_lanczos_dense_noalloc(np.zeros((4, 4)), None, mds.EIG_MIN, 4, np.zeros(5))
    with pytest.raises(ValueError):
        mds.manidsdp_lanczos_dense_noalloc(np.zeros(16), None, mds.EIG_MIN, 4)


@pytest.mark.parametrize("q,t", [(2, 3), (3, 1), (4, 2), (5, 3), (8, 4), (20, 2)])
def test_sparse_bqp_index_map_and_rhs_bit_exact_vs_oracle(q, t):
    from oracle import multiblock as mb
    from synthetic import sparse_bqp_instance
    N, m, m_mono, idx = mds.manidsdp_sparse_bqp_index_map(q, t)
    ref, nm = mb.index_map(q, t)
    assert (N, m, m_mono) == (ref.shape[0], mb.num_classes(q, t), nm)
    assert np.array_equal(idx, ref)
    Qs, cs = sparse_bqp_instance(q, t, q + t)
    assert np.array_equal(mds.manidsdp_sparse_bqp_rhs(q, t, Qs, cs), mb.rhs(q, t, Qs, cs))
    assert np.array_equal(mds.manidsdp_sparse_bqp_rhs(q, t, Qs, None),
                          mb.rhs(q, t, Qs, [np.zeros(q)] * t))


def test_batch_setup_rejects_bad_instances_before_touching_the_gpu():
    """The batched entry points validate every instance on the host first."""
    N1, m1, idx1 = mds.manidsdp_bqp_index_map(4, 2)
    N2, m2, idx2 = mds.manidsdp_bqp_index_map(20, 1)
    good = ([N1, N2], [m1, m2], [idx1, idx2], [np.zeros(m1), np.zeros(m2)])
    bad_sym = idx2.copy(); bad_sym[0, 1] = (bad_sym[0, 1] + 1) % m2
    cases = [
        ([N1, N2], [m1, m2], [idx1, bad_sym], good[3]),                 # not symmetric
        ([N1, N2], [m1, m2 + 1], [idx1, idx2], [np.zeros(m1), np.zeros(m2 + 1)]),  # empty class
    ]
    for Ns, ms, idx, b in cases:
        with pytest.raises(mds.ManidsdpError) as e:
            mds.manidsdp_batch_setup(Ns, ms, idx, b)
        assert e.value.status == mds.E_ARG
    # N above the one-CTA limit of 128: the order-2 moment matrix at q = 15 has N = 121,
    # at q = 16 N = 137
    N3, m3, idx3 = mds.manidsdp_bqp_index_map(16, 2)
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_batch_setup([N3], [m3], [idx3], [np.zeros(m3)])
    assert e.value.status == mds.E_ARG
    for field, value in (("p_max", 33), ("p0", 0), ("precision_mode", 4), ("gamma", 0.5),
                         ("direct", 1), ("sigma_stall", 1.5)):
        prm = mds.manidsdp_default_params()
        prm.p_max = 32
        setattr(prm, field, value)
        with pytest.raises(mds.ManidsdpError) as e:
            mds.manidsdp_batch_setup(*good, params=prm)
        assert e.value.status == mds.E_ARG
    with pytest.raises(ValueError):  # sizes inconsistent with the arrays
        mds.manidsdp_batch_setup([N1], [m1], [idx1, idx2], [np.zeros(m1)])
    b_nan = np.zeros(m1); b_nan[0] = np.nan
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_batch_setup([N1], [m1], [idx1], [b_nan])
    assert e.value.status == mds.E_NONFINITE


def test_complex_setup_rejects_the_direct_formulation_before_touching_the_gpu():
    """The first-order complex relaxation has no frozen-y formulation (every entry is
    its own class, R = 0): setup_ex refuses params.direct = 1 for it."""
    prm = mds.manidsdp_default_params()
    prm.direct = 1
    Q = np.eye(4, dtype=complex)
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_setup_complex(Q, prm)
    assert e.value.status == mds.E_ARG
