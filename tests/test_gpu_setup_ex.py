"""manidsdp_setup_ex's layouts give the same problem as manidsdp_setup: a
packed-upper index map (mirrored by the library) and a cost C given in CSR form
(expanded on setup) solve to bit-identical results; malformed descriptors are
rejected with E_ARG."""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from synthetic import gaussian_factor
from tests.gpu_util import instance

pytestmark = pytest.mark.gpu


def solve(ctx, N, p0, seed):
    rep, p = mds.manidsdp_solve(ctx, gaussian_factor(N, p0, seed), p0)
    mds.manidsdp_destroy(ctx)
    return rep


def packed_upper(idx):
    N = idx.shape[0]
    return np.ascontiguousarray(idx[np.triu_indices(N)], dtype=np.int32)


@pytest.mark.parametrize("q,seed", [(5, 0), (8, 1)])
def test_packed_upper_index_map_solves_identically(q, seed):
    inst = instance(q, seed)
    N, m = inst["N"], inst["m"]
    a = solve(mds.manidsdp_setup(N, m, inst["idx"], inst["b"]), N, 2, seed)
    b = solve(mds.manidsdp_setup_ex(N, m, packed_upper(inst["idx"]), inst["b"],
                                    idx_layout=mds.IDX_PACKED_UPPER), N, 2, seed)
    assert a.status == mds.OK and b.status == mds.OK
    assert (a.value, a.eta_max, a.outer, a.hessvecs) == (b.value, b.eta_max, b.outer, b.hessvecs)


def test_csr_cost_solves_like_the_dense_cost():
    q, seed = 6, 2
    inst = instance(q, seed)
    N, m = inst["N"], inst["m"]
    rng = np.random.default_rng(9)
    C = np.zeros((N, N))
    mask = np.triu(rng.random((N, N)) < 0.1, 1)
    C[mask] = 0.1 * rng.standard_normal(mask.sum())
    C = C + C.T
    rows, cols = np.nonzero(C)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int64)
    a = solve(mds.manidsdp_setup(N, m, inst["idx"], inst["b"], mds.C_DENSE, C), N, 2, seed)
    b = solve(mds.manidsdp_setup_ex(N, m, inst["idx"], inst["b"], c_kind=mds.C_CSR,
                                    c_rowptr=rowptr, c_col=cols.astype(np.int32),
                                    c_val=np.ascontiguousarray(C[rows, cols])), N, 2, seed)
    assert a.status == mds.OK and b.status == mds.OK
    assert (a.value, a.eta_max, a.outer) == (b.value, b.eta_max, b.outer)


def test_malformed_descriptors_are_rejected():
    inst = instance(4, 0)
    N, m = inst["N"], inst["m"]
    rowptr = np.zeros(N + 1, dtype=np.int64)
    rowptr[1:] = 1
    rowptr = np.cumsum(rowptr)  # one entry per row: column 0 everywhere -> not symmetric
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_setup_ex(N, m, inst["idx"], inst["b"], c_kind=mds.C_CSR, c_rowptr=rowptr,
                              c_col=np.zeros(N, np.int32), c_val=np.arange(1.0, N + 1))
    assert e.value.status == mds.E_ARG
    bad = packed_upper(inst["idx"]).copy()
    bad[0] = m + 5  # class out of range after mirroring
    with pytest.raises(mds.ManidsdpError) as e:
        mds.manidsdp_setup_ex(N, m, bad, inst["b"], idx_layout=mds.IDX_PACKED_UPPER)
    assert e.value.status == mds.E_ARG
