"""Sparse BQPs with overlapping variable blocks (Section 6, sparse BQPs) through
the C ABI: the embedded multi-block relaxation (manidsdp_sparse_bqp_index_map)
solved on the GPU, against the FP64 oracle on the oracle's own map and against
the brute-force minimum.  Bar: eta_max <= 1e-8, value within 1e-9 of the oracle,
value <= the brute-force minimum (weak duality)."""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import manidsdp as om, moment, multiblock as mb
from synthetic import gaussian_factor, sparse_bqp_instance
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("q,t,seed,prec,tc", [(5, 3, 1, mds.PREC_FP64, 0),
                                              (6, 3, 2, mds.PREC_FP64, 0),
                                              (6, 3, 2, mds.PREC_MIXED, 1)])
def test_sparse_bqp_solve_matches_oracle_and_brute_force(q, t, seed, prec, tc):
    torch_cuda()
    N, m, m_mono, idx = mds.manidsdp_sparse_bqp_index_map(q, t)
    Qs, cs = sparse_bqp_instance(q, t, seed)
    b = mds.manidsdp_sparse_bqp_rhs(q, t, Qs, cs)
    prm = mds.manidsdp_default_params()
    prm.precision_mode = prec
    prm.tensor_cores = tc
    ctx = mds.manidsdp_setup(N, m, idx, b, params=prm)
    try:
        rep, _ = mds.manidsdp_solve(ctx, gaussian_factor(N, 2, seed), 2)
    finally:
        mds.manidsdp_destroy(ctx)
    ref_idx, _ = mb.index_map(q, t)
    ref_b = mb.rhs(q, t, Qs, cs)
    prob = om.make_problem(ref_idx, moment.multiplicities(ref_idx, len(ref_b)), ref_b)
    ref = om.solve(prob, gaussian_factor(N, 2, seed))
    fmin, _ = mb.brute_min(q, t, Qs, cs)
    assert rep.status == mds.OK and rep.eta_max <= 1e-8
    assert abs(rep.value - ref["value"]) <= 1e-9 * abs(ref["value"])
    assert rep.value <= fmin + 1e-8 * (1 + abs(fmin))
