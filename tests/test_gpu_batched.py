"""The batched solver (manidsdp_batch_*, manidsdp_solve_batched): thousands of
independent BQP relaxations in one persistent launch, each CTA running
Algorithm 1 on whole instances, against the FP64 oracle.

- a strided sample of the 4096-instance mix (first-order n in [16, 64],
  second-order n in [6, 14]) solved to tol 1e-10 in both precision forms: every
  value equal to the oracle's to 1e-9 relative, eta_max <= 1e-10, b'y_i = value;
- second-order instances against brute force over {-1,1}^n: the relaxation value
  is a lower bound, attained when the solve ended on an accepted rank-one rounding;
- the full mix at the default tolerance: every instance eta_max <= 1e-8;
- results independent of the grid (each instance is solved by one CTA, so the
  arithmetic does not depend on the number of CTAs), and the tuner's choice valid;
- the one-call manidsdp_solve_batched agrees with setup + solve;
- the batched backward: dV/dQ by central differences on 64 entries (129 solves in
  one launch) against 2 y[x_i x_j] from the returned multipliers.
"""
import numpy as np
import pytest

import paper_2512_04406_gb300 as mds
from oracle import brute, manidsdp as om
from tests.gpu_util import batch_mix, oracle_problem, torch_cuda

pytestmark = pytest.mark.gpu

SAMPLE = list(range(0, 3072, 97)) + list(range(3072, 4096, 41))


def params(prec, **kw):
    prm = mds.manidsdp_default_params()
    prm.p_max = 32
    prm.precision_mode = prec
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


@pytest.fixture(scope="module")
def sample():
    return batch_mix(select=SAMPLE)


@pytest.fixture(scope="module")
def oracle_values(sample):
    vals = []
    for q, order, Q, c, Y0 in zip(sample["q"], sample["order"], sample["Q"], sample["c"],
                                  sample["Y0"]):
        r = om.solve(oracle_problem(q, Q, c, order), Y0, dict(p_max=32, tol=1e-10))
        assert max(r["eta"]) <= 1e-10
        vals.append(r["value"])
    return np.array(vals)


@pytest.mark.parametrize("prec", [mds.PREC_FP64, mds.PREC_MIXED])
def test_batched_sample_matches_oracle(sample, oracle_values, prec):
    torch_cuda()
    bt = mds.manidsdp_batch_setup(sample["N"], sample["m"], sample["idx"], sample["b"],
                                  params(prec, tol=1e-10))
    try:
        y = np.empty(int(np.sum(sample["m"])))
        res, ms = mds.manidsdp_batch_solve(bt, sample["Y0cat"], y)
    finally:
        mds.manidsdp_batch_destroy(bt)
    vals = np.array([r.value for r in res])
    err = np.abs(vals - oracle_values) / np.abs(oracle_values)
    print(f"prec={prec}: {len(res)} instances in {ms:.1f} ms, max rel diff {err.max():.2e}, "
          f"max outer {max(r.outer for r in res)}, max p {max(r.p for r in res)}")
    assert all(r.status == mds.OK for r in res), [(i, r.status) for i, r in enumerate(res)
                                                  if r.status != mds.OK]
    assert max(r.eta_max for r in res) <= 1e-10
    assert err.max() <= 1e-9
    off = 0
    for r, b, m in zip(res, sample["b"], sample["m"]):
        assert abs(b @ y[off:off + m] - r.value) <= 1e-12 * (1 + abs(r.value))
        off += m


def test_batched_second_order_against_brute_force(sample):
    torch_cuda()
    sel = [k for k, o in enumerate(sample["order"]) if o == 2]
    bt = mds.manidsdp_batch_setup([sample["N"][k] for k in sel], [sample["m"][k] for k in sel],
                                  [sample["idx"][k] for k in sel], [sample["b"][k] for k in sel],
                                  params(mds.PREC_MIXED))
    try:
        Y0 = np.concatenate([sample["Y0"][k].ravel() for k in sel])
        res, _ = mds.manidsdp_batch_solve(bt, Y0)
    finally:
        mds.manidsdp_batch_destroy(bt)
    tight = 0
    for k, r in zip(sel, res):
        assert r.status == mds.OK
        fmin, _ = brute.bqp_min(sample["Q"][k], sample["c"][k])
        scale = 1 + abs(fmin)
        assert r.value <= fmin + 1e-9 * scale  # a relaxation: a lower bound
        if r.p == 1:  # ended on a rank-one rounding: the bound is attained
            assert abs(r.value - fmin) <= 1e-9 * scale
            tight += 1
    print(f"{tight} of {len(sel)} second-order instances tight")
    assert tight >= len(sel) // 2


def test_batched_full_mix_default_tolerance():
    torch_cuda()
    mix = batch_mix()
    bt = mds.manidsdp_batch_setup(mix["N"], mix["m"], mix["idx"], mix["b"],
                                  params(mds.PREC_MIXED))
    try:
        res, ms = mds.manidsdp_batch_solve(bt, mix["Y0cat"])
        res2, ms2 = mds.manidsdp_batch_solve(bt, mix["Y0cat"])
    finally:
        mds.manidsdp_batch_destroy(bt)
    print(f"4096 instances: {ms:.1f} ms ({4096 / ms * 1e3:.0f} solves/s), again {ms2:.1f} ms; "
          f"max outer {max(r.outer for r in res)}, max p {max(r.p for r in res)}")
    bad = [(i, r.status, r.eta_max) for i, r in enumerate(res) if r.status != mds.OK]
    assert not bad, bad[:10]
    assert max(r.eta_max for r in res) <= 1e-8
    assert [r.value for r in res] == [r.value for r in res2]


def test_batched_grid_independent_and_tuner(sample):
    torch_cuda()
    bt = mds.manidsdp_batch_setup(sample["N"], sample["m"], sample["idx"], sample["b"],
                                  params(mds.PREC_MIXED))
    try:
        mds.manidsdp_batch_set_launch(bt, 256, 1)
        a, _ = mds.manidsdp_batch_solve(bt, sample["Y0cat"])
        mds.manidsdp_batch_set_launch(bt, 256, 0)
        b, _ = mds.manidsdp_batch_solve(bt, sample["Y0cat"])
        th, per = mds.manidsdp_batch_tune(bt, sample["Y0cat"])
        c, _ = mds.manidsdp_batch_solve(bt, sample["Y0cat"])
    finally:
        mds.manidsdp_batch_destroy(bt)
    assert [r.value for r in a] == [r.value for r in b]
    assert th in (128, 256, 512) and per >= 1
    assert all(r.status == mds.OK and r.eta_max <= 1e-8 for r in c)
    if th == 256:
        assert [r.value for r in c] == [r.value for r in a]
    one = mds.manidsdp_solve_batched(sample["N"], sample["m"], sample["idx"], sample["b"],
                                     sample["Y0cat"], params(mds.PREC_MIXED))
    # the setup inside the one call picks up the shape just tuned
    assert [r.value for r in one] == [r.value for r in c]


@pytest.mark.parametrize("density,seed", [(0.05, 5), (None, 3)])
def test_batched_dV_dQ_central_differences_64_entries(density, seed):
    """dV/dQ_ij by central differences, h = 1e-6, on 64 random upper-triangle entries
    of a q = 12 instance (the sparse-Q recipe at 5 % support, and a dense Q): the
    129 solves (base and 2 x 64 perturbed) in one batched launch.  Since
    b[x_i x_j] = Q_ij + Q_ji, the envelope theorem gives dV/dQ_ij (symmetric
    perturbation E_ij + E_ji) = 2 y[x_i x_j] of the base solve; both instances are
    tight (rank-one rounding accepted), where the closed form 2 x_i x_j of the
    optimal vertex also holds."""
    from synthetic import bqp_instance, gaussian_factor
    torch_cuda()
    q, h = 12, 1e-6
    Q, c = bqp_instance(q, seed, density)
    N, m, idx = mds.manidsdp_bqp_index_map(q, 2)
    rng = np.random.default_rng(11)
    upper = [(i, j) for i in range(q) for j in range(i + 1, q)]
    pairs = [upper[k] for k in rng.choice(len(upper), 64, replace=False)]
    Qs = [Q]
    for i, j in pairs:
        for s in (1.0, -1.0):
            Qp = Q.copy()
            Qp[i, j] += s * h
            Qp[j, i] += s * h
            Qs.append(Qp)
    bs = [mds.manidsdp_bqp_rhs(q, Qk, c, 2) for Qk in Qs]
    Y0 = np.concatenate([gaussian_factor(N, 2, seed).ravel()] * len(Qs))
    prm = params(mds.PREC_FP64, tol=1e-12)
    bt = mds.manidsdp_batch_setup([N] * len(Qs), [m] * len(Qs), [idx] * len(Qs), bs, prm)
    try:
        y = np.empty(m * len(Qs))
        res, _ = mds.manidsdp_batch_solve(bt, Y0, y)
    finally:
        mds.manidsdp_batch_destroy(bt)
    assert all(r.status == mds.OK for r in res)
    assert all(r.p == 1 for r in res)  # every solve ended on an accepted rounding
    y0 = y[:m]
    for t, (i, j) in enumerate(pairs):
        fd = (res[1 + 2 * t].value - res[2 + 2 * t].value) / (2 * h)
        k = 1 + q + sum(q - 1 - u for u in range(i)) + (j - i - 1)  # class of x_i x_j
        assert abs(fd - 2 * y0[k]) <= 1e-5 * max(1.0, abs(fd)), (i, j, fd, 2 * y0[k])
        assert abs(abs(2 * y0[k]) - 2.0) <= 1e-9  # = 2 x_i x_j at the optimal vertex
