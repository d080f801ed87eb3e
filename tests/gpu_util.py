"""Shared set-up for the GPU parity tests: the same seeded instance built once by
the library's host helpers (product path) and once by the oracle."""
import numpy as np

import paper_2512_04406_gb300 as mds
from oracle import manidsdp as om, moment, operators as ops, subproblem as sp
from synthetic import bqp_instance, gaussian_factor


def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def instance(q, seed=0, order=2, density=None):
    Q, c = bqp_instance(q, seed, density)
    N, m, idx = mds.manidsdp_bqp_index_map(q, order)
    b = mds.manidsdp_bqp_rhs(q, Q, c, order)
    ref_idx = moment.index_map(q, order)
    ref_b = moment.rhs(q, Q, c, order)
    prob = om.make_problem(ref_idx, moment.multiplicities(ref_idx, len(ref_b)), ref_b)
    return dict(q=q, Q=Q, c=c, N=N, m=m, idx=idx, b=b, prob=prob)


def random_state(inst, p, seed=1, xt_scale=0.3):
    """Unit-row Y, a multiplier in ker A (Lemma 3.2) and a random tangent U."""
    rng = np.random.default_rng(seed)
    N = inst["N"]
    prob = inst["prob"]
    Y = rng.standard_normal((N, p)); Y /= np.linalg.norm(Y, axis=1)[:, None]
    W = rng.standard_normal((N, N)); W = W + W.T
    Xt = xt_scale * ops.Q(W, prob["idx"], prob["mult"])
    U = sp.proj_tangent(Y, rng.standard_normal((N, p)))
    return Y, Xt, U


def relerr(a, ref):
    a = np.asarray(a); ref = np.asarray(ref)
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))
