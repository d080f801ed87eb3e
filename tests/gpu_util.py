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


def batch_mix(n1=3072, n2=1024, select=None):
    """The batch of independent BQP relaxations: n1 first-order relaxations with
    n uniform on [16, 64], then n2 second-order ones with n uniform on [6, 14]
    (Q, c iid N(0, 1), instance i seeded 1000 + i), built by the library's host
    helpers; starting factors N_i x 2 Gaussian (seed 1000 + i).  select: the
    instance numbers to keep (default all).  Returns a dict of per-instance lists
    and the concatenated starting factors."""
    from synthetic import batched_bqp_sizes
    s1, s2 = batched_bqp_sizes(n1, n2, 16, 64, 6, 14)
    spec = [(int(n), 1) for n in s1] + [(int(n), 2) for n in s2]
    keep = range(len(spec)) if select is None else select
    out = dict(i=[], q=[], order=[], N=[], m=[], idx=[], b=[], Q=[], c=[], Y0=[])
    for i in keep:
        q, order = spec[i]
        Q, c = bqp_instance(q, 1000 + i)
        N, m, idx = mds.manidsdp_bqp_index_map(q, order)
        for k, v in (("i", i), ("q", q), ("order", order), ("N", N), ("m", m), ("idx", idx),
                     ("b", mds.manidsdp_bqp_rhs(q, Q, c, order)), ("Q", Q), ("c", c),
                     ("Y0", gaussian_factor(N, 2, 1000 + i))):
            out[k].append(v)
    out["Y0cat"] = np.concatenate([y.ravel() for y in out["Y0"]])
    return out


def oracle_problem(q, Q, c, order):
    idx = moment.index_map(q, order)
    b = moment.rhs(q, Q, c, order)
    return om.make_problem(idx, moment.multiplicities(idx, len(b)), b)
