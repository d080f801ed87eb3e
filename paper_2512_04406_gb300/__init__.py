"""Python binding of libmanidsdp: the GB300 hot path of ManiDSDP (arXiv 2512.04406).

Thin ctypes marshalling over the C ABI declared in ``include/manidsdp.h``; the
function names are the C names.  Arrays may be NumPy arrays (host memory) or
torch tensors (host or CUDA); every computation runs in the library's CUDA
kernels.  There is no CPU fallback: importing this package fails when the
shared library has not been built (``python -m paper_2512_04406_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

__all__ = [
    "ManidsdpError", "Params", "Report", "Context",
    "manidsdp_default_params", "manidsdp_strerror", "manidsdp_setup", "manidsdp_destroy",
    "manidsdp_set_state", "manidsdp_set_params", "manidsdp_get_multiplier",
    "manidsdp_get_dual_matrix",
    "manidsdp_subproblem_eval",
    "manidsdp_hessvec", "manidsdp_lanczos", "manidsdp_solve", "manidsdp_bqp_index_map",
    "manidsdp_bqp_rhs", "PREC_FP64", "PREC_MIXED", "EIG_MIN", "EIG_MAX", "C_ZERO", "C_DENSE",
    "lib_path", "manidsdp_launch_count", "manidsdp_hessvec_stage_ms", "manidsdp_ucqp_index_map",
    "manidsdp_ucqp_rhs", "Problem", "manidsdp_setup_ex", "manidsdp_setup_complex", "C_CSR",
    "IDX_FULL", "IDX_PACKED_UPPER", "BatchOut", "Batch", "manidsdp_batch_setup",
    "manidsdp_batch_solve", "manidsdp_batch_tune", "manidsdp_batch_set_launch",
    "manidsdp_batch_destroy", "manidsdp_solve_batched", "manidsdp_set_direct_y",
]

OK, E_ARG, E_NONFINITE, E_NOCONV, E_TIMEOUT, E_CUDA, E_NOMEM = 0, -1, -2, -3, -4, -5, -6
E_TOOLARGE = -7
C_ZERO, C_DENSE, C_CSR = 0, 1, 2
IDX_FULL, IDX_PACKED_UPPER = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
EIG_MIN, EIG_MAX = 0, 1

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"libmanidsdp.so is not built ({_LIB_PATH}); run `python -m paper_2512_04406_gb300.build`")
_lib = ctypes.CDLL(_LIB_PATH)


def lib_path() -> str:
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "sigma0", "sigma_min", "sigma_max", "gamma", "kappa1", "kappa2", "tol",
        "tol_grad_min", "tol_grad_max", "tol_grad_factor", "rank_tol", "neg_tol", "tcg_floor",
        "tcg_abs", "carry_t0", "round_eta", "tc_lowprec_eta")] + [
        (n, ctypes.c_int32) for n in (
            "p0", "p_min", "p_max", "delta_max", "max_outer", "max_rtr", "max_tcg",
            "carry_halvings", "lanczos_k", "precision_mode", "verbose", "profile", "tcg_device",
            "warm_start", "tensor_cores", "direct")] + [("sigma_stall", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Report(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "eta_p", "eta_d", "eta_g", "value", "pobj", "lambda_min", "lambda_max", "sigma",
        "ms_hessvec", "ms_eval", "ms_grad", "ms_lanczos", "ms_rank", "hessvec_p_sum")] + [
        (n, ctypes.c_int32) for n in (
            "outer", "rtr_iters", "hessvecs", "p", "lanczos_matvecs", "status", "evals",
            "grads")]

    @property
    def eta_max(self):
        return max(self.eta_p, self.eta_d, self.eta_g)

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Context(ctypes.c_void_p):
    """Opaque manidsdp_ctx*."""


class Problem(ctypes.Structure):
    """manidsdp_problem (the descriptor of manidsdp_setup_ex)."""
    _fields_ = [("N", ctypes.c_int32), ("m", ctypes.c_int64), ("idx", ctypes.c_void_p),
                ("idx_layout", ctypes.c_int32), ("b", ctypes.c_void_p), ("c_kind", ctypes.c_int32),
                ("c_dense", ctypes.c_void_p), ("c_rowptr", ctypes.c_void_p),
                ("c_col", ctypes.c_void_p), ("c_val", ctypes.c_void_p),
                ("is_complex", ctypes.c_int32), ("q_re", ctypes.c_void_p),
                ("q_im", ctypes.c_void_p)]


class BatchOut(ctypes.Structure):
    """manidsdp_batch_out: one instance's result of a batched solve."""
    _fields_ = [("value", ctypes.c_double), ("eta_p", ctypes.c_double),
                ("eta_d", ctypes.c_double), ("eta_g", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("status", ctypes.c_int32),
                ("p", ctypes.c_int32), ("outer", ctypes.c_int32), ("hessvecs", ctypes.c_int32),
                ("cycles", ctypes.c_int64 * 5)]

    @property
    def eta_max(self):
        return max(self.eta_p, self.eta_d, self.eta_g)


class Batch(ctypes.c_void_p):
    """Opaque manidsdp_batch*."""


_P = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_sig = {
    "manidsdp_default_params": (None, [ctypes.POINTER(Params)]),
    "manidsdp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "manidsdp_launch_count": (ctypes.c_longlong, []),
    "manidsdp_hessvec_stage_ms": (ctypes.c_int, [Context, _dp, ctypes.c_int]),
    "manidsdp_setup": (ctypes.c_int, [ctypes.POINTER(Context), ctypes.c_int32, ctypes.c_int64, _P,
                                      _P, ctypes.c_int32, _P, ctypes.POINTER(Params), _P]),
    "manidsdp_destroy": (None, [Context]),
    "manidsdp_setup_ex": (ctypes.c_int, [ctypes.POINTER(Context), ctypes.POINTER(Problem),
                                         ctypes.POINTER(Params), _P]),
    "manidsdp_set_state": (ctypes.c_int, [Context, _P, ctypes.c_double]),
    "manidsdp_set_direct_y": (ctypes.c_int, [Context, _P]),
    "manidsdp_set_params": (ctypes.c_int, [Context, ctypes.POINTER(Params)]),
    "manidsdp_get_multiplier": (ctypes.c_int, [Context, _P]),
    "manidsdp_get_dual_matrix": (ctypes.c_int, [Context, _P]),
    "manidsdp_subproblem_eval": (ctypes.c_int, [Context, _P, ctypes.c_int32, _dp, _P, _P, _P,
                                                _dp]),
    "manidsdp_hessvec": (ctypes.c_int, [Context, _P, _P, ctypes.c_int32, _P, ctypes.c_int32]),
    "manidsdp_lanczos": (ctypes.c_int, [Context, _P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, _dp, _P, ctypes.POINTER(ctypes.c_int32)]),
    "manidsdp_solve": (ctypes.c_int, [Context, _P, ctypes.c_int32, _P,
                                      ctypes.POINTER(ctypes.c_int32), _P, _P, _P,
                                      ctypes.POINTER(Report)]),
    "manidsdp_bqp_index_map": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int64), _P]),
    "manidsdp_bqp_rhs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "manidsdp_ucqp_index_map": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int64), _P]),
    "manidsdp_ucqp_rhs": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P]),
    "manidsdp_sparse_bqp_index_map": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_int32),
                                                     ctypes.POINTER(ctypes.c_int64),
                                                     ctypes.POINTER(ctypes.c_int64), _P]),
    "manidsdp_sparse_bqp_rhs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "manidsdp_lanczos_dense_noalloc": (ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.c_int32,
                                                      ctypes.c_int32,
                                                      ctypes.POINTER(ctypes.c_double), _P,
                                                      ctypes.POINTER(ctypes.c_int32), _P]),
    "manidsdp_batch_setup": (ctypes.c_int, [ctypes.POINTER(Batch), ctypes.c_int32, _P, _P, _P, _P,
                                            ctypes.POINTER(Params), _P]),
    "manidsdp_batch_solve": (ctypes.c_int, [Batch, _P, _P, _P, ctypes.POINTER(ctypes.c_float)]),
    "manidsdp_batch_tune": (ctypes.c_int, [Batch, _P, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "manidsdp_batch_set_launch": (ctypes.c_int, [Batch, ctypes.c_int32, ctypes.c_int32]),
    "manidsdp_batch_destroy": (None, [Batch]),
    "manidsdp_solve_batched": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P,
                                              ctypes.POINTER(Params), _P, _P, _P]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class ManidsdpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {manidsdp_strerror(status)} ({status})")


def _check(st: int, where: str, allow=(OK,)):
    if st not in allow:
        raise ManidsdpError(st, where)
    return st


def _ptr(a, dtype=None, writable=False):
    """Raw address of a contiguous NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if writable and not a.flags.writeable:
            raise ValueError("array is read-only")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def manidsdp_default_params() -> Params:
    p = Params()
    _lib.manidsdp_default_params(ctypes.byref(p))
    return p


def manidsdp_launch_count() -> int:
    return int(_lib.manidsdp_launch_count())


def manidsdp_hessvec_stage_ms(ctx: Context, reset: bool = True):
    """Per-stage device time of the Hessian-vector products (params.profile == 2)."""
    arr = (ctypes.c_double * 5)()
    _check(_lib.manidsdp_hessvec_stage_ms(ctx, arr, 1 if reset else 0), "manidsdp_hessvec_stage_ms")
    return dict(zip(("prep", "class_means", "gather_gemm", "gram", "epilogue"), list(arr)))


def manidsdp_strerror(status: int) -> str:
    return _lib.manidsdp_strerror(status).decode()


def manidsdp_setup(N: int, m: int, idx, b, c_kind: int = C_ZERO, c_dense=None,
                   params: Params | None = None, stream: int | None = None) -> Context:
    ctx = Context()
    st = _lib.manidsdp_setup(ctypes.byref(ctx), N, m, _ptr(idx, np.int32), _ptr(b, np.float64),
                             c_kind, _ptr(c_dense, np.float64),
                             ctypes.byref(params) if params is not None else None, stream)
    _check(st, "manidsdp_setup")
    return ctx


def manidsdp_setup_ex(N: int, m: int = 0, idx=None, b=None, idx_layout: int = IDX_FULL,
                      c_kind: int = C_ZERO, c_dense=None, c_rowptr=None, c_col=None, c_val=None,
                      is_complex: int = 0, q_re=None, q_im=None, params: Params | None = None,
                      stream: int | None = None) -> Context:
    """manidsdp_setup_ex: packed-upper index maps, a CSR cost C, or the first-order
    complex relaxation (is_complex = 1 with q_re, q_im)."""
    prob = Problem(N=N, m=m, idx=_ptr(idx, np.int32), idx_layout=idx_layout,
                   b=_ptr(b, np.float64), c_kind=c_kind, c_dense=_ptr(c_dense, np.float64),
                   c_rowptr=_ptr(c_rowptr, np.int64), c_col=_ptr(c_col, np.int32),
                   c_val=_ptr(c_val, np.float64), is_complex=is_complex,
                   q_re=_ptr(q_re, np.float64), q_im=_ptr(q_im, np.float64))
    ctx = Context()
    st = _lib.manidsdp_setup_ex(ctypes.byref(ctx), ctypes.byref(prob),
                                ctypes.byref(params) if params is not None else None, stream)
    _check(st, "manidsdp_setup_ex")
    return ctx


def manidsdp_setup_complex(Q, params: Params | None = None, stream: int | None = None) -> Context:
    """The first-order complex relaxation of min z^H Q z over |z_i| = 1 for a
    Hermitian (NumPy complex) Q; factors are n x 2p real arrays [Re | Im]."""
    Q = np.asarray(Q)
    qre = np.ascontiguousarray(Q.real, dtype=np.float64)
    qim = np.ascontiguousarray(Q.imag, dtype=np.float64)
    return manidsdp_setup_ex(Q.shape[0], is_complex=1, q_re=qre, q_im=qim, params=params,
                             stream=stream)


def manidsdp_destroy(ctx: Context) -> None:
    _lib.manidsdp_destroy(ctx)


def manidsdp_set_params(ctx: Context, params: Params) -> None:
    _check(_lib.manidsdp_set_params(ctx, ctypes.byref(params)), "manidsdp_set_params")


def manidsdp_set_state(ctx: Context, Xt=None, sigma: float = 1.0) -> None:
    _check(_lib.manidsdp_set_state(ctx, _ptr(Xt, np.float64), sigma), "manidsdp_set_state")


def manidsdp_set_direct_y(ctx: Context, y) -> None:
    _check(_lib.manidsdp_set_direct_y(ctx, _ptr(y, np.float64)), "manidsdp_set_direct_y")


def manidsdp_get_multiplier(ctx: Context, Xt) -> None:
    _check(_lib.manidsdp_get_multiplier(ctx, _ptr(Xt, np.float64, True)),
           "manidsdp_get_multiplier")


def manidsdp_get_dual_matrix(ctx: Context, XD) -> None:
    _check(_lib.manidsdp_get_dual_matrix(ctx, _ptr(XD, np.float64, True)),
           "manidsdp_get_dual_matrix")


def manidsdp_subproblem_eval(ctx: Context, Y, p: int, rgrad=None, z=None, y=None):
    """Returns (psi, ||R||); fills the given device outputs."""
    psi, rn = ctypes.c_double(), ctypes.c_double()
    st = _lib.manidsdp_subproblem_eval(ctx, _ptr(Y, np.float64), p, ctypes.byref(psi),
                                       _ptr(rgrad, np.float64, True), _ptr(z, np.float64, True),
                                       _ptr(y, np.float64, True), ctypes.byref(rn))
    _check(st, "manidsdp_subproblem_eval")
    return psi.value, rn.value


def manidsdp_hessvec(ctx: Context, Y, U, p: int, HU, precision: int = PREC_FP64) -> None:
    st = _lib.manidsdp_hessvec(ctx, _ptr(Y, np.float64), _ptr(U, np.float64), p,
                               _ptr(HU, np.float64, True), precision)
    _check(st, "manidsdp_hessvec")


def manidsdp_lanczos(ctx: Context, Y, p: int, which: int = EIG_MIN, k: int = 0, v=None):
    lam = ctypes.c_double()
    steps = ctypes.c_int32()
    st = _lib.manidsdp_lanczos(ctx, _ptr(Y, np.float64), p, which, k, ctypes.byref(lam),
                               _ptr(v, np.float64, True), ctypes.byref(steps))
    _check(st, "manidsdp_lanczos")
    return lam.value, steps.value


def manidsdp_lanczos_dense_noalloc(X, d=None, which: int = EIG_MIN, k: int = 0, v=None,
                                   stream: int | None = None):
    """Extreme eigenpair of X - Diag(d) for a device N x N FP64 matrix X (and an
    optional device N-vector d), computed in the library's static scratch with no
    device allocation.  Returns (lambda, steps); v (N FP64) receives the vector.

    The C entry point cannot see array sizes, so the shapes are checked here: X
    must be N x N, d and v must hold N entries; anything else raises ValueError
    before the library is called."""
    if len(X.shape) != 2 or int(X.shape[0]) != int(X.shape[1]):
        raise ValueError("manidsdp_lanczos_dense_noalloc: X must be a square N x N matrix")
    N = int(X.shape[0])
    for name, a in (("d", d), ("v", v)):
        if a is not None and tuple(int(s) for s in a.shape) != (N,):
            raise ValueError(f"manidsdp_lanczos_dense_noalloc: {name} must have shape ({N},)")
    lam = ctypes.c_double()
    steps = ctypes.c_int32()
    st = _lib.manidsdp_lanczos_dense_noalloc(N, _ptr(X, np.float64), _ptr(d, np.float64), which, k,
                                            ctypes.byref(lam), _ptr(v, np.float64, True),
                                            ctypes.byref(steps), stream)
    _check(st, "manidsdp_lanczos_dense_noalloc")
    return lam.value, steps.value


def manidsdp_solve(ctx: Context, Y0, p0: int, Y_out=None, y_out=None, z_out=None, Xt_out=None,
                   raise_on_noconv: bool = False):
    """Algorithm 1.  Returns (Report, p_final); status NOCONV is reported in
    Report.status unless raise_on_noconv."""
    rep = Report()
    pout = ctypes.c_int32()
    st = _lib.manidsdp_solve(ctx, _ptr(Y0, np.float64), p0, _ptr(Y_out, np.float64, True),
                             ctypes.byref(pout), _ptr(y_out, np.float64, True),
                             _ptr(z_out, np.float64, True), _ptr(Xt_out, np.float64, True),
                             ctypes.byref(rep))
    _check(st, "manidsdp_solve", allow=(OK,) if raise_on_noconv else (OK, E_NOCONV))
    return rep, pout.value


def manidsdp_bqp_index_map(q: int, order: int = 2):
    """Returns (N, m, idx[N, N] int32) for the BQP moment relaxation of the given order."""
    N, m = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.manidsdp_bqp_index_map(q, order, ctypes.byref(N), ctypes.byref(m), None),
           "manidsdp_bqp_index_map")
    idx = np.empty((N.value, N.value), dtype=np.int32)
    _check(_lib.manidsdp_bqp_index_map(q, order, ctypes.byref(N), ctypes.byref(m),
                                       _ptr(idx, np.int32, True)), "manidsdp_bqp_index_map")
    return N.value, m.value, idx


def manidsdp_bqp_rhs(q: int, Q, c=None, order: int = 2) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    N, m = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.manidsdp_bqp_index_map(q, order, ctypes.byref(N), ctypes.byref(m), None),
           "manidsdp_bqp_rhs")
    b = np.empty(m.value)
    _check(_lib.manidsdp_bqp_rhs(q, order, _ptr(Q), _ptr(c), _ptr(b, np.float64, True)),
           "manidsdp_bqp_rhs")
    return b


def manidsdp_sparse_bqp_index_map(q: int, t: int):
    """Returns (N, m, m_mono, idx[N, N] int32) of the embedded multi-block relaxation
    of a sparse BQP with t overlapping blocks of q variables."""
    N, m, mm = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.manidsdp_sparse_bqp_index_map(q, t, ctypes.byref(N), ctypes.byref(m),
                                              ctypes.byref(mm), None),
           "manidsdp_sparse_bqp_index_map")
    idx = np.empty((N.value, N.value), dtype=np.int32)
    _check(_lib.manidsdp_sparse_bqp_index_map(q, t, ctypes.byref(N), ctypes.byref(m),
                                              ctypes.byref(mm), _ptr(idx, np.int32, True)),
           "manidsdp_sparse_bqp_index_map")
    return N.value, m.value, mm.value, idx


def manidsdp_sparse_bqp_rhs(q: int, t: int, Qs, cs=None):
    """b (m FP64) for the blocks' Q_k (t x q x q) and c_k (t x q)."""
    _, m, _ = _sparse_sizes(q, t)
    Qa = np.ascontiguousarray(np.asarray(Qs, dtype=np.float64).reshape(t, q, q))
    ca = None if cs is None else np.ascontiguousarray(np.asarray(cs, dtype=np.float64).reshape(t, q))
    b = np.empty(m)
    _check(_lib.manidsdp_sparse_bqp_rhs(q, t, _ptr(Qa), _ptr(ca), _ptr(b, np.float64, True)),
           "manidsdp_sparse_bqp_rhs")
    return b


def _sparse_sizes(q: int, t: int):
    N, m, mm = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.manidsdp_sparse_bqp_index_map(q, t, ctypes.byref(N), ctypes.byref(m),
                                              ctypes.byref(mm), None),
           "manidsdp_sparse_bqp_index_map")
    return N.value, m.value, mm.value


def manidsdp_ucqp_index_map(q: int):
    """Returns (N, m, idx[N, N] int32) of the real second-order UCQP relaxation."""
    N, m = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.manidsdp_ucqp_index_map(q, ctypes.byref(N), ctypes.byref(m), None),
           "manidsdp_ucqp_index_map")
    idx = np.empty((N.value, N.value), dtype=np.int32)
    _check(_lib.manidsdp_ucqp_index_map(q, ctypes.byref(N), ctypes.byref(m),
                                        _ptr(idx, np.int32, True)), "manidsdp_ucqp_index_map")
    return N.value, m.value, idx


def manidsdp_ucqp_rhs(q: int, Q, c=None) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    N, m = ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.manidsdp_ucqp_index_map(q, ctypes.byref(N), ctypes.byref(m), None),
           "manidsdp_ucqp_rhs")
    b = np.empty(m.value)
    _check(_lib.manidsdp_ucqp_rhs(q, _ptr(Q), _ptr(c), _ptr(b, np.float64, True)),
           "manidsdp_ucqp_rhs")
    return b


def _batch_arrays(Ns, ms, idx, b):
    """Concatenated host arrays of a batch: (ninst, N int32, m int64, idx int32, b FP64).
    idx and b are lists of per-instance arrays or already-concatenated arrays."""
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int64)
    if len(Ns) != len(ms):
        raise ValueError("N and m must have one entry per instance")
    if isinstance(idx, (list, tuple)):
        idx = np.concatenate([np.asarray(a, dtype=np.int32).ravel() for a in idx])
    if isinstance(b, (list, tuple)):
        b = np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in b])
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if idx.size != int((Ns.astype(np.int64) ** 2).sum()) or b.size != int(ms.sum()):
        raise ValueError("idx must hold sum N_i^2 entries and b sum m_i entries")
    return len(Ns), Ns, ms, idx, b


def manidsdp_batch_setup(Ns, ms, idx, b, params: Params | None = None,
                         stream: int | None = None) -> Batch:
    """manidsdp_batch_setup over per-instance index maps idx[i] (N_i x N_i) and
    right-hand sides b[i] (m_i); lists or concatenated arrays.  The arrays are
    kept alive on the returned handle (the library copies them at setup)."""
    n, Ns, ms, idx, b = _batch_arrays(Ns, ms, idx, b)
    bt = Batch()
    st = _lib.manidsdp_batch_setup(ctypes.byref(bt), n, _ptr(Ns), _ptr(ms), _ptr(idx), _ptr(b),
                                   ctypes.byref(params) if params is not None else None, stream)
    _check(st, "manidsdp_batch_setup")
    bt._meta = (n, Ns, ms)
    return bt


def _y0_len(bt: Batch, p0: int) -> int:
    return int(bt._meta[1].astype(np.int64).sum()) * p0


def manidsdp_batch_solve(bt: Batch, Y0, y=None, raise_on_noconv: bool = False):
    """Returns (list of BatchOut, device ms).  Y0: the N_i x p0 starting factors
    concatenated (host array or CUDA tensor).  y: optional output of sum m_i FP64."""
    n = bt._meta[0]
    res = (BatchOut * n)()
    ms = ctypes.c_float()
    st = _lib.manidsdp_batch_solve(bt, _ptr(Y0, np.float64), ctypes.cast(res, _P),
                                   _ptr(y, np.float64, True), ctypes.byref(ms))
    _check(st, "manidsdp_batch_solve", allow=(OK,) if raise_on_noconv else (OK, E_NOCONV))
    return list(res), ms.value


def manidsdp_batch_tune(bt: Batch, Y0):
    """Returns the chosen (threads per CTA, CTAs per SM)."""
    th, per = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.manidsdp_batch_tune(bt, _ptr(Y0, np.float64), ctypes.byref(th),
                                    ctypes.byref(per)), "manidsdp_batch_tune")
    return th.value, per.value


def manidsdp_batch_set_launch(bt: Batch, threads: int, ctas_per_sm: int = 0) -> None:
    _check(_lib.manidsdp_batch_set_launch(bt, threads, ctas_per_sm), "manidsdp_batch_set_launch")


def manidsdp_batch_destroy(bt: Batch) -> None:
    _lib.manidsdp_batch_destroy(bt)


def manidsdp_solve_batched(Ns, ms, idx, b, Y0, params: Params | None = None, y=None,
                           stream: int | None = None, raise_on_noconv: bool = False):
    """One call (setup, solve, destroy).  Returns the list of BatchOut."""
    n, Ns, ms, idx, b = _batch_arrays(Ns, ms, idx, b)
    res = (BatchOut * n)()
    st = _lib.manidsdp_solve_batched(n, _ptr(Ns), _ptr(ms), _ptr(idx), _ptr(b),
                                     _ptr(Y0, np.float64),
                                     ctypes.byref(params) if params is not None else None,
                                     ctypes.cast(res, _P), _ptr(y, np.float64, True), stream)
    _check(st, "manidsdp_solve_batched", allow=(OK,) if raise_on_noconv else (OK, E_NOCONV))
    return list(res)
