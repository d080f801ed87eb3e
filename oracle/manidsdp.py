"""Algorithm 1 (ManiDSDP) in FP64, step by step.

Per outer iteration k (Algorithm 1):
  3. approximately minimise Psi_k on the oblique manifold N_p by RTR, warm-started
     at Y^k after a step along the carried direction U;
  4-8. S = Y Y';  y = (A A*)^{-1} A(S + C);  Xt <- Xt - sigma R with
     R = A*(y) - S - C;  z = diag((Xt + D) S);  X = Xt + D - Diag(z);
  9. if lambda_min(X) < 0 carry U = [0, V] (Theorem 4.5; Section 5.1);
  10. update the factorisation size p;
  11. sigma rule (Eq. (5.1)).
Stop when eta_max = max(eta_p, eta_d, eta_g) <= tol (the stopping criterion of Section 6).

Readings where the paper is silent (each also listed in the design notes):
  * Y^0: the printed Y^0 = 0 is not on N_p; we start from a caller-supplied
    Gaussian matrix with rows normalised.
  * Inner tolerance: RTR stops when ||grad|| <= eps_k with
    eps_k = max(tol_grad_min, min(tol_grad_max, tol_grad_factor * ||R^k|| / (1 + ||b||))),
    eps_0 = tol_grad_max, tol_grad_factor = 1: the same scaled residual the sigma
    rule (5.1) weighs against ||grad||, so the inner solve always has work while R
    is nonzero, and a subproblem solved to its tolerance leaves sigma unchanged
    (a factor 0.1 made sigma double after every solved subproblem, stiffening the
    quartic penalty until the trust region collapsed).
  * Rank update (the paper defers to ManiSDP, Section 5.1, not reproduced in the
    paper): after the multiplier update, directions of Y whose eigenvalue in
    Y'Y falls below rank_tol * lambda_max(Y'Y) are dropped (Y <- Y V_r, rows
    renormalised), keeping p >= p_min; then, if lambda_min(X) < -neg_tol * (1 + |lambda_max(X)|),
    delta = min(#such eigenvalues among the delta_max smallest, delta_max) zero
    columns are appended, p <= p_max.
  * Inexact subproblems (Algorithm 1 asks only for an approximate solve): RTR
    stops at eps_k or after max_rtr = 15 iterations, tCG after max_tcg = 60
    Hessian-vector products.  With this budget the sigma rule (5.1) sees the
    gradient the capped solve leaves and lowers sigma while the subproblems are
    far from solved; the rank grows by up to delta_max = 16 directions per outer
    iteration and directions below rank_tol = 1e-6 lambda_max(Y'Y) are dropped.
    (Solving every subproblem to eps_k, up to 200 RTR iterations, stalled on the
    q = 80 relaxation with p held at 256: RTR at its cap in every outer
    iteration.)
  * Stall safeguard (sigma_stall = 0.5; 0 turns it off): after a subproblem
    solved to eps_k in which neither branch of (5.1) fired, sigma doubles when the
    scaled residual did not drop below sigma_stall times the previous one.  With
    eps_k tracking ||R|| a solved subproblem leaves ||grad|| close to eps_k, so the
    increase branch of (5.1) (kappa_2 = 10) cannot fire and a sigma lowered during
    capped early subproblems stays low.
  * tCG also stops once ||r_j|| <= tcg_abs * eps_k (tcg_abs = 0.1): the RTR
    asks for ||grad|| <= eps_k, so resolving the model gradient further is wasted.
  * Use of the carried U (step 3, "supplied with"): if the exact curvature
    <U, Hess Psi_{k+1}(Yhat)[U]> (Proposition 5.1) is negative, take
    Y <- Retr(Yhat + t U) for the largest t in t0 2^-j, j = 0..carry_halvings-1
    (t0 = carry_t0, or sqrt(N) when carry_t0 <= 0),
    that decreases Psi_{k+1} by at least 1e-4 t^2 |<U, Hess U>| / 2;
    otherwise drop the appended columns.
  * Eigenvectors are normalised to a positive first nonzero entry.
  * Rank-one rounding (the locking discussion notes that an exact rounding step
    turns near-locking into finite locking): after an outer iteration with
    eta_max <= round_eta, round Y to Yr = sign(Y w) (N x 1, w the top eigenvector of
    Y'Y).  If Yr Yr' is consistent with the classes (R = 0) and its certificate
    X_r = Xt + D - Diag(diag((Xt + D) Yr Yr')) with the current multiplier has
    lambda_min >= -tol (1 + |lambda_max|), the KKT residuals of (Yr, y_r, Xt) are
    at rounding level and the solve stops there.
"""
from __future__ import annotations

import math

import numpy as np

from . import direct as direct_mod
from . import operators as ops
from . import subproblem as sp
from .lanczos import lanczos
from .rtr import rtr

DEFAULTS = dict(
    sigma0=1.0, sigma_min=1e-3, sigma_max=1e6, gamma=2.0, kappa1=0.1, kappa2=10.0,
    p0=2, p_min=2, p_max=512, delta_max=16,
    max_outer=300, max_rtr=15, max_tcg=60, tol=1e-8,
    tol_grad_min=1e-11, tol_grad_max=1e-2, tol_grad_factor=1.0, tcg_floor=1e-10, tcg_abs=0.1,
    rank_tol=1e-6, neg_tol=1e-10, carry_halvings=30, carry_t0=0.0, round_eta=1e-2,
    lanczos_k=2000, sigma_stall=0.5,
)


def make_problem(idx, mult, b, C=None):
    return dict(idx=idx, mult=mult, b=b, C=C, D=ops.D_matrix(b, idx, mult), N=idx.shape[0])


def make_problem_general(Amat, b, C=None):
    """A general constraint operator: Amat is m x N^2, row i the vectorised
    symmetric matrix A_i, so A(Z)_i = <A_i, Z> and A*(v) = sum_i v_i A_i.  A A*
    is factored once by Cholesky (the remark after Algorithm 1); D = A*((A A*)^{-1} b)."""
    from scipy.linalg import cho_factor, cho_solve
    Amat = np.asarray(Amat, dtype=np.float64)
    N = int(round(math.sqrt(Amat.shape[1])))
    assert N * N == Amat.shape[1]
    Mfac = cho_factor(Amat @ Amat.T)
    D = (Amat.T @ cho_solve(Mfac, b)).reshape(N, N)
    return dict(Amat=Amat, Mfac=Mfac, N=N, b=np.asarray(b, dtype=np.float64), C=C, D=D,
                idx=None, mult=None)


def _rownorm(Y):
    return Y / np.linalg.norm(Y, axis=1)[:, None]


def _signfix(V):
    V = V.copy()
    for j in range(V.shape[1]):
        nz = np.nonzero(np.abs(V[:, j]) > 1e-14)[0]
        if len(nz) and V[nz[0], j] < 0:
            V[:, j] = -V[:, j]
    return V


def extreme_eigs(X, n_small, method="dense", lanczos_k=300, v0=None):
    """The n_small smallest eigenpairs and the largest eigenvalue of X."""
    N = X.shape[0]
    if method == "dense":
        w, V = np.linalg.eigh(X)
        return w[:n_small], _signfix(V[:, :n_small]), float(w[-1])
    if v0 is None:
        v0 = np.ones(N)
    lo, vecs, _ = lanczos(lambda v: X @ v, N, lanczos_k, v0, "min", n_small)
    hi, _, _ = lanczos(lambda v: X @ v, N, lanczos_k, v0, "max", 1)
    return lo, _signfix(vecs.T), float(hi[0])


def kkt_residuals(prob, y, S, X, z, lam_min, lam_max):
    """eta_p, eta_d, eta_g of Section 6."""
    C = prob["C"]
    Cz = 0.0 if C is None else C
    R = ops.Astar_prob(y, prob) - S - Cz
    normC = 0.0 if C is None else float(np.linalg.norm(C))
    eta_p = float(np.linalg.norm(R)) / (1.0 + normC)
    eta_d = max(0.0, -lam_min) / (1.0 + abs(lam_max))
    pobj = (0.0 if C is None else float(np.sum(C * (X + np.diag(z))))) + float(np.sum(z))
    dobj = float(prob["b"] @ y)
    eta_g = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    return eta_p, eta_d, eta_g, pobj, dobj


def solve(prob, Y0, params=None, eig="dense", history=None, direct=False):
    """Algorithm 1.  With direct=True each subproblem is the direct formulation's
    (oracle/direct.py: y frozen at the previous y-update instead of y(S)); the
    outer loop is otherwise the same."""
    prm = dict(DEFAULTS)
    if params:
        prm.update(params)
    b, C, D = prob["b"], prob["C"], prob["D"]
    N = prob["N"]
    Cz = 0.0 if C is None else C
    Y = _rownorm(np.array(Y0, dtype=np.float64))
    p = Y.shape[1]
    y_prev = ops.y_prob(Y @ Y.T + Cz, prob) if direct else None
    Xt = np.zeros((N, N))
    sigma = prm["sigma0"]
    U = None
    rscale = None
    Delta_bar = math.pi * math.sqrt(N)
    totals = dict(rtr=0, hessvecs=0)
    result = None
    for k in range(prm["max_outer"]):
        if direct:
            f = lambda Yv: direct_mod.cost(Yv, prob, Xt, sigma, y_prev)
            egrad = lambda Yv: direct_mod.egrad_S(Yv, prob, Xt, sigma, y_prev)
            rhess = lambda Yv, Uv, G: direct_mod.rhess(Yv, Uv, prob, Xt, sigma, y_prev, G)
        else:
            f = lambda Yv: sp.cost(Yv, prob, Xt, sigma)
            egrad = lambda Yv: sp.egrad_S(Yv, prob, Xt, sigma)
            rhess = lambda Yv, Uv, G: sp.rhess(Yv, Uv, prob, Xt, sigma, G)
        # step 3a: the carried direction
        if U is not None:
            G0 = egrad(Y)
            curv = float(np.sum(U * rhess(Y, U, G0)))
            moved = False
            if curv < 0.0:
                f0 = f(Y)
                t = prm["carry_t0"] if prm["carry_t0"] > 0 else math.sqrt(N)
                for _ in range(prm["carry_halvings"]):
                    Yt = sp.retract(Y, t * U)
                    if f(Yt) <= f0 - 1e-4 * 0.5 * t * t * abs(curv):
                        Y = Yt
                        moved = True
                        break
                    t *= 0.5
            if not moved:
                Y = Y[:, :p - U_cols]
                p = Y.shape[1]
            U = None
        # step 3b: RTR on Psi_k
        tol_k = prm["tol_grad_max"] if rscale is None else max(
            prm["tol_grad_min"], min(prm["tol_grad_max"], prm["tol_grad_factor"] * rscale))
        Gcache = {}

        def grad(Yv):
            G = egrad(Yv)
            Gcache["Y"], Gcache["G"] = Yv, G
            return sp.proj_tangent(Yv, 2.0 * G @ Yv)

        def hess(Yv, Uv):
            G = Gcache["G"] if Gcache.get("Y") is Yv else egrad(Yv)
            return rhess(Yv, Uv, G)

        Y, info = rtr(Y, f, grad, hess, sp.retract, Delta_bar, tol_k,
                      max_iter=prm["max_rtr"], max_tcg=prm["max_tcg"], tcg_floor=prm["tcg_floor"],
                      tcg_abs=prm["tcg_abs"])
        totals["rtr"] += info["iters"]
        totals["hessvecs"] += info["hessvecs"]
        gnorm = info["gradnorm"]
        # steps 4-8
        S = Y @ Y.T
        y = ops.y_prob(S if C is None else S + C, prob)
        y_prev = y
        R = ops.Astar_prob(y, prob) - S - Cz
        Xt = Xt - sigma * R
        z = sp.rowdot((Xt + D) @ Y, Y)
        X = Xt + D - np.diag(z)
        lam, V, lam_max = extreme_eigs(X, max(1, prm["delta_max"]), eig, prm["lanczos_k"])
        eta_p, eta_d, eta_g, pobj, dobj = kkt_residuals(prob, y, S, X, z, float(lam[0]), lam_max)
        eta = max(eta_p, eta_d, eta_g)
        if history is not None:
            history.append(dict(k=k, p=p, sigma=sigma, eta_p=eta_p, eta_d=eta_d, eta_g=eta_g,
                                lam_min=float(lam[0]), gnorm=gnorm, rtr=info["iters"],
                                hessvecs=info["hessvecs"], dobj=dobj))
        result = dict(Y=Y, y=y, Xt=Xt, z=z, X=X, S=S, eta=(eta_p, eta_d, eta_g), value=dobj,
                      pobj=pobj, outer=k + 1, p=p, sigma=sigma, lam_min=float(lam[0]),
                      lam_max=lam_max, totals=totals)
        if eta <= prm["tol"]:
            break
        # rank-one rounding
        if eta <= prm["round_eta"]:
            w_, Wv_ = np.linalg.eigh(Y.T @ Y)
            Yr = np.sign(Y @ Wv_[:, -1])[:, None]
            Yr[Yr == 0] = 1.0
            Sr = Yr @ Yr.T
            yr = ops.y_prob(Sr if C is None else Sr + C, prob)
            Rr = ops.Astar_prob(yr, prob) - Sr - Cz
            if np.abs(Rr).max() == 0.0:
                zr = sp.rowdot((Xt + D) @ Yr, Yr)
                Xr = Xt + D - np.diag(zr)
                lr, _, lmaxr = extreme_eigs(Xr, 1, eig, prm["lanczos_k"])
                er = kkt_residuals(prob, yr, Sr, Xr, zr, float(lr[0]), lmaxr)
                if max(er[:3]) <= prm["tol"]:
                    result = dict(Y=Yr, y=yr, Xt=Xt, z=zr, X=Xr, S=Sr, eta=er[:3], value=er[4],
                                  pobj=er[3], outer=k + 1, p=1, sigma=sigma,
                                  lam_min=float(lr[0]), lam_max=lmaxr, totals=totals,
                                  rounded=True)
                    if history is not None:
                        history.append(dict(k=k, p=1, sigma=sigma, eta_p=er[0], eta_d=er[1],
                                            eta_g=er[2], lam_min=float(lr[0]), gnorm=0.0, rtr=0,
                                            hessvecs=0, dobj=er[4], rounded=True))
                    break
        # step 10 (first half): drop numerically null directions of Y
        w, Wv = np.linalg.eigh(Y.T @ Y)
        keep = w > prm["rank_tol"] * w[-1]
        keep[-prm["p_min"]:] = True
        if keep.sum() < p:
            Y = _rownorm(Y @ Wv[:, keep])
            p = Y.shape[1]
        # step 11: sigma rule, Eq. (5.1)
        lhs = float(np.linalg.norm(R)) / (1.0 + float(np.linalg.norm(b)))
        lhs_prev = rscale
        rscale = lhs
        if lhs < prm["kappa1"] * gnorm:
            sigma = max(sigma / prm["gamma"], prm["sigma_min"])
        elif lhs > prm["kappa2"] * gnorm:
            sigma = min(prm["gamma"] * sigma, prm["sigma_max"])
        elif (prm["sigma_stall"] > 0 and lhs_prev is not None and gnorm <= tol_k
              and lhs > prm["sigma_stall"] * lhs_prev):
            # the stall safeguard (off by default): rule (5.1) cannot raise sigma once
            # eps_k tracks ||R||
            sigma = min(prm["gamma"] * sigma, prm["sigma_max"])
        # steps 9 and 10 (second half): negative curvature -> rank augmentation
        thr = -prm["neg_tol"] * (1.0 + abs(lam_max))
        neg = np.nonzero(lam < thr)[0]
        delta = min(len(neg), prm["delta_max"], prm["p_max"] - p)
        if delta > 0:
            Vn = V[:, neg[:delta]]
            Y = np.hstack([Y, np.zeros((N, delta))])
            U = np.hstack([np.zeros((N, p)), Vn])
            U_cols = delta
            p = p + delta
    return result
