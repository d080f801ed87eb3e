"""Riemannian trust region with truncated conjugate gradient.

The paper solves each factorised subproblem with the Riemannian trust-region
method of Absil, Baker and Gallivan (Section 4); it fixes no constants.  This is
the textbook method in its plain form:

  tCG (Steihaug-Toint) on the model m(eta) = f + <g, eta> + 1/2 <eta, H eta>
  inside ||eta|| <= Delta: stop on negative curvature or on reaching the
  boundary (step to the boundary), or when
  ||r_j|| <= ||r_0|| max(min(||r_0||^theta, kappa), floor).

  rho = (f(x) - f(R_x(eta)) + reg) / (m(0) - m(eta) + reg);
  Delta <- Delta/4 if rho < 1/4; Delta <- min(2 Delta, Delta_bar) if rho > 3/4 and
  the step reached the boundary; accept when rho > rho'.

Readings (stated, since the paper is silent): Delta_bar = pi sqrt(N) (the typical
distance on a product of N unit spheres), Delta_0 = Delta_bar / 8, rho' = 0.1,
kappa = 0.1, theta = 1, floor = 1e-10 (a reading: with theta = 1 the target
||r_0||^2 falls below what FP64 Hessian-vector products resolve once ||g|| is
small); reg = max(1, |f(x)|) * 1e3 * eps guards rho against
cancellation when both decreases reach rounding level.
"""
from __future__ import annotations

import math

import numpy as np


def inner(a, b) -> float:
    return float(np.sum(a * b))


def tcg(x, g, hess, Delta, kappa=0.1, theta=1.0, max_iter=1000, floor=1e-10, abs_tol=0.0):
    """Truncated CG.  Returns (eta, Heta, n_iter, stop_reason).  The relative
    residual target min(||r_0||^theta, kappa) is floored at ``floor``: below
    it the Hessian-vector products themselves are not that accurate."""
    eta = np.zeros_like(g)
    Heta = np.zeros_like(g)
    r = g.copy()
    rr = inner(r, r)
    r0 = math.sqrt(rr)
    delta = -r
    ee = 0.0            # <eta, eta>
    ed = 0.0            # <eta, delta>
    dd = rr             # <delta, delta>
    stop = "maxiter"
    j = 0
    for j in range(1, max_iter + 1):
        Hd = hess(x, delta)
        kap = inner(delta, Hd)
        alpha = rr / kap if kap != 0.0 else math.inf
        ee_new = ee + 2.0 * alpha * ed + alpha * alpha * dd
        if kap <= 0.0 or ee_new >= Delta * Delta:
            # step to the boundary along delta: ||eta + tau delta|| = Delta, tau > 0
            tau = (-ed + math.sqrt(ed * ed + dd * (Delta * Delta - ee))) / dd
            eta = eta + tau * delta
            Heta = Heta + tau * Hd
            stop = "negcurv" if kap <= 0.0 else "boundary"
            return eta, Heta, j, stop
        eta = eta + alpha * delta
        Heta = Heta + alpha * Hd
        ee = ee_new
        r = r + alpha * Hd
        rr_new = inner(r, r)
        if math.sqrt(rr_new) <= max(r0 * max(min(r0 ** theta, kappa), floor), abs_tol):
            stop = "converged"
            return eta, Heta, j, stop
        beta = rr_new / rr
        rr = rr_new
        delta = -r + beta * delta
        ed = beta * (ed + alpha * dd)
        dd = rr + beta * beta * dd
    return eta, Heta, j, stop


def rtr(x0, f, grad, hess, retr, Delta_bar, tol_grad, max_iter=200, max_tcg=1000,
        Delta0=None, rho_prime=0.1, kappa=0.1, theta=1.0, tcg_floor=1e-10, tcg_abs=0.0,
        log=None):
    """Riemannian trust region.  ``grad`` returns the Riemannian gradient;
    ``hess(x, u)`` the Riemannian Hessian applied to a tangent vector.
    Returns (x, info)."""
    x = x0
    fx = f(x)
    Delta = Delta_bar / 8.0 if Delta0 is None else Delta0
    info = {"iters": 0, "hessvecs": 0, "accepted": 0, "gradnorm": None}
    g = grad(x)
    gn = math.sqrt(inner(g, g))
    for it in range(max_iter):
        if gn <= tol_grad:
            break
        eta, Heta, nin, stop = tcg(x, g, hess, Delta, kappa, theta, max_tcg, tcg_floor,
                                   tcg_abs * tol_grad)
        info["hessvecs"] += nin
        x_new = retr(x, eta)
        f_new = f(x_new)
        model_dec = -(inner(g, eta) + 0.5 * inner(eta, Heta))
        reg = max(1.0, abs(fx)) * 1e3 * np.finfo(float).eps
        rho = (fx - f_new + reg) / (model_dec + reg) if model_dec + reg > 0 else -math.inf
        at_boundary = stop in ("negcurv", "boundary")
        if rho < 0.25:
            Delta = Delta / 4.0
        elif rho > 0.75 and at_boundary:
            Delta = min(2.0 * Delta, Delta_bar)
        if rho > rho_prime:
            x, fx = x_new, f_new
            g = grad(x)
            gn = math.sqrt(inner(g, g))
            info["accepted"] += 1
        if log is not None:
            log.append(dict(it=it, f=fx, gn=gn, rho=rho, Delta=Delta, tcg=nin, stop=stop))
        info["iters"] = it + 1
    info["gradnorm"] = gn
    info["f"] = fx
    return x, info
