"""Preconditioned conjugate gradients (oracle; test infrastructure only).

``pcg`` is Algorithm 1 (and, with the UNO preconditioner, Algorithm 2) step by step, with the
stopping test taken relative to the initial residual: the loop runs while
``||r||_inf > tol * ||r0||_inf`` (the relative residual of Sec. 7.1 and App. E; with ``u0 = 0``
this is ``||r||_inf / ||f||_inf``).

``fcg_pr`` is the flexible variant used to cross-check a mixed-precision solver: the same loop
with the Polak-Ribiere coefficient ``beta = r_{m+1}.(s_{m+1} - s_m) / (r_m . s_m)``.
"""
from __future__ import annotations

import numpy as np


def pcg(apply_A, f, apply_P, tol: float, max_iter: int, u0=None):
    """Returns ``(u, iterations, residual_history)``; history holds ``||r||_inf`` per check."""
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64)
    r = f - apply_A(u)                       # initial residual
    d = np.zeros_like(f)                     # search direction
    gamma1 = 1.0
    r0 = float(np.max(np.abs(r))) if r.size else 0.0
    hist = [r0]
    it = 0
    while float(np.max(np.abs(r))) > tol * r0 and it < max_iter:
        s = apply_P(r)                       # apply preconditioner
        gamma0 = gamma1
        gamma1 = float(r @ s)
        d = s + (gamma1 / gamma0) * d        # update search direction
        p = apply_A(d)                       # matrix-vector product
        alpha = gamma1 / float(d @ p)        # optimal step width
        r = r - alpha * p                    # update residual
        u = u + alpha * d                    # update solution approximation
        it += 1
        hist.append(float(np.max(np.abs(r))))
    return u, it, hist


def fcg_pr(apply_A, f, apply_P, tol: float, max_iter: int, u0=None):
    """Flexible PCG with the Polak-Ribiere coefficient; same interface as ``pcg``."""
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64)
    r = f - apply_A(u)
    d = np.zeros_like(f)
    s_old = np.zeros_like(f)
    gamma1 = 1.0
    r0 = float(np.max(np.abs(r))) if r.size else 0.0
    hist = [r0]
    it = 0
    while float(np.max(np.abs(r))) > tol * r0 and it < max_iter:
        s = apply_P(r)
        gamma0 = gamma1
        gamma1 = float(r @ s)
        beta = (gamma1 - float(r @ s_old)) / gamma0
        d = s + beta * d
        p = apply_A(d)
        alpha = gamma1 / float(d @ p)
        r = r - alpha * p
        u = u + alpha * d
        s_old = s
        it += 1
        hist.append(float(np.max(np.abs(r))))
    return u, it, hist


def cg_iteration_estimate(cond: float, tol: float) -> float:
    """Iterations after which the bound of Eq. (cg-convergence), ``2 C^m``, drops below tol."""
    C = (np.sqrt(cond) - 1.0) / (np.sqrt(cond) + 1.0)
    return float(np.log(tol / 2.0) / np.log(C))
