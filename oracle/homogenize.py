"""Homogenization solves, effective tensors and sensitivities (oracle; tests only).

* ``solve``: for every macroscopic load, assemble f, run PCG (Algorithm 1) with no, Jacobi
  (Sec. 4.2) or UNO preconditioning (Algorithm 2), and project the fluctuation to zero mean
  (Sec. 6.1 / 6.2 require a zero-mean fluctuation field).
* ``effective_tensor``: volume average of the flux / stress, ``<C (eps_bar + eps(u))>``,
  evaluated with the element-averaged gradient (exact for trilinear fields).  For thermal
  problems with q = -kappa grad(theta) this is ``kappa_eff g_bar = -<q>``.
* ``energy_tensor``: ``W_lm = <(eps_bar_l + eps(u_l)) . C (eps_bar_m + eps(u_m))>`` by 2x2x2
  Gauss quadrature; equals the effective tensor at the discrete solution.
* ``sensitivity``: derivative of ``W`` with respect to the phase properties with the
  fluctuations held fixed, which is the total derivative because the discrete equations make
  ``W`` stationary in the fluctuations (K is self-adjoint, so the adjoint states are the forward
  solutions).
* ``direct_solve``: dense solve of the bordered system with zero-mean constraints (tiny grids).
"""
from __future__ import annotations

import numpy as np

from . import fem, pcg as _pcg, uno


def n_comp(physics: int) -> int:
    return 1 if physics == 1 else 3


def zero_mean(u: np.ndarray, c: int) -> np.ndarray:
    v = u.reshape(-1, c)
    return (v - v.mean(axis=0, keepdims=True)).ravel()


def preconditioner(kind: str, K, physics: int, props, shape, Q=None, L0: float = 1.0):
    c = n_comp(physics)
    if kind == "none":
        return lambda r: r.copy()
    if kind == "jacobi":
        diag = K.diagonal()
        return lambda r: r / diag
    if kind == "uno":
        if Q is None:
            Q = uno.reference_medium_Q(physics, props, shape, L0)
        return lambda r: fem.from_soa(uno.uno_apply(Q, fem.to_soa(r, c, shape)))
    raise ValueError(kind)


def solve(phase, props, physics: int, loads, precond: str = "uno", tol: float = 1e-8,
          max_iter: int = 100000, Q=None, flexible: bool = False, L0: float = 1.0):
    """Solve every load case; returns dict(u=list of zero-mean interleaved fields, iters, hist,
    K, f)."""
    shape = phase.shape
    c = n_comp(physics)
    K = fem.assemble_K(phase, props, physics, L0)
    P = preconditioner(precond, K, physics, props, shape, Q, L0)
    algo = _pcg.fcg_pr if flexible else _pcg.pcg
    us, its, hists, fs = [], [], [], []
    for load in np.atleast_2d(loads):
        f = fem.assemble_f(phase, props, physics, load, L0)
        u, it, hist = algo(lambda x: K @ x, f, P, tol, max_iter)
        us.append(zero_mean(u, c))
        its.append(it)
        hists.append(hist)
        fs.append(f)
    return dict(u=us, iters=its, hist=hists, K=K, f=fs)


def _D_per_element(phase, props, physics):
    props = np.asarray(props, dtype=np.float64)
    Ds = np.stack([fem.material_matrix(physics, props[p]) for p in range(props.shape[0])])
    return Ds[phase.ravel()]


def effective_tensor(phase, props, physics: int, us, loads, L0: float = 1.0) -> np.ndarray:
    """Averaged flux/stress per load: ``out[i, l] = <C (eps_bar_l + eps(u_l))>_i``.

    With the unit loads in order this is the effective tensor (row-major, Mandel for c=3).
    """
    shape = phase.shape
    D = _D_per_element(phase, props, physics)
    loads = np.atleast_2d(loads)
    out = np.zeros((D.shape[1], len(us)))
    for l, (u, load) in enumerate(zip(us, loads)):
        eps = fem.element_mean_strain(u, shape, physics, L0) + load[None, :]
        out[:, l] = np.einsum("eij,ej->i", D, eps) / D.shape[0]
    return out


def _gauss_strains(u, shape, physics, L0):
    """Strain (gradient) of u at the 8 Gauss points of every element: ``[n_elem, 8, dim]``."""
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    pts, _ = fem.gauss_points()
    ue = u[fem.element_dofs(shape, c)]
    return np.stack([ue @ (fem.b_matrix(physics, pts[q]) / h).T for q in range(8)], axis=1)


def energy_tensor(phase, props, physics: int, us, loads, L0: float = 1.0) -> np.ndarray:
    shape = phase.shape
    D = _D_per_element(phase, props, physics)
    loads = np.atleast_2d(loads)
    eps = [_gauss_strains(u, shape, physics, L0) + ld[None, None, :] for u, ld in zip(us, loads)]
    L = len(us)
    W = np.zeros((L, L))
    for a in range(L):
        for b in range(L):
            W[a, b] = np.einsum("eqi,eij,eqj->", eps[a], D, eps[b]) / (8.0 * D.shape[0])
    return W


def sensitivity(phase, props, physics: int, us, loads, L0: float = 1.0) -> np.ndarray:
    """``dW_lm / d prop``: thermal props ``kappa_p`` -> ``[n_phases, L, L]``; elastic props
    ``(E_p, nu_p)`` -> ``[2 n_phases, L, L]`` ordered ``E_0, nu_0, E_1, nu_1, ...``."""
    shape = phase.shape
    props = np.asarray(props, dtype=np.float64)
    loads = np.atleast_2d(loads)
    eps = [_gauss_strains(u, shape, physics, L0) + ld[None, None, :] for u, ld in zip(us, loads)]
    ph = phase.ravel()
    n = float(ph.size)
    L = len(us)
    n_ph = props.shape[0]
    if physics == 1:
        out = np.zeros((n_ph, L, L))
        for p in range(n_ph):
            sel = ph == p
            for a in range(L):
                for b in range(L):
                    out[p, a, b] = np.einsum("eqi,eqi->", eps[a][sel], eps[b][sel]) / (8.0 * n)
        return out
    m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    dD_dlam = np.outer(m, m)
    dD_dmu = 2.0 * np.eye(6)
    out = np.zeros((2 * n_ph, L, L))
    for p in range(n_ph):
        E, nu = props[p]
        dlam_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        dmu_dE = 1.0 / (2.0 * (1.0 + nu))
        dlam_dnu = E * (1.0 + 2.0 * nu * nu) / ((1.0 + nu) ** 2 * (1.0 - 2.0 * nu) ** 2)
        dmu_dnu = -E / (2.0 * (1.0 + nu) ** 2)
        sel = ph == p
        for a in range(L):
            for b in range(L):
                wl = np.einsum("eqi,ij,eqj->", eps[a][sel], dD_dlam, eps[b][sel]) / (8.0 * n)
                wm = np.einsum("eqi,ij,eqj->", eps[a][sel], dD_dmu, eps[b][sel]) / (8.0 * n)
                out[2 * p, a, b] = wl * dlam_dE + wm * dmu_dE
                out[2 * p + 1, a, b] = wl * dlam_dnu + wm * dmu_dnu
    return out


def direct_solve(K, f: np.ndarray, c: int) -> np.ndarray:
    """Dense bordered solve ``[[K, C^T], [C, 0]] [u; lam] = [f; 0]`` with ``C u = 0`` imposing a
    zero mean on every component (the null space of the periodic problem)."""
    Kd = K.toarray()
    ndof = Kd.shape[0]
    C = np.zeros((c, ndof))
    for j in range(c):
        C[j, j::c] = 1.0
    A = np.block([[Kd, C.T], [C, np.zeros((c, c))]])
    rhs = np.concatenate([f, np.zeros(c)])
    return np.linalg.solve(A, rhs)[:ndof]


def true_residual(K, u: np.ndarray, f: np.ndarray) -> float:
    """``||f - K u||_inf / ||f||_inf``."""
    fn = float(np.max(np.abs(f)))
    return float(np.max(np.abs(f - K @ u))) / fn if fn > 0 else 0.0
