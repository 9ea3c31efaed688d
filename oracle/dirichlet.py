"""Dirichlet boundary conditions with the sine transform (oracle; test infrastructure only).

Follows Sec. 4.1 (regular grid of N1 x N2 x N3 voxels with (N1+1)(N2+1)(N3+1) nodes; with
Dirichlet BC on every face only the (N1-1)(N2-1)(N3-1) interior nodes are free), Sec. 6.1 and
6.2 (the fluctuation vanishes on the boundary: kinematic uniform boundary conditions), and the
Dirichlet row of Table (fnocg-mode-selection-2d): the unitary transform of the UNO
preconditioner is the sine transform, real, with no conjugate modes.

Conventions
-----------
* Full-grid node ``(i1, i2, i3)``, ``0 <= i_a <= N_a``; element ``e = (i1, i2, i3)``,
  ``i_a < N_a``, owns the nodes ``i + o``, ``o in {0,1}^3`` (no wrap).
* Free node ``j = i - 1``, ``0 <= j_a < M_a = N_a - 1``; interleaved DOF ``c*free + comp``;
  SoA arrays ``[c, M1, M2, M3]``.
* Sine transform: ``S[k, j] = sqrt(2/N) sin(pi (j+1) (k+1) / N)`` for ``j, k < N - 1``, the
  orthonormal DST-I (symmetric, its own inverse); 3D: ``T = S1 x S2 x S3`` on every component.
* Reference weights (a reading; FANS does not exist for Dirichlet BC): ``Q(k)`` is the inverse
  of the c x c block ``t_k^T K_ref t_k`` of the transformed homogeneous operator at the mode k
  (``t_k`` the sine basis vector).  The sine transform diagonalizes every product of 1D
  stiffness and mass matrices, so for c = 1 this is the exact inverse of the homogeneous
  operator; for c = 3 the couplings of different components are products with the
  antisymmetric first-difference matrix, whose diagonal in the sine basis vanishes.
* No zero-mean projection: with Dirichlet BC the fluctuation is unique.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem, pcg as _pcg


def n_comp(physics: int) -> int:
    return 1 if physics == 1 else 3


def free_shape(shape):
    return tuple(int(n) - 1 for n in shape)


def full_element_nodes(shape) -> np.ndarray:
    """Full-grid node indices of the 8 corners of every element, (n_elem, 8)."""
    N1, N2, N3 = shape
    i1, i2, i3 = np.meshgrid(np.arange(N1), np.arange(N2), np.arange(N3), indexing="ij")
    i1, i2, i3 = i1.ravel(), i2.ravel(), i3.ravel()
    out = np.empty((i1.size, 8), dtype=np.int64)
    for a, (o1, o2, o3) in enumerate(fem.CORNERS):
        out[:, a] = ((i1 + o1) * (N2 + 1) + (i2 + o2)) * (N3 + 1) + (i3 + o3)
    return out


def free_nodes(shape) -> np.ndarray:
    """Full-grid indices of the free (interior) nodes in the order of the free numbering."""
    N1, N2, N3 = shape
    j1, j2, j3 = np.meshgrid(np.arange(1, N1), np.arange(1, N2), np.arange(1, N3), indexing="ij")
    return ((j1 * (N2 + 1) + j2) * (N3 + 1) + j3).ravel()


def free_dofs(shape, c: int) -> np.ndarray:
    fn = free_nodes(shape)
    return (c * fn[:, None] + np.arange(c)[None, :]).ravel()


def assemble_K_full(phase: np.ndarray, props, physics: int, L0: float = 1.0) -> sp.csr_matrix:
    """Stiffness matrix of all (N1+1)(N2+1)(N3+1) nodes (no boundary conditions)."""
    shape = phase.shape
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    props = np.asarray(props, dtype=np.float64)
    en = full_element_nodes(shape)
    dofs = (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 8 * c)
    ph = phase.ravel()
    nd = 8 * c
    rows, cols, vals = [], [], []
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        Ke = fem.element_stiffness(physics, fem.material_matrix(physics, props[p]), h)
        d = dofs[sel]
        rows.append(np.repeat(d, nd, axis=1).ravel())
        cols.append(np.tile(d, (1, nd)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (sel.size, nd * nd)).ravel())
    ndof = c * int(np.prod(np.asarray(shape) + 1))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    return K


def assemble_K(phase: np.ndarray, props, physics: int, L0: float = 1.0) -> sp.csr_matrix:
    """Stiffness matrix of the free DOFs (rows and columns of the boundary nodes removed)."""
    fd = free_dofs(phase.shape, n_comp(physics))
    return assemble_K_full(phase, props, physics, L0)[fd][:, fd].tocsr()


def assemble_f(phase: np.ndarray, props, physics: int, load, L0: float = 1.0) -> np.ndarray:
    """Right-hand side on the free DOFs: ``f = - sum_e A_e^T int_e B^T C eps_bar dV`` (the same
    element loads as for periodic BC, Sec. 6.1 / 6.2), kept at the interior nodes; with the
    fluctuation zero on the boundary no boundary term enters."""
    shape = phase.shape
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    en = full_element_nodes(shape)
    dofs = (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 8 * c)
    ph = phase.ravel()
    f = np.zeros(c * int(np.prod(np.asarray(shape) + 1)))
    props = np.asarray(props, dtype=np.float64)
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        fe = fem.element_load(physics, fem.material_matrix(physics, props[p]), load, h)
        np.add.at(f, dofs[sel].ravel(), np.broadcast_to(fe, (sel.size, fe.size)).ravel())
    return f[free_dofs(shape, c)]


def extend_to_full(u: np.ndarray, shape, c: int) -> np.ndarray:
    """Free-DOF vector -> full-grid vector with zeros on the boundary nodes."""
    full = np.zeros(c * int(np.prod(np.asarray(shape) + 1)))
    full[free_dofs(shape, c)] = u
    return full


def element_mean_strain(u: np.ndarray, shape, physics: int, L0: float = 1.0) -> np.ndarray:
    """Element-averaged gradient / Mandel strain of a free-DOF field (zero on the boundary)."""
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    Bm = fem.element_average_b(physics, h)
    en = full_element_nodes(shape)
    dofs = (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 8 * c)
    return extend_to_full(u, shape, c)[dofs] @ Bm.T


def effective_tensor(phase, props, physics: int, us, loads, L0: float = 1.0) -> np.ndarray:
    """Averaged flux / stress per load, ``out[i, l] = <C (eps_bar_l + eps(u_l))>_i``."""
    props = np.asarray(props, dtype=np.float64)
    D = np.stack([fem.material_matrix(physics, props[p]) for p in range(props.shape[0])])[phase.ravel()]
    loads = np.atleast_2d(loads)
    out = np.zeros((D.shape[1], len(us)))
    for l, (u, load) in enumerate(zip(us, loads)):
        eps = element_mean_strain(u, phase.shape, physics, L0) + load[None, :]
        out[:, l] = np.einsum("eij,ej->i", D, eps) / D.shape[0]
    return out


# ---------------------------------------------------------------- sine transform

def dst_matrix(N: int) -> np.ndarray:
    """Orthonormal DST-I on the N - 1 interior points of an axis with N voxels."""
    j = np.arange(1, N)
    return np.sqrt(2.0 / N) * np.sin(np.pi * np.outer(j, j) / N)


def _along(x: np.ndarray, S: np.ndarray, axis: int) -> np.ndarray:
    return np.moveaxis(np.tensordot(S, np.moveaxis(x, axis, 0), axes=(1, 0)), 0, axis)


def dst3(x: np.ndarray) -> np.ndarray:
    """T x on the last three axes (``[..., M1, M2, M3]``); T is its own inverse."""
    out = np.asarray(x, dtype=np.float64)
    nd = out.ndim
    for a in range(3):
        out = _along(out, dst_matrix(out.shape[nd - 3 + a] + 1), nd - 3 + a)
    return out


def uno_apply(Q: np.ndarray, r: np.ndarray) -> np.ndarray:
    """``s = T^T Q T r`` for SoA ``r [c, M1, M2, M3]`` and blocks ``Q [M1, M2, M3, c, c]``."""
    R = dst3(r)
    S = np.einsum("xyzij,jxyz->ixyz", Q, R)
    return dst3(S)


# ---------------------------------------------------------------- reference weights

def _ref_D(physics: int, props):
    """Material matrix of the reference medium: the arithmetic mean over the phases of kappa,
    or of the Lame constants (the reading used for periodic BC)."""
    props = np.asarray(props, dtype=np.float64)
    if physics == 1:
        return float(np.mean(props)) * np.eye(3)
    lm = np.array([fem.lame(E, nu) for (E, nu) in props])
    lam, mu = lm[:, 0].mean(), lm[:, 1].mean()
    m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    return lam * np.outer(m, m) + 2.0 * mu * np.eye(6)


def transformed_blocks(physics: int, D: np.ndarray, shape, L0: float = 1.0) -> np.ndarray:
    """``t_k^T K t_k`` for every mode k and component pair of the homogeneous medium D:
    ``[M1, M2, M3, c, c]``.  K is the interior stencil (27 offsets d, coefficients from the 8
    element matrices around a node), so ``t_k^T K_ab t_k = sum_d k_ab(d) prod_a g_a(k_a, d_a)``
    with ``g(k, d) = sum_j S[k, j] S[k, j + d]`` over the j with both points inside."""
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    Ke = fem.element_stiffness(physics, D, h)
    # stencil of an interior node: row (node, a) of K against column (node + d, b)
    sten = np.zeros((3, 3, 3, c, c))
    for o in fem.CORNERS:          # the element whose local corner o is the node
        ia = 4 * o[0] + 2 * o[1] + o[2]
        for ib, ob in enumerate(fem.CORNERS):
            d = ob - o
            sten[d[0] + 1, d[1] + 1, d[2] + 1] += Ke[c * ia:c * ia + c, c * ib:c * ib + c]
    g = []
    for N in shape:
        S = dst_matrix(N)
        gd = np.zeros((N - 1, 3))
        for di, d in enumerate((-1, 0, 1)):
            lo, hi = max(0, -d), min(N - 1, N - 1 - d)
            gd[:, di] = np.sum(S[:, lo:hi] * S[:, lo + d:hi + d], axis=1)
        g.append(gd)
    out = np.einsum("xa,yb,zc,abcij->xyzij", g[0], g[1], g[2], sten)
    return out


def reference_Q(physics: int, props, shape, L0: float = 1.0) -> np.ndarray:
    """Reference weights ``Q(k) = (t_k^T K_ref t_k)^{-1}``, ``[M1, M2, M3, c, c]``."""
    B = transformed_blocks(physics, _ref_D(physics, props), shape, L0)
    return np.linalg.inv(B)


def mode_list(M: int):
    """Modes of the Dirichlet set [0, 2M]^3 (Table (fnocg-mode-selection-2d)), k1 slowest; mode
    index k_a is the sine basis vector of frequency k_a + 1."""
    K = 2 * M + 1
    return [(k1, k2, k3) for k1 in range(K) for k2 in range(K) for k3 in range(K)]


def modes_Q(w: np.ndarray, M: int, shape, c: int) -> np.ndarray:
    """Blocks ``[M1, M2, M3, c, c]`` of the paper's layout for Dirichlet BC: the bypass
    ``psi(w[0])`` on every mode plus ``psi(w[1 + i])`` on the i-th mode of [0, 2M]^3
    (Eq. (fnocg-parametrization); no conjugate modes for the sine transform)."""
    from . import uno
    w = np.asarray(w, dtype=np.float64)
    modes = mode_list(M)
    if w.shape != (1 + len(modes), uno.n_unique(c)):
        raise ValueError("weights must be [1 + n_modes, C]")
    Ms = free_shape(shape)
    if any(2 * M + 1 > m for m in Ms):
        raise ValueError("mode set larger than the free grid")
    Q = np.broadcast_to(uno.psi(w[0], c), Ms + (c, c)).copy()
    for i, (k1, k2, k3) in enumerate(modes):
        Q[k1, k2, k3] += uno.psi(w[1 + i], c)
    return Q


# ---------------------------------------------------------------- solves

def solve(phase, props, physics: int, loads, precond: str = "uno", tol: float = 1e-8,
          max_iter: int = 100000, Q=None, flexible: bool = False, L0: float = 1.0):
    """PCG (Algorithm 1 / 2) on the free DOFs for every load; returns dict(u, iters, hist, K, f)
    with interleaved free-DOF fields."""
    shape = phase.shape
    c = n_comp(physics)
    K = assemble_K(phase, props, physics, L0)
    fs_ = free_shape(shape)
    if precond == "none":
        P = lambda r: r.copy()
    elif precond == "jacobi":
        dg = K.diagonal()
        P = lambda r: r / dg
    elif precond == "uno":
        if Q is None:
            Q = reference_Q(physics, props, shape, L0)
        P = lambda r: fem.from_soa(uno_apply(Q, fem.to_soa(r, c, fs_)))
    else:
        raise ValueError(precond)
    algo = _pcg.fcg_pr if flexible else _pcg.pcg
    us, its, hists, fs = [], [], [], []
    for load in np.atleast_2d(loads):
        f = assemble_f(phase, props, physics, load, L0)
        u, it, hist = algo(lambda x: K @ x, f, P, tol, max_iter)
        us.append(u)
        its.append(it)
        hists.append(hist)
        fs.append(f)
    return dict(u=us, iters=its, hist=hists, K=K, f=fs)
