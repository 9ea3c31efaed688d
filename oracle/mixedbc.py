"""Boundary conditions chosen per axis: periodic or Dirichlet (oracle; test infrastructure only).

Follows Sec. 4.1 (free nodes of a regular grid under periodic, Dirichlet or mixed BC, Fig.
(regular-grid)), Sec. 6.2 (mixed BC: the fluctuation periodic across the faces of some axes and
zero on the faces of the others) and Table (fnocg-mode-selection-2d): the unitary transform of
the UNO is the Fourier transform along the periodic axes composed with the sine transform along
the Dirichlet axes (the paper's FFT^x o DST^y), applied to every component.

Conventions
-----------
* ``bc``: three booleans, True = Dirichlet along that axis.
* Nodes per axis: N_a (periodic, node N_a is node 0) or N_a + 1 (Dirichlet, nodes 0 and N_a
  fixed); element ``i`` owns the nodes ``i + o``, ``o in {0,1}^3`` (mod N_a on periodic axes).
* Free nodes per axis: M_a = N_a (periodic) or N_a - 1 (Dirichlet, free index = node - 1);
  interleaved DOF ``c*free + comp``; SoA arrays ``[c, M1, M2, M3]``.
* Axis transforms (unitary): periodic ``F[k, j] = exp(-2 pi i j k / N) / sqrt(N)``; Dirichlet the
  orthonormal DST-I of ``oracle.dirichlet``.  ``P r = Re(T^H Q T r)`` with real symmetric blocks
  Q(k); on periodic axes the blocks must satisfy Q(-k) = Q(k) for a real output (conjugate
  modes), which ``symmetrize`` enforces.
* Reference weights: ``Q(k) = (t_k^H K_ref t_k)^{-1}`` with ``t_k`` the basis vector of mode k
  (the FANS fundamental solution when every axis is periodic, with Q(0) = 0 there; the reading
  of ``oracle.dirichlet`` otherwise).
* The fluctuation is projected to zero mean only when every axis is periodic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dirichlet as _dr, fem, pcg as _pcg


def n_comp(physics: int) -> int:
    return 1 if physics == 1 else 3


def free_shape(shape, bc):
    return tuple(int(n) - (1 if d else 0) for n, d in zip(shape, bc))


def _nodes_per_axis(shape, bc):
    return tuple(int(n) + (1 if d else 0) for n, d in zip(shape, bc))


def element_nodes(shape, bc) -> np.ndarray:
    """Node indices (of the full node grid) of the 8 corners of every element, (n_elem, 8)."""
    NN = _nodes_per_axis(shape, bc)
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    idx = [i.ravel() for i in idx]
    out = np.empty((idx[0].size, 8), dtype=np.int64)
    for a, o in enumerate(fem.CORNERS):
        x = [(idx[k] + o[k]) % shape[k] if not bc[k] else idx[k] + o[k] for k in range(3)]
        out[:, a] = (x[0] * NN[1] + x[1]) * NN[2] + x[2]
    return out


def free_nodes(shape, bc) -> np.ndarray:
    """Full-grid indices of the free nodes in the order of the free numbering."""
    NN = _nodes_per_axis(shape, bc)
    rng = [np.arange(1, n) if d else np.arange(n) for n, d in zip(shape, bc)]
    j = np.meshgrid(*rng, indexing="ij")
    return ((j[0] * NN[1] + j[1]) * NN[2] + j[2]).ravel()


def free_dofs(shape, bc, c: int) -> np.ndarray:
    fn = free_nodes(shape, bc)
    return (c * fn[:, None] + np.arange(c)[None, :]).ravel()


def _elem_dofs(shape, bc, c):
    en = element_nodes(shape, bc)
    return (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 8 * c)


def assemble_K(phase: np.ndarray, props, physics: int, bc, L0: float = 1.0) -> sp.csr_matrix:
    """Stiffness matrix of the free DOFs."""
    shape = phase.shape
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    props = np.asarray(props, dtype=np.float64)
    dofs = _elem_dofs(shape, bc, c)
    ph = phase.ravel()
    nd = 8 * c
    rows, cols, vals = [], [], []
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        Ke = fem.element_stiffness(physics, fem.material_matrix(physics, props[p]), h)
        dd = dofs[sel]
        rows.append(np.repeat(dd, nd, axis=1).ravel())
        cols.append(np.tile(dd, (1, nd)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (sel.size, nd * nd)).ravel())
    ndof = c * int(np.prod(_nodes_per_axis(shape, bc)))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    fd = free_dofs(shape, bc, c)
    return K[fd][:, fd].tocsr()


def assemble_f(phase: np.ndarray, props, physics: int, bc, load, L0: float = 1.0) -> np.ndarray:
    """``f = - sum_e A_e^T int_e B^T C eps_bar dV`` on the free DOFs (Sec. 6.1 / 6.2)."""
    shape = phase.shape
    c = n_comp(physics)
    h = fem.spacing(shape, L0)
    dofs = _elem_dofs(shape, bc, c)
    ph = phase.ravel()
    f = np.zeros(c * int(np.prod(_nodes_per_axis(shape, bc))))
    props = np.asarray(props, dtype=np.float64)
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        fe = fem.element_load(physics, fem.material_matrix(physics, props[p]), load, h)
        np.add.at(f, dofs[sel].ravel(), np.broadcast_to(fe, (sel.size, fe.size)).ravel())
    return f[free_dofs(shape, bc, c)]


def extend_to_full(u: np.ndarray, shape, bc, c: int) -> np.ndarray:
    full = np.zeros(c * int(np.prod(_nodes_per_axis(shape, bc))))
    full[free_dofs(shape, bc, c)] = u
    return full


def element_mean_strain(u: np.ndarray, shape, bc, physics: int, L0: float = 1.0) -> np.ndarray:
    c = n_comp(physics)
    Bm = fem.element_average_b(physics, fem.spacing(shape, L0))
    return extend_to_full(u, shape, bc, c)[_elem_dofs(shape, bc, c)] @ Bm.T


def effective_tensor(phase, props, physics: int, bc, us, loads, L0: float = 1.0) -> np.ndarray:
    props = np.asarray(props, dtype=np.float64)
    D = np.stack([fem.material_matrix(physics, props[p]) for p in range(props.shape[0])])[phase.ravel()]
    loads = np.atleast_2d(loads)
    out = np.zeros((D.shape[1], len(us)))
    for l, (u, load) in enumerate(zip(us, loads)):
        eps = element_mean_strain(u, phase.shape, bc, physics, L0) + load[None, :]
        out[:, l] = np.einsum("eij,ej->i", D, eps) / D.shape[0]
    return out


# ---------------------------------------------------------------- transforms

def axis_matrix(N: int, dirichlet: bool) -> np.ndarray:
    """Unitary transform of one axis: DST-I on the N - 1 interior points, or the DFT on N."""
    if dirichlet:
        return _dr.dst_matrix(N).astype(np.complex128)
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N) / np.sqrt(N)


def transform(x: np.ndarray, shape, bc, inverse: bool = False) -> np.ndarray:
    """T x (or T^H x) on the last three axes."""
    out = np.asarray(x, dtype=np.complex128)
    nd = out.ndim
    for a in range(3):
        A = axis_matrix(shape[a], bc[a])
        if inverse:
            A = A.conj().T
        out = np.moveaxis(np.tensordot(A, np.moveaxis(out, nd - 3 + a, 0), axes=(1, 0)), 0, nd - 3 + a)
    return out


def symmetrize(Q: np.ndarray, bc) -> np.ndarray:
    """Q(k) <- (Q(k) + Q(-k)) / 2 with -k taken on the periodic axes (conjugate modes)."""
    R = Q.copy()
    for a in range(3):
        if not bc[a]:
            R = np.flip(R, axis=a)
            R = np.roll(R, 1, axis=a)
    return 0.5 * (Q + R)


def uno_apply(Q: np.ndarray, r: np.ndarray, shape, bc) -> np.ndarray:
    """``s = Re(T^H Q T r)`` for SoA ``r [c, M1, M2, M3]`` and blocks ``Q [M1, M2, M3, c, c]``."""
    R = transform(r, shape, bc)
    S = np.einsum("xyzij,jxyz->ixyz", Q, R)
    s = transform(S, shape, bc, inverse=True)
    if np.max(np.abs(s.imag)) > 1e-10 * max(1.0, np.max(np.abs(s.real))):
        raise AssertionError("preconditioned residual is not real: Q(-k) != Q(k)?")
    return s.real


def transformed_blocks(physics: int, D: np.ndarray, shape, bc, L0: float = 1.0) -> np.ndarray:
    """``t_k^H K t_k`` of the homogeneous medium D for every mode: the stencil of a free node
    (27 offsets) against ``g_a(k, d) = sum_j conj(T[k, j]) T[k, j + d]`` per axis (periodic:
    j + d mod N; Dirichlet: both points inside).  Real for a symmetric stencil."""
    c = n_comp(physics)
    Ke = fem.element_stiffness(physics, D, fem.spacing(shape, L0))
    sten = np.zeros((3, 3, 3, c, c))
    for o in fem.CORNERS:
        ia = 4 * o[0] + 2 * o[1] + o[2]
        for ib, ob in enumerate(fem.CORNERS):
            d = ob - o
            sten[d[0] + 1, d[1] + 1, d[2] + 1] += Ke[c * ia:c * ia + c, c * ib:c * ib + c]
    g = []
    for N, dd in zip(shape, bc):
        T = axis_matrix(N, dd)
        M = T.shape[0]
        gd = np.zeros((M, 3), dtype=np.complex128)
        for di, d in enumerate((-1, 0, 1)):
            if dd:
                lo, hi = max(0, -d), min(M, M - d)
                gd[:, di] = np.sum(T[:, lo:hi].conj() * T[:, lo + d:hi + d], axis=1)
            else:
                gd[:, di] = np.sum(T.conj() * np.roll(T, -d, axis=1), axis=1)
        g.append(gd)
    B = np.einsum("xa,yb,zc,abcij->xyzij", g[0], g[1], g[2], sten)
    if np.max(np.abs(B.imag)) > 1e-12 * np.max(np.abs(B.real)):
        raise AssertionError("transformed stencil is not real")
    return B.real


def reference_Q(physics: int, props, shape, bc, L0: float = 1.0) -> np.ndarray:
    """``Q(k) = (t_k^H K_ref t_k)^{-1}``; Q(0) = 0 when every axis is periodic (null space)."""
    B = transformed_blocks(physics, _dr._ref_D(physics, props), shape, bc, L0)
    Q = np.zeros_like(B)
    flat_b, flat_q = B.reshape(-1, B.shape[-2], B.shape[-1]), Q.reshape(-1, B.shape[-2], B.shape[-1])
    start = 0 if any(bc) else 1
    flat_q[start:] = np.linalg.inv(flat_b[start:])
    return Q


def solve(phase, props, physics: int, bc, loads, precond: str = "uno", tol: float = 1e-8,
          max_iter: int = 100000, Q=None, L0: float = 1.0):
    """PCG (Algorithm 1 / 2) on the free DOFs for every load; dict(u, iters, hist, K, f)."""
    shape = phase.shape
    c = n_comp(physics)
    K = assemble_K(phase, props, physics, bc, L0)
    fs_ = free_shape(shape, bc)
    if precond == "none":
        P = lambda r: r.copy()
    elif precond == "jacobi":
        dg = K.diagonal()
        P = lambda r: r / dg
    elif precond == "uno":
        if Q is None:
            Q = reference_Q(physics, props, shape, bc, L0)
        P = lambda r: fem.from_soa(uno_apply(Q, fem.to_soa(r, c, fs_), shape, bc))
    else:
        raise ValueError(precond)
    us, its, hists, fs = [], [], [], []
    for load in np.atleast_2d(loads):
        f = assemble_f(phase, props, physics, bc, load, L0)
        u, it, hist = _pcg.pcg(lambda x: K @ x, f, P, tol, max_iter)
        if not any(bc):
            v = u.reshape(-1, c)
            u = (v - v.mean(axis=0, keepdims=True)).ravel()
        us.append(u)
        its.append(it)
        hists.append(hist)
        fs.append(f)
    return dict(u=us, iters=its, hist=hists, K=K, f=fs)
