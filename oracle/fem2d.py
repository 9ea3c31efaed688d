"""Two-dimensional problems on bilinear quadrilaterals (oracle; test infrastructure only).

Follows Sec. 4.1 (regular 2D grid, free nodes per BC, Fig. (regular-grid)), Sec. 6.1 (thermal,
c = 1) and Sec. 6.2 (linear elasticity under plane strain, c = 2, Mandel strains
[11, 22, sqrt2*12]) and Table (fnocg-mode-selection-2d) (Fourier transform along periodic
axes, sine transform along Dirichlet axes).  Square pixels of edge h = L0 / N1, 2x2 Gauss
quadrature (exact for bilinear elements); in 2D the element stiffness does not depend on h.

* ``bc``: two booleans, True = Dirichlet faces along that axis; node and free-index conventions
  as in ``oracle.mixedbc`` restricted to two axes; interleaved DOF ``c*free + comp``.
* Reference weights: ``Q(k) = (t_k^H K_ref t_k)^{-1}`` (FANS when both axes are periodic, Q(0) = 0).
* The fluctuation is projected to zero mean only when both axes are periodic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import dirichlet as _dr, fem, pcg as _pcg

CORNERS2 = np.array([[o1, o2] for o1 in (0, 1) for o2 in (0, 1)])
SQ2 = np.sqrt(2.0)


def n_comp(physics: int) -> int:
    return 1 if physics == 1 else 2


def material_matrix(physics: int, prop) -> np.ndarray:
    """kappa I2 (thermal) or the plane-strain Mandel stiffness lam m m^T + 2 mu I3 with
    m = [1, 1, 0] (elastic, (E, nu))."""
    if physics == 1:
        return float(prop) * np.eye(2)
    lam, mu = fem.lame(prop[0], prop[1])
    m = np.array([1.0, 1.0, 0.0])
    return lam * np.outer(m, m) + 2.0 * mu * np.eye(3)


def _shape_grads(xi):
    G = np.zeros((4, 2))
    for a, o in enumerate(CORNERS2):
        f = [xi[k] if o[k] else 1.0 - xi[k] for k in range(2)]
        s = [1.0 if o[k] else -1.0 for k in range(2)]
        G[a, 0] = s[0] * f[1]
        G[a, 1] = s[1] * f[0]
    return G


def b_matrix(physics: int, xi) -> np.ndarray:
    G = _shape_grads(xi)
    if physics == 1:
        return G.T.copy()
    B = np.zeros((3, 8))
    for a in range(4):
        B[0, 2 * a] = G[a, 0]
        B[1, 2 * a + 1] = G[a, 1]
        B[2, 2 * a] = G[a, 1] / SQ2
        B[2, 2 * a + 1] = G[a, 0] / SQ2
    return B


def gauss_points():
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    return np.array([[a, b] for a in g for b in g]), np.full(4, 0.25)


def element_stiffness(physics: int, D: np.ndarray) -> np.ndarray:
    """``int_e B^T D B dA`` with B in physical units: h^-1 B_xi and dA = h^2 dxi, so h cancels."""
    pts, w = gauss_points()
    nd = 4 * n_comp(physics)
    K = np.zeros((nd, nd))
    for q in range(4):
        B = b_matrix(physics, pts[q])
        K += w[q] * B.T @ D @ B
    return K


def element_load(physics: int, D: np.ndarray, load, h: float) -> np.ndarray:
    """``- int_e B^T D eps_bar dA = - h int_unit B_xi^T D eps_bar dxi``."""
    pts, w = gauss_points()
    f = np.zeros(4 * n_comp(physics))
    for q in range(4):
        f -= w[q] * b_matrix(physics, pts[q]).T @ (D @ np.asarray(load, dtype=np.float64))
    return h * f


def free_shape(shape, bc):
    return tuple(int(n) - (1 if d else 0) for n, d in zip(shape, bc))


def _nodes(shape, bc):
    return tuple(int(n) + (1 if d else 0) for n, d in zip(shape, bc))


def element_nodes(shape, bc) -> np.ndarray:
    NN = _nodes(shape, bc)
    i1, i2 = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    i1, i2 = i1.ravel(), i2.ravel()
    out = np.empty((i1.size, 4), dtype=np.int64)
    for a, o in enumerate(CORNERS2):
        x1 = i1 + o[0] if bc[0] else (i1 + o[0]) % shape[0]
        x2 = i2 + o[1] if bc[1] else (i2 + o[1]) % shape[1]
        out[:, a] = x1 * NN[1] + x2
    return out


def free_dofs(shape, bc, c: int) -> np.ndarray:
    NN = _nodes(shape, bc)
    r = [np.arange(1, n) if d else np.arange(n) for n, d in zip(shape, bc)]
    j1, j2 = np.meshgrid(r[0], r[1], indexing="ij")
    fn = (j1 * NN[1] + j2).ravel()
    return (c * fn[:, None] + np.arange(c)[None, :]).ravel()


def _edofs(shape, bc, c):
    en = element_nodes(shape, bc)
    return (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 4 * c)


def assemble_K(phase, props, physics: int, bc) -> sp.csr_matrix:
    shape = phase.shape
    c = n_comp(physics)
    props = np.asarray(props, dtype=np.float64)
    dofs = _edofs(shape, bc, c)
    nd = 4 * c
    rows, cols, vals = [], [], []
    for p in range(props.shape[0]):
        sel = np.nonzero(phase.ravel() == p)[0]
        if sel.size == 0:
            continue
        Ke = element_stiffness(physics, material_matrix(physics, props[p]))
        d = dofs[sel]
        rows.append(np.repeat(d, nd, axis=1).ravel())
        cols.append(np.tile(d, (1, nd)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (sel.size, nd * nd)).ravel())
    ndof = c * int(np.prod(_nodes(shape, bc)))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    fd = free_dofs(shape, bc, c)
    return K[fd][:, fd].tocsr()


def assemble_f(phase, props, physics: int, bc, load, L0: float = 1.0) -> np.ndarray:
    shape = phase.shape
    c = n_comp(physics)
    h = L0 / shape[0]
    dofs = _edofs(shape, bc, c)
    f = np.zeros(c * int(np.prod(_nodes(shape, bc))))
    props = np.asarray(props, dtype=np.float64)
    for p in range(props.shape[0]):
        sel = np.nonzero(phase.ravel() == p)[0]
        if sel.size == 0:
            continue
        fe = element_load(physics, material_matrix(physics, props[p]), load, h)
        np.add.at(f, dofs[sel].ravel(), np.broadcast_to(fe, (sel.size, fe.size)).ravel())
    return f[free_dofs(shape, bc, c)]


def effective_tensor(phase, props, physics: int, bc, us, loads, L0: float = 1.0) -> np.ndarray:
    """``out[i, l] = <C (eps_bar_l + eps(u_l))>_i`` with the element-mean gradient."""
    shape = phase.shape
    c = n_comp(physics)
    h = L0 / shape[0]
    pts, w = gauss_points()
    Bm = sum(w[q] * b_matrix(physics, pts[q]) for q in range(4)) / h
    props = np.asarray(props, dtype=np.float64)
    D = np.stack([material_matrix(physics, props[p]) for p in range(props.shape[0])])[phase.ravel()]
    out = np.zeros((D.shape[1], len(us)))
    for l, (u, load) in enumerate(zip(us, np.atleast_2d(loads))):
        full = np.zeros(c * int(np.prod(_nodes(shape, bc))))
        full[free_dofs(shape, bc, c)] = u
        eps = full[_edofs(shape, bc, c)] @ Bm.T + load[None, :]
        out[:, l] = np.einsum("eij,ej->i", D, eps) / D.shape[0]
    return out


def axis_matrix(N: int, dirichlet: bool) -> np.ndarray:
    if dirichlet:
        return _dr.dst_matrix(N).astype(np.complex128)
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N) / np.sqrt(N)


def transform(x, shape, bc, inverse=False):
    out = np.asarray(x, dtype=np.complex128)
    nd = out.ndim
    for a in range(2):
        A = axis_matrix(shape[a], bc[a])
        if inverse:
            A = A.conj().T
        out = np.moveaxis(np.tensordot(A, np.moveaxis(out, nd - 2 + a, 0), axes=(1, 0)), 0, nd - 2 + a)
    return out


def uno_apply(Q, r, shape, bc):
    """``Re(T^H Q T r)`` for SoA ``r [c, M1, M2]`` and blocks ``Q [M1, M2, c, c]``."""
    R = transform(r, shape, bc)
    s = transform(np.einsum("xyij,jxy->ixy", Q, R), shape, bc, inverse=True)
    if np.max(np.abs(s.imag)) > 1e-10 * max(1.0, np.max(np.abs(s.real))):
        raise AssertionError("preconditioned residual is not real")
    return s.real


def reference_Q(physics: int, props, shape, bc) -> np.ndarray:
    """``(t_k^H K_ref t_k)^{-1}`` of the arithmetic-mean medium, by the stencil of a free node."""
    props = np.asarray(props, dtype=np.float64)
    if physics == 1:
        D = float(np.mean(props)) * np.eye(2)
    else:
        lm = np.array([fem.lame(E, nu) for (E, nu) in props])
        lam, mu = lm[:, 0].mean(), lm[:, 1].mean()
        m = np.array([1.0, 1.0, 0.0])
        D = lam * np.outer(m, m) + 2.0 * mu * np.eye(3)
    c = n_comp(physics)
    Ke = element_stiffness(physics, D)
    sten = np.zeros((3, 3, c, c))
    for ia, o in enumerate(CORNERS2):
        for ib, ob in enumerate(CORNERS2):
            d = ob - o
            sten[d[0] + 1, d[1] + 1] += Ke[c * ia:c * ia + c, c * ib:c * ib + c]
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
    B = np.einsum("xa,yb,abij->xyij", g[0], g[1], sten).real
    Q = np.zeros_like(B)
    fb, fq = B.reshape(-1, c, c), Q.reshape(-1, c, c)
    start = 0 if any(bc) else 1
    fq[start:] = np.linalg.inv(fb[start:])
    return Q


def solve(phase, props, physics: int, bc, loads, precond: str = "uno", tol: float = 1e-8,
          max_iter: int = 100000, Q=None):
    """PCG (Algorithm 1) for every load; ``precond="uno"`` with the blocks ``Q [M1, M2, c, c]``
    (default: the reference medium, ``reference_Q``)."""
    shape = phase.shape
    c = n_comp(physics)
    K = assemble_K(phase, props, physics, bc)
    fs_ = free_shape(shape, bc)
    if precond == "uno":
        if Q is None:
            Q = reference_Q(physics, props, shape, bc)
        to_soa = lambda v: v.reshape(fs_ + (c,)).transpose(2, 0, 1)
        from_soa = lambda a: np.ascontiguousarray(a.transpose(1, 2, 0)).ravel()
        P = lambda r: from_soa(uno_apply(Q, to_soa(r), shape, bc))
    elif precond == "jacobi":
        dg = K.diagonal()
        P = lambda r: r / dg
    else:
        P = lambda r: r.copy()
    us, its = [], []
    for load in np.atleast_2d(loads):
        f = assemble_f(phase, props, physics, bc, load)
        u, it, _ = _pcg.pcg(lambda x: K @ x, f, P, tol, max_iter)
        if not any(bc):
            v = u.reshape(-1, c)
            u = (v - v.mean(axis=0, keepdims=True)).ravel()
        us.append(u)
        its.append(it)
    return dict(u=us, iters=its, K=K)
