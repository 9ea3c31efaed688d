"""Finite elements on a regular periodic voxel grid (oracle; test infrastructure only).

Follows Sec. 4.1 (Galerkin FE on a regular grid, periodic BC: n = N1*N2*N3 free nodes) and
the problem statements of Sec. 6.1 (Fourier's law, q = -kappa grad(theta)) and Sec. 6.2
(linear elasticity, C = 3 lambda P1 + 2 mu I^s, Mandel notation of App. A).

Conventions
-----------
* Node ``(i1, i2, i3)``, ``0 <= i_a < N_a``; flat node index ``(i1*N2 + i2)*N3 + i3``.
* Element (voxel) ``e = (i1, i2, i3)`` owns the 8 nodes ``((i + o) mod N)``, ``o in {0,1}^3``,
  local corner index ``4*o1 + 2*o2 + o3``.
* Grid spacing ``h = L0 / N`` (cubic voxels; ``L0`` the RVE edge along axis 1).
* DOF vector in the paper's interleaved order (Sec. 2.1 "Notation"): ``dof = c*node + comp``.
* Mandel order (App. A): ``[11, 22, 33, sqrt2*12, sqrt2*13, sqrt2*23]``.
* Elements are integrated with 2x2x2 Gauss quadrature, exact for trilinear bricks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

SQ2 = np.sqrt(2.0)
CORNERS = np.array([[o1, o2, o3] for o1 in (0, 1) for o2 in (0, 1) for o3 in (0, 1)])


def gauss_points():
    """2x2x2 Gauss-Legendre points and weights on the unit cube."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    pts = np.array([[a, b, c] for a in g for b in g for c in g])
    w = np.full(8, 1.0 / 8.0)
    return pts, w


def shape_values(xi):
    """Trilinear shape functions of the 8 corners at ``xi`` in the unit cube."""
    v = np.ones(8)
    for a in range(3):
        v *= np.where(CORNERS[:, a] == 1, xi[a], 1.0 - xi[a])
    return v


def shape_grads(xi):
    """Gradients (w.r.t. unit-cube coordinates) of the 8 shape functions: shape (8, 3)."""
    G = np.ones((8, 3))
    for a in range(3):
        for b in range(3):
            if a == b:
                G[:, a] *= np.where(CORNERS[:, b] == 1, 1.0, -1.0)
            else:
                G[:, a] *= np.where(CORNERS[:, b] == 1, xi[b], 1.0 - xi[b])
    return G


def b_matrix(physics: int, xi) -> np.ndarray:
    """Strain-displacement matrix on the unit cube.

    thermal (c=1): gradient, shape (3, 8);  elastic (c=3): Mandel strain, shape (6, 24)
    with element DOF order ``3*corner + comp``.
    """
    G = shape_grads(xi)
    if physics == 1:
        return G.T.copy()
    B = np.zeros((6, 24))
    for a in range(8):
        g = G[a]
        B[0, 3 * a + 0] = g[0]
        B[1, 3 * a + 1] = g[1]
        B[2, 3 * a + 2] = g[2]
        # sqrt2 * eps12 = (d2 u1 + d1 u2) / sqrt2, etc.
        B[3, 3 * a + 0] = g[1] / SQ2
        B[3, 3 * a + 1] = g[0] / SQ2
        B[4, 3 * a + 0] = g[2] / SQ2
        B[4, 3 * a + 2] = g[0] / SQ2
        B[5, 3 * a + 1] = g[2] / SQ2
        B[5, 3 * a + 2] = g[1] / SQ2
    return B


def lame(E, nu):
    """Lame constants of an isotropic material from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def material_matrix(physics: int, prop) -> np.ndarray:
    """Material tangent: ``kappa * I3`` (thermal) or Mandel ``3 lam P1 + 2 mu I^s`` (elastic)."""
    if physics == 1:
        return float(prop) * np.eye(3)
    lam, mu = lame(prop[0], prop[1])
    m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    # 3 P1 = m m^T in Mandel notation, I^s = identity
    return lam * np.outer(m, m) + 2.0 * mu * np.eye(6)


def element_stiffness(physics: int, D: np.ndarray, h: float) -> np.ndarray:
    """``K_e = int_e B^T D B dV = h * int_unit B_xi^T D B_xi dxi`` by Gauss quadrature."""
    pts, w = gauss_points()
    nd = 8 if physics == 1 else 24
    K = np.zeros((nd, nd))
    for q in range(8):
        B = b_matrix(physics, pts[q])
        K += w[q] * B.T @ D @ B
    return h * K


def element_load(physics: int, D: np.ndarray, load, h: float) -> np.ndarray:
    """``f_e = - int_e B^T D eps_bar dV = - h^2 int_unit B_xi^T D eps_bar dxi``."""
    pts, w = gauss_points()
    nd = 8 if physics == 1 else 24
    f = np.zeros(nd)
    for q in range(8):
        B = b_matrix(physics, pts[q])
        f -= w[q] * B.T @ (D @ np.asarray(load, dtype=np.float64))
    return h * h * f


def element_average_b(physics: int, h: float) -> np.ndarray:
    """Element average of the physical B matrix: ``(1/h^3) int_e B dV = (1/h) int_unit B_xi``."""
    pts, w = gauss_points()
    Bm = sum(w[q] * b_matrix(physics, pts[q]) for q in range(8))
    return Bm / h


def element_nodes(shape) -> np.ndarray:
    """Node indices of the 8 corners of every element: shape (n_elem, 8)."""
    N1, N2, N3 = shape
    i1, i2, i3 = np.meshgrid(np.arange(N1), np.arange(N2), np.arange(N3), indexing="ij")
    i1, i2, i3 = i1.ravel(), i2.ravel(), i3.ravel()
    out = np.empty((i1.size, 8), dtype=np.int64)
    for a, (o1, o2, o3) in enumerate(CORNERS):
        out[:, a] = (((i1 + o1) % N1) * N2 + (i2 + o2) % N2) * N3 + (i3 + o3) % N3
    return out


def element_dofs(shape, c: int) -> np.ndarray:
    """Interleaved DOF indices of every element, ``c*node + comp``: shape (n_elem, 8c)."""
    en = element_nodes(shape)
    if c == 1:
        return en
    return (c * en[:, :, None] + np.arange(c)[None, None, :]).reshape(en.shape[0], 8 * c)


def spacing(shape, L0: float = 1.0) -> float:
    return L0 / shape[0]


def assemble_K(phase: np.ndarray, props, physics: int, L0: float = 1.0) -> sp.csr_matrix:
    """Assembled periodic stiffness matrix (Eq. (fem-linear-system)), interleaved DOFs."""
    shape = phase.shape
    c = 1 if physics == 1 else 3
    h = spacing(shape, L0)
    props = np.asarray(props, dtype=np.float64)
    dofs = element_dofs(shape, c)
    ph = phase.ravel()
    nd = 8 * c
    rows, cols, vals = [], [], []
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        Ke = element_stiffness(physics, material_matrix(physics, props[p]), h)
        d = dofs[sel]
        rows.append(np.repeat(d, nd, axis=1).ravel())
        cols.append(np.tile(d, (1, nd)).ravel())
        vals.append(np.broadcast_to(Ke.ravel(), (sel.size, nd * nd)).ravel())
    ndof = c * int(np.prod(shape))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(ndof, ndof)).tocsr()
    K.sum_duplicates()
    return K


def assemble_f(phase: np.ndarray, props, physics: int, load, L0: float = 1.0) -> np.ndarray:
    """Right-hand side of the fluctuation problem for one macroscopic load.

    Thermal (Sec. 6.1): with theta = theta_bar + g_bar.x + theta_tilde, the weak form of
    div(kappa (g_bar + grad theta_tilde)) = 0 gives K theta_tilde = f with
    ``f = - sum_e A_e^T int_e grad(N)^T kappa g_bar dV``; elastic (Sec. 6.2) likewise with
    ``f = - sum_e A_e^T int_e B^T C eps_bar dV`` (eps_bar in Mandel notation).
    """
    shape = phase.shape
    c = 1 if physics == 1 else 3
    h = spacing(shape, L0)
    dofs = element_dofs(shape, c)
    ph = phase.ravel()
    f = np.zeros(c * int(np.prod(shape)))
    props = np.asarray(props, dtype=np.float64)
    for p in range(props.shape[0]):
        sel = np.nonzero(ph == p)[0]
        if sel.size == 0:
            continue
        fe = element_load(physics, material_matrix(physics, props[p]), load, h)
        np.add.at(f, dofs[sel].ravel(), np.broadcast_to(fe, (sel.size, fe.size)).ravel())
    return f


def element_mean_strain(u: np.ndarray, shape, physics: int, L0: float = 1.0) -> np.ndarray:
    """Element-averaged gradient (thermal, (n_elem, 3)) or Mandel strain (elastic, (n_elem, 6))."""
    c = 1 if physics == 1 else 3
    h = spacing(shape, L0)
    Bm = element_average_b(physics, h)
    ue = u[element_dofs(shape, c)]
    return ue @ Bm.T


def to_soa(u: np.ndarray, c: int, shape) -> np.ndarray:
    """Interleaved DOF vector -> array ``[c, N1, N2, N3]``."""
    return u.reshape(tuple(shape) + (c,)).transpose(3, 0, 1, 2).copy()


def from_soa(a: np.ndarray) -> np.ndarray:
    """Array ``[c, N1, N2, N3]`` -> interleaved DOF vector."""
    return np.ascontiguousarray(a.transpose(1, 2, 3, 0)).ravel()


def residual_at_nodes(phase: np.ndarray, props, physics: int, u: np.ndarray, load, nodes,
                      L0: float = 1.0) -> np.ndarray:
    """``(f - K u)`` at the listed nodes ``[(i1, i2, i3), ...]``, one node at a time from the
    element matrices of the (up to) 8 elements around it; no global assembly (for full-size
    spot checks).  ``u`` interleaved; returns ``[len(nodes), c]``."""
    shape = phase.shape
    c = 1 if physics == 1 else 3
    h = spacing(shape, L0)
    props = np.asarray(props, dtype=np.float64)
    Ks = [element_stiffness(physics, material_matrix(physics, props[p]), h) for p in range(props.shape[0])]
    fs = [element_load(physics, material_matrix(physics, props[p]), load, h) for p in range(props.shape[0])]
    N = np.asarray(shape)
    out = np.zeros((len(nodes), c))
    for q, node in enumerate(nodes):
        node = np.asarray(node)
        for a, o in enumerate(CORNERS):  # element e = node - o holds the node as corner a
            e = (node - o) % N
            p = phase[tuple(e)]
            idx = []
            for ob in CORNERS:
                nb = (e + ob) % N
                flat = (nb[0] * shape[1] + nb[1]) * shape[2] + nb[2]
                idx.extend([c * flat + j for j in range(c)])
            ue = u[np.array(idx)]
            rows = slice(c * a, c * a + c)
            out[q] += fs[p][rows] - Ks[p][rows] @ ue
    return out
