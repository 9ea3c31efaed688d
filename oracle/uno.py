"""UNO preconditioner by definition (oracle; test infrastructure only).

* Operator: ``s = T^{-1}( Phi(k) T r )`` with a real symmetric c x c block ``Phi(k)`` per
  frequency, Eq. (fnocg-op-fundsol); algebraically ``P = T^H Q T`` with the block-diagonal-in-
  frequency matrix Q, Eq. (FNOCG-prec-fields-disc) / Eq. (prec-sparse-def).
* Local SPD parametrization psi (Sec. 5.2.2): ``psi(w) = w^2`` for c = 1 and the
  Cholesky-like ``L L^T`` of Eq. (local-param-3) (App. B.1) for c = 3.
* Storage of the unique block entries in the paper's order (App. B.2):
  ``v1 = Q11, v2 = Q22, v3 = Q12, v4 = Q33, v5 = Q23, v6 = Q13``.
* FANS reference-medium fundamental solution (Sec. 4.3.4): ``Q(k) = S_ref(k)^{-1}`` where
  ``S_ref(k)`` is the Fourier symbol of the stiffness matrix of a homogeneous reference
  medium, obtained here by transforming the assembled stencil (a column of K_ref);
  ``Q(0) = 0`` on the null space of the periodic problem (Remark after Algorithm 2).
* Safety check of the Remark after Algorithm 2: ``lambda_min(Q(k)) > eps`` for all k != 0.
* The paper's own weight layout (Eq. (fnocg-operator), Eq. (fnocg-parametrization)): an inner
  bypass ``W = psi(w_0)`` acting on every mode plus a kernel ``psi(w_i)`` on the modes of a
  set ``K_M = [-M, M]^2 x [0, M] minus {0}`` (periodic row of Table (fnocg-mode-selection-2d)),
  zero elsewhere; the conjugate modes (negative k3) are the Hermitian half of the spectrum.
"""
from __future__ import annotations

import numpy as np

from . import dft, fem

PAPER_ORDER = [(0, 0), (1, 1), (0, 1), (2, 2), (1, 2), (0, 2)]  # v1..v6


def n_unique(c: int) -> int:
    return c * (c + 1) // 2


def psi(theta: np.ndarray, c: int) -> np.ndarray:
    """Local parametrization: ``theta[..., C] -> SPD blocks [..., c, c]``."""
    theta = np.asarray(theta, dtype=np.float64)
    if c == 1:
        return (theta[..., 0] ** 2)[..., None, None]
    t1, t2, t3, t4, t5, t6 = (theta[..., i] for i in range(6))
    L = np.zeros(theta.shape[:-1] + (3, 3))
    L[..., 0, 0] = t1
    L[..., 1, 0] = t3
    L[..., 1, 1] = t2
    L[..., 2, 0] = t6
    L[..., 2, 1] = t5
    L[..., 2, 2] = t4
    return L @ np.swapaxes(L, -1, -2)


def entries_from_blocks(Q: np.ndarray) -> np.ndarray:
    """Blocks ``[..., c, c]`` -> unique entries ``[..., C]`` in the paper's order."""
    c = Q.shape[-1]
    if c == 1:
        return Q[..., 0, :].copy()
    return np.stack([Q[..., i, j] for (i, j) in PAPER_ORDER], axis=-1)


def blocks_from_entries(v: np.ndarray, c: int) -> np.ndarray:
    """Unique entries ``[..., C]`` in the paper's order -> symmetric blocks ``[..., c, c]``."""
    v = np.asarray(v, dtype=np.float64)
    if c == 1:
        return v[..., None]
    Q = np.zeros(v.shape[:-1] + (3, 3))
    for m, (i, j) in enumerate(PAPER_ORDER):
        Q[..., i, j] = v[..., m]
        Q[..., j, i] = v[..., m]
    return Q


def reference_props(physics: int, props):
    """Reference medium: arithmetic mean over the phases of kappa, or of the Lame constants."""
    props = np.asarray(props, dtype=np.float64)
    if physics == 1:
        return float(np.mean(props))
    lm = np.array([fem.lame(E, nu) for (E, nu) in props])
    return float(np.mean(lm[:, 0])), float(np.mean(lm[:, 1]))


def _reference_D(physics: int, ref):
    if physics == 1:
        return ref * np.eye(3)
    lam, mu = ref
    m = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    return lam * np.outer(m, m) + 2.0 * mu * np.eye(6)


def stencil_kernel(physics: int, ref, shape, L0: float = 1.0) -> np.ndarray:
    """Column of the homogeneous stiffness matrix at node 0: ``k[i, j, x] = K[(x,i), (0,j)]``.

    Gathered from the 8 elements that contain node 0 (periodic wrap), shape ``[c, c, N1,N2,N3]``.
    """
    c = 1 if physics == 1 else 3
    h = fem.spacing(shape, L0)
    Ke = fem.element_stiffness(physics, _reference_D(physics, ref), h)
    k = np.zeros((c, c) + tuple(shape))
    N = np.asarray(shape)
    for o in fem.CORNERS:  # element e = -o contains node 0 as its local corner o
        a0 = 4 * o[0] + 2 * o[1] + o[2]
        for b, ob in enumerate(fem.CORNERS):
            x = (ob - o) % N  # node of local corner b
            for i in range(c):
                for j in range(c):
                    k[i, j, x[0], x[1], x[2]] += Ke[c * b + i, c * a0 + j]
    return k


def reference_symbol(physics: int, ref, shape, L0: float = 1.0) -> np.ndarray:
    """Fourier symbol ``S(k) = sum_x k(x) exp(-2 pi i k.x/N)`` on the half grid, ``[..., c, c]``."""
    k = stencil_kernel(physics, ref, shape, L0)
    n = float(np.prod(shape))
    S = dft.rfftn_u(k) * np.sqrt(n)  # unnormalized transform of the kernel
    if np.max(np.abs(S.imag)) > 1e-10 * max(1.0, np.max(np.abs(S.real))):
        raise AssertionError("reference symbol is not real")
    return np.moveaxis(np.moveaxis(S.real, 0, -1), 0, -1)  # [N1,N2,N3h, i, j]


def reference_medium_Q(physics: int, props, shape, L0: float = 1.0) -> np.ndarray:
    """FANS weights ``Q(k) = S_ref(k)^{-1}`` (k != 0), ``Q(0) = 0``; half grid ``[..., c, c]``."""
    S = reference_symbol(physics, reference_props(physics, props), shape, L0)
    Q = np.zeros_like(S)
    flat = S.reshape(-1, S.shape[-2], S.shape[-1])
    out = Q.reshape(flat.shape)
    for i in range(1, flat.shape[0]):  # index 0 is k = 0
        out[i] = np.linalg.inv(flat[i])
    return Q


def symmetrize_half(Q: np.ndarray, N3: int) -> np.ndarray:
    """Make the blocks even, ``Q(-k) = Q(k)``, on the self-conjugate half-grid planes.

    On ``k3 = 0`` (and ``k3 = N3/2`` for even N3) both ``(k1,k2)`` and ``(-k1,-k2)`` are stored;
    they are replaced by their average so that the output of the preconditioner is real.
    """
    Q = Q.copy()
    N1, N2 = Q.shape[0], Q.shape[1]
    i1 = (-np.arange(N1)) % N1
    i2 = (-np.arange(N2)) % N2
    planes = [0] + ([N3 // 2] if N3 % 2 == 0 else [])
    for p in planes:
        P = Q[:, :, p]
        Q[:, :, p] = 0.5 * (P + P[i1][:, i2])
    return Q


def uno_apply(Q: np.ndarray, r: np.ndarray) -> np.ndarray:
    """``s = T^H Q T r`` for ``r[c, N1, N2, N3]`` and half-grid blocks ``Q[N1,N2,N3h,c,c]``."""
    N3 = r.shape[-1]
    R = dft.rfftn_u(r)
    S = np.einsum("xyzij,jxyz->ixyz", Q, R)
    return dft.irfftn_u(S, N3)


def min_eigenvalue(Q: np.ndarray, skip_zero_mode: bool = True) -> float:
    """Smallest eigenvalue over all blocks (the spectrum of P, Lemma 1)."""
    flat = Q.reshape(-1, Q.shape[-2], Q.shape[-1])
    ev = np.linalg.eigvalsh(flat)
    if skip_zero_mode:
        ev = ev[1:]
    return float(ev.min())


def spd_check(Q: np.ndarray, eps: float) -> bool:
    """Safety check of the Remark after Algorithm 2 on all modes k != 0."""
    return min_eigenvalue(Q) > eps


def mode_list(M: int):
    """The modes of ``K_M`` (periodic boundary conditions, d = 3) in the weight order used here:
    k1 from -M to M (slowest), then k2 from -M to M, then k3 from 0 to M, without k = 0."""
    return [(k1, k2, k3) for k1 in range(-M, M + 1) for k2 in range(-M, M + 1) for k3 in range(0, M + 1)
            if (k1, k2, k3) != (0, 0, 0)]


def modes_entries(w: np.ndarray, M: int, shape, c: int) -> np.ndarray:
    """Unique entries ``[N1, N2, N3h, C]`` of ``W + K(k)`` before the self-conjugate planes are
    made even: ``w[0]`` parametrizes the bypass, ``w[1 + i]`` the i-th mode of ``mode_list(M)``."""
    N1, N2, N3 = shape
    w = np.asarray(w, dtype=np.float64)
    modes = mode_list(M)
    if w.shape != (1 + len(modes), n_unique(c)):
        raise ValueError("weights must be [1 + n_modes, C]")
    if 2 * M + 1 > N1 or 2 * M + 1 > N2 or M > N3 // 2:
        raise ValueError("mode set larger than the grid")
    v = np.zeros((N1, N2, N3 // 2 + 1, n_unique(c)))
    v[...] = entries_from_blocks(psi(w[0], c))
    for i, (k1, k2, k3) in enumerate(modes):
        v[k1 % N1, k2 % N2, k3] += entries_from_blocks(psi(w[1 + i], c))
    return v


def modes_Q(w: np.ndarray, M: int, shape, c: int) -> np.ndarray:
    """Half-grid blocks of the paper's parametrization, even on the self-conjugate planes."""
    return symmetrize_half(blocks_from_entries(modes_entries(w, M, shape, c), c), shape[2])
