"""Learned UNO weights for 2D problems with periodic BC, c = 1 and c = 2 (oracle; test
infrastructure only).

* Local parametrization (Sec. 5.2.2): c = 1, psi(w) = w^2; c = 2, Eq. (local-param-2), the
  Cholesky-like product of the lower triangular [[w1, 0], [w3, w2]] with its transpose:
  psi(w) = [[w1 w1, w1 w3], [w1 w3, w2 w2 + w3 w3]] (diagonal not forced positive).
* Block entries in the order of Sec. 5.4 for c = 2: v1 = Q_xx, v2 = Q_yy, v3 = Q_xy (the band
  matrix [[diag v1, diag v3], [diag v3, diag v2]]).
* Mode set of the periodic row of Table (fnocg-mode-selection-2d) for d = 2:
  K_M = [-M, M] x [0, M] minus {0}, n_modes = (2M + 1)(M + 1) - 1, ordered k1 (from -M), then k2
  (from 0); the conjugate modes (-k1, -k2) of those with k2 > 0 carry the same block, so P is
  real.  Weight layout (Eq. (fnocg-operator), Eq. (fnocg-parametrization)): an inner bypass
  psi(w_0) on every mode plus psi(w_i) on the i-th mode of K_M.
* Loss (Eq. (fnocg-loss)) over N_s samples, L = (1/N_s) sum_j ||P f_j - u_j||^2 with
  P = T^H Q T and T the unitary 2D DFT (``fem2d.transform``); from the features of
  Eq. (features-c-1) / Eq. (features-c-2) it is, for c = 2 and summed over all modes of the
  full grid, L = a1 . (v1^2 + v3^2) + a2 . (v2^2 + v3^2) + a3 . (v1 v3 + v2 v3)
  - b1 . v1 - b2 . v2 - b3 . v3 + delta, with the gradient and Hessian printed there.
"""
from __future__ import annotations

import numpy as np

from . import fem2d


def n_entries(c: int) -> int:
    return c * (c + 1) // 2


def psi(w: np.ndarray, c: int) -> np.ndarray:
    """``w [..., C] -> SPD blocks [..., c, c]`` (Sec. 5.2.2)."""
    w = np.asarray(w, dtype=np.float64)
    if c == 1:
        return (w[..., 0] ** 2)[..., None, None]
    L = np.zeros(w.shape[:-1] + (2, 2))
    L[..., 0, 0] = w[..., 0]
    L[..., 1, 1] = w[..., 1]
    L[..., 1, 0] = w[..., 2]
    return L @ np.swapaxes(L, -1, -2)


def entries(Q: np.ndarray) -> np.ndarray:
    """Blocks ``[..., c, c]`` -> entries ``[..., C]``: c = 2 gives (Q_xx, Q_yy, Q_xy)."""
    if Q.shape[-1] == 1:
        return Q[..., 0, :].copy()
    return np.stack([Q[..., 0, 0], Q[..., 1, 1], Q[..., 0, 1]], axis=-1)


def blocks(v: np.ndarray, c: int) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    if c == 1:
        return v[..., None]
    Q = np.zeros(v.shape[:-1] + (2, 2))
    Q[..., 0, 0] = v[..., 0]
    Q[..., 1, 1] = v[..., 1]
    Q[..., 0, 1] = Q[..., 1, 0] = v[..., 2]
    return Q


def mode_list(M: int):
    """K_M of the periodic row of Table (fnocg-mode-selection-2d), d = 2."""
    return [(k1, k2) for k1 in range(-M, M + 1) for k2 in range(0, M + 1) if (k1, k2) != (0, 0)]


def modes_Q(w: np.ndarray, M: int, shape, c: int) -> np.ndarray:
    """Blocks ``[N1, N2, c, c]`` on the full 2D grid of the bypass-plus-modes weights
    ``w [1 + n_modes, C]`` (needs 2M < N1 and 2M < N2); the conjugate (-k1, -k2) of a mode with
    k2 > 0 gets its block.  The line k2 = 0 holds both (k1, 0) and (-k1, 0) as learned modes;
    their blocks are averaged there (the 2D form of the symmetrization on the self-conjugate
    planes of the 3D half grid), so P is real for any weights."""
    N1, N2 = shape
    if not (2 * M < N1 and 2 * M < N2):
        raise ValueError("mode set larger than the grid")
    w = np.asarray(w, dtype=np.float64).reshape(-1, n_entries(c))
    Q = np.broadcast_to(psi(w[0], c), (N1, N2, c, c)).copy()
    for i, (k1, k2) in enumerate(mode_list(M)):
        B = psi(w[0], c) + psi(w[1 + i], c)
        Q[k1 % N1, k2 % N2] = B
        if k2 > 0:
            Q[(-k1) % N1, (-k2) % N2] = B
    row = Q[:, 0].copy()
    Q[:, 0] = 0.5 * (row + row[(-np.arange(N1)) % N1])
    return Q


def spectra(fields: np.ndarray) -> np.ndarray:
    """Unitary 2D DFT of a batch ``[N_s, c, N1, N2]`` (both axes periodic)."""
    shape = fields.shape[-2:]
    return fem2d.transform(fields, shape, (False, False))


def loss_by_definition(Q, f_batch, u_batch) -> float:
    """Eq. (fnocg-loss): mean over samples of ||P f - u||^2, P applied in real space."""
    shape = f_batch.shape[-2:]
    total = 0.0
    for f, u in zip(f_batch, u_batch):
        s = fem2d.uno_apply(Q, f, shape, (False, False))
        total += float(np.sum((s - u) ** 2))
    return total / len(f_batch)


def features(R: np.ndarray, U: np.ndarray):
    """Features per mode of the full grid from the spectra ``R = T f``, ``U = T u``
    ``[N_s, c, N1, N2]``: c = 1 Eq. (features-c-1), c = 2 Eq. (features-c-2).  Returns
    ``a, b [N1, N2, C]`` and ``delta`` (mean ||u||^2)."""
    Ns, c = R.shape[:2]
    delta = float(np.sum(np.abs(U) ** 2)) / Ns
    if c == 1:
        a = np.sum(np.abs(R[:, 0]) ** 2, axis=0) / Ns
        b = 2.0 * np.sum((np.conj(R[:, 0]) * U[:, 0]).real, axis=0) / Ns
        return a[..., None], b[..., None], delta
    Rx, Ry, Ux, Uy = R[:, 0], R[:, 1], U[:, 0], U[:, 1]
    a1 = np.sum(np.conj(Rx) * Rx, axis=0).real / Ns
    a2 = np.sum(np.conj(Ry) * Ry, axis=0).real / Ns
    a3 = np.sum(np.conj(Rx) * Ry + np.conj(Ry) * Rx, axis=0).real / Ns
    b1 = 2.0 * np.sum((np.conj(Rx) * Ux).real, axis=0) / Ns
    b2 = 2.0 * np.sum((np.conj(Ry) * Uy).real, axis=0) / Ns
    b3 = 2.0 * np.sum((np.conj(Rx) * Uy + np.conj(Ry) * Ux).real, axis=0) / Ns
    return np.stack([a1, a2, a3], axis=-1), np.stack([b1, b2, b3], axis=-1), delta


def loss_from_features(v, a, b, delta: float) -> float:
    """The loss of Sec. 5.4 as a function of the entries ``v [N1, N2, C]``."""
    if v.shape[-1] == 1:
        return float(np.sum(a[..., 0] * v[..., 0] ** 2 - b[..., 0] * v[..., 0])) + delta
    v1, v2, v3 = v[..., 0], v[..., 1], v[..., 2]
    a1, a2, a3 = a[..., 0], a[..., 1], a[..., 2]
    return float(np.sum(a1 * (v1 * v1 + v3 * v3) + a2 * (v2 * v2 + v3 * v3) + a3 * (v1 * v3 + v2 * v3)
                        - b[..., 0] * v1 - b[..., 1] * v2 - b[..., 2] * v3)) + delta


def grad_entries(v, a, b) -> np.ndarray:
    """dL/dv of Sec. 5.4 (c = 1: 2 a v - b; c = 2 the three components printed there)."""
    if v.shape[-1] == 1:
        return 2.0 * a * v - b
    v1, v2, v3 = v[..., 0], v[..., 1], v[..., 2]
    a1, a2, a3 = a[..., 0], a[..., 1], a[..., 2]
    return np.stack([2 * a1 * v1 + a3 * v3 - b[..., 0],
                     2 * a2 * v2 + a3 * v3 - b[..., 1],
                     2 * a1 * v3 + 2 * a2 * v3 + a3 * (v1 + v2) - b[..., 2]], axis=-1)


def hess_entries(a) -> np.ndarray:
    """d^2 L / dv dv per mode ``[N1, N2, C, C]`` of Sec. 5.4 (constant in v)."""
    if a.shape[-1] == 1:
        return 2.0 * a[..., None]
    a1, a2, a3 = a[..., 0], a[..., 1], a[..., 2]
    H = np.zeros(a.shape[:-1] + (3, 3))
    H[..., 0, 0] = 2 * a1
    H[..., 1, 1] = 2 * a2
    H[..., 2, 2] = 2 * (a1 + a2)
    H[..., 0, 2] = H[..., 2, 0] = a3
    H[..., 1, 2] = H[..., 2, 1] = a3
    return H


def modes_loss(w, M: int, shape, c: int, a, b, delta: float) -> float:
    """The loss of the bypass-plus-modes weights from the features."""
    return loss_from_features(entries(modes_Q(w, M, shape, c)), a, b, delta)
