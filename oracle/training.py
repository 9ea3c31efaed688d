"""UNO training loss and gradients (oracle; test infrastructure only).

* Loss (Eq. (fnocg-loss)): ``L = (1/N_s) sum_j || P_theta f_j - u_j ||^2`` with
  ``P_theta = T^H Q(theta) T``; ``loss_by_definition`` evaluates it by applying the
  preconditioner in real space.
* Closed forms of Sec. 5.4: after transforming the data once, ``L`` is a quadratic in the
  block entries v; for c = 1 (Eq. (features-c-1)) ``L = a . (v*v) - b . v + delta`` and
  ``dL/dv = 2 a * v - b`` with ``a = mean |T f|^2`` and ``b = 2 mean Re(conj(T f) T u)``.
  Here the sums over the full grid are taken on the half grid with the multiplicity of each
  mode (1 on the self-conjugate planes, 2 elsewhere).
* ``grad_entries_general``: the gradient for any c from
  ``dL/dQ_ij(k) = (2/N_s) sum_j w_k Re(conj(Q R - U)_i R_j)`` with the symmetric entries
  collected in the paper's order (App. B.2), then chained through psi.
"""
from __future__ import annotations

import numpy as np

from . import dft, uno


def spectra(fields: np.ndarray) -> np.ndarray:
    """Unitary half-grid spectra of a batch ``[B, c, N1, N2, N3] -> [B, c, N1, N2, N3h]``."""
    return dft.rfftn_u(fields)


def loss_by_definition(Q, f_batch, u_batch) -> float:
    total = 0.0
    for f, u in zip(f_batch, u_batch):
        s = uno.uno_apply(Q, f)
        total += float(np.sum((s - u) ** 2))
    return total / len(f_batch)


def loss_from_spectra(Q, R, U, shape) -> float:
    w = dft.half_multiplicity(shape)
    S = np.einsum("xyzij,bjxyz->bixyz", Q, R)
    return float(np.sum(w * np.abs(S - U) ** 2)) / R.shape[0]


def features_c1(R, U, shape):
    """Features a, b of Eq. (features-c-1) on the half grid (multiplicity included)."""
    w = dft.half_multiplicity(shape)
    a = w * np.mean(np.abs(R[:, 0]) ** 2, axis=0)
    b = w * 2.0 * np.mean(np.real(np.conj(R[:, 0]) * U[:, 0]), axis=0)
    return a, b


def features_general(R, U, shape):
    """Features a_m, b_m of Sec. 5.4 for any c, per half-grid mode with multiplicity, m over the
    unique entries (i, j) in the paper's order (Eq. (features-c-1), Eq. (features-c-2), App. C):
    a_m = mean conj(R_i) R_j (+ conj(R_j) R_i for i != j), b_m = 2 mean Re of the same with the
    second factor taken from U.  Returns ``[N1, N2, N3h, C]`` arrays."""
    c = R.shape[1]
    w = dft.half_multiplicity(shape)
    pairs = [(0, 0)] if c == 1 else uno.PAPER_ORDER
    a = np.zeros(R.shape[2:] + (len(pairs),))
    b = np.zeros_like(a)
    for m, (i, j) in enumerate(pairs):
        ta = np.conj(R[:, i]) * R[:, j]
        tb = np.conj(R[:, i]) * U[:, j]
        if i != j:
            ta = ta + np.conj(R[:, j]) * R[:, i]
            tb = tb + np.conj(R[:, j]) * U[:, i]
        a[..., m] = w * np.mean(ta.real, axis=0)
        b[..., m] = w * 2.0 * np.mean(tb.real, axis=0)
    return a, b


def loss_from_features(v, a, b) -> float:
    """Loss without delta from the features (Sec. 5.4, App. C): with Q(v) the symmetric block of
    the unique entries v, sum_k sum_m a_m (Q^2)_m - b_m v_m, (Q^2)_m the entry (i, j) of Q Q."""
    C = v.shape[-1]
    c = 1 if C == 1 else 3
    Q = uno.blocks_from_entries(v, c)
    Q2 = uno.entries_from_blocks(Q @ Q)
    return float(np.sum(a * Q2) - np.sum(b * v))


def grad_v_c1(v, R, U, shape):
    """``dL/dv = 2 a * v - b`` (Sec. 5.4, c = 1)."""
    a, b = features_c1(R, U, shape)
    return 2.0 * a * v - b


def grad_entries_general(Q, R, U, shape):
    """Gradient of the loss w.r.t. the unique entries ``[N1,N2,N3h,C]`` (paper order)."""
    c = Q.shape[-1]
    w = dft.half_multiplicity(shape)
    S = np.einsum("xyzij,bjxyz->bixyz", Q, R)
    E = S - U
    G = 2.0 * np.real(np.einsum("bixyz,bjxyz->xyzij", np.conj(E), R)) * w[..., None, None]
    G /= R.shape[0]
    if c == 1:
        return G[..., 0, :]
    out = np.zeros(G.shape[:3] + (6,))
    for m, (i, j) in enumerate(uno.PAPER_ORDER):
        out[..., m] = G[..., i, j] if i == j else G[..., i, j] + G[..., j, i]
    return out


def grad_theta(theta, grad_entries, c: int):
    """Chain rule through psi: ``dL/dtheta`` from ``dL/dv``."""
    theta = np.asarray(theta, dtype=np.float64)
    if c == 1:
        return 2.0 * theta * grad_entries
    eps = 1e-7
    out = np.zeros_like(theta)
    for m in range(theta.shape[-1]):
        tp = theta.copy()
        tm = theta.copy()
        tp[..., m] += eps
        tm[..., m] -= eps
        dv = (uno.entries_from_blocks(uno.psi(tp, 3)) - uno.entries_from_blocks(uno.psi(tm, 3))) / (2 * eps)
        out[..., m] = np.sum(dv * grad_entries, axis=-1)
    return out


def grad_modes(w, M: int, shape, c: int, grad_entries):
    """Chain rule for the bypass-plus-modes weights: ``dL/dw`` ``[1 + n_modes, C]`` from the
    gradient w.r.t. the (even) half-grid entries.  The entries are the even part of the raw
    ones, an averaging that is its own adjoint; the bypass acts on every mode."""
    g_raw = uno.symmetrize_half(np.asarray(grad_entries, dtype=np.float64), shape[2])
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    out[0] = grad_theta(w[0], g_raw.reshape(-1, g_raw.shape[-1]).sum(axis=0), c)
    for i, (k1, k2, k3) in enumerate(uno.mode_list(M)):
        out[1 + i] = grad_theta(w[1 + i], g_raw[k1 % shape[0], k2 % shape[1], k3], c)
    return out


def modes_loss_c1(w, M: int, shape, a, b):
    """Loss of Eq. (loss-precomputed) for c = 1 from the features a, b (without the constant
    delta) for the bypass-plus-modes weights ``w`` [1 + n_modes, 1]."""
    v = uno.entries_from_blocks(uno.modes_Q(w, M, shape, 1))[..., 0]
    return float(np.sum(a * v * v - b * v))


def optimum_modes_c1(a, b, M: int, shape):
    """Global minimizer of the c = 1 loss over the bypass-plus-modes weights (Sec. 5.4 for the
    layout of Eq. (fnocg-parametrization)).  With beta = psi(w_0) and v_k = beta + psi(w_k) on
    K_M, the loss sum_k a_k v_k^2 - b_k v_k separates: for fixed beta each mode of K_M takes
    v_k = max(beta, b_k / (2 a_k)), every other mode v_k = beta, and the remaining function of
    beta is convex with a nondecreasing piecewise-linear derivative whose root is bracketed and
    found by bisection.  The k = 0 mode (a = b = 0 for zero-mean data) does not take part.
    Returns w [1 + n_modes, 1]."""
    N1, N2, N3 = shape
    modes = uno.mode_list(M)
    inK = np.zeros(a.shape, dtype=bool)
    for (k1, k2, k3) in modes:
        inK[k1 % N1, k2 % N2, k3] = True
    # the mode set is even on the self-conjugate planes (its (k1, k2) range is symmetric), so
    # the features there pair up and the optimum is even without the averaging step
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(a > 0, b / (2.0 * a), -np.inf)

    def dphi(beta):
        active = (~inK) | (c < beta)
        return float(np.sum((2.0 * a * beta - b)[active]))

    lo, hi = 0.0, 1.0
    while dphi(hi) < 0:
        hi *= 2.0
    if dphi(lo) >= 0:
        beta = 0.0
    else:
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if dphi(mid) < 0:
                lo = mid
            else:
                hi = mid
        beta = 0.5 * (lo + hi)
    w = np.zeros((1 + len(modes), 1))
    w[0, 0] = np.sqrt(beta)
    for i, (k1, k2, k3) in enumerate(modes):
        ck = c[k1 % N1, k2 % N2, k3]
        w[1 + i, 0] = np.sqrt(max(ck - beta, 0.0)) if np.isfinite(ck) else 0.0
    return w
