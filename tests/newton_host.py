"""Host restatement (NumPy, FP64) of the device Newton-Raphson of Algorithm 4 (k_newton.cu):
the same arrow-shaped Hessian, Schur-complement step and Levenberg-Marquardt damping, written
with the chain rule through psi in array form.  Test infrastructure: pinned against the
oracle's optima on the CPU and compared with the library's device result on the GPU."""
from __future__ import annotations

import numpy as np

from paper_2508_02681_gb300.training import _L3, _ORDER3, _mode_index, mode_set_2d


def _entry_mats():
    """Symmetric unit matrices E_e = dQ/dv_e of the six unique entries (paper order)."""
    E = np.zeros((6, 3, 3))
    for e, (i, j) in enumerate(_ORDER3):
        E[e, i, j] = E[e, j, i] = 1.0
    return E


def _entries(Mx):
    return np.stack([Mx[..., i, j] for (i, j) in _ORDER3], axis=-1)


_E6 = _entry_mats()
# d^2 (Q Q)_m / dv_e dv_f = (E_e E_f + E_f E_e)_m
_T6 = _entries(np.einsum("eij,fjk->efik", _E6, _E6) + np.einsum("fij,ejk->efik", _E6, _E6))
# psi: F_p = dL/dw_p (unit matrix at the position of parameter p in L)
_F6 = np.zeros((6, 3, 3))
for _p, (_r, _q) in enumerate(_L3):
    _F6[_p, _r, _q] = 1.0
# d^2 v / dw_p dw_q = entries(F_p F_q^T + F_q F_p^T), constant
_D2 = np.moveaxis(_entries(np.einsum("pij,qkj->pqik", _F6, _F6) + np.einsum("qij,pkj->pqik", _F6, _F6)), -1, 0)


def _psi_jac(w):
    """v = entries(L L^T) and J = dv/dw for weights [..., 6] (c = 3)."""
    L = np.zeros(w.shape[:-1] + (3, 3))
    for i, (r, q) in enumerate(_L3):
        L[..., r, q] = w[..., i]
    v = _entries(L @ np.swapaxes(L, -1, -2))
    dQ = np.einsum("pij,...kj->...pik", _F6, L)
    J = np.swapaxes(_entries(dQ + np.swapaxes(dQ, -1, -2)), -1, -2)  # [..., e, p]
    return v, J


def second_order_modes_c3(a, b, M: int, w0, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 for c = 3 (App. C) on the paper's weight layout: Newton-Raphson on
    w = [w_0; w_1 .. w_n] (six psi parameters each, Q = L L^T) for the loss
    L = sum_k sum_m a_m (Q^2)_m - b_m v_m with v = psi(w_0) + psi(w_i) on the i-th mode of K_M
    and psi(w_0) elsewhere.  Gradient and Hessian by the chain rule through psi (Sec. 5.4);
    the Hessian is an arrow of 6 x 6 blocks (the bypass couples to every mode), each step an
    O(n) block Schur-complement solve with Levenberg-Marquardt damping when a step does not
    lower the loss.  Returns (w [1 + n_modes, 6], loss history without delta)."""
    shape = a.shape[:2] + (2 * (a.shape[2] - 1),)
    i1, i2, i3 = _mode_index(shape, M)
    ak, bk = a[i1, i2, i3], b[i1, i2, i3]            # [n, 6]
    a_rest = a.reshape(-1, 6).sum(axis=0) - ak.sum(axis=0)
    b_rest = b.reshape(-1, 6).sum(axis=0) - bk.sum(axis=0)
    Hk = np.einsum("efm,nm->nef", _T6, ak)           # Hessian of L in v per mode
    Hr = np.einsum("efm,m->ef", _T6, a_rest)
    w = np.asarray(w0, dtype=np.float64).reshape(-1, 6).copy()

    def loss(x):
        v0, _ = _psi_jac(x[0])
        vi = v0 + _psi_jac(x[1:])[0]
        return float(0.5 * v0 @ Hr @ v0 - b_rest @ v0
                     + np.sum(0.5 * np.einsum("ne,nef,nf->n", vi, Hk, vi) - np.sum(bk * vi, axis=1)))

    hist = [loss(w)]
    lam = 0.0
    I6 = np.eye(6)
    for _ in range(iters):
        v0, J0 = _psi_jac(w[0])
        u, Ji = _psi_jac(w[1:])
        vi = v0 + u
        Gi = np.einsum("nef,nf->ne", Hk, vi) - bk     # dL_i / dv
        Gall = Hr @ v0 - b_rest + Gi.sum(axis=0)
        g0 = J0.T @ Gall
        gi = np.einsum("nep,ne->np", Ji, Gi)
        H00 = J0.T @ (Hr + Hk.sum(axis=0)) @ J0 + np.einsum("e,epq->pq", Gall, _D2)
        H0i = np.einsum("ep,nef,nfq->npq", J0, Hk, Ji)              # [n, 6(w0), 6(wi)]
        Hii = np.einsum("nep,nef,nfq->npq", Ji, Hk, Ji) + np.einsum("ne,epq->npq", Gi, _D2)
        while True:
            D = Hii + lam * I6
            ok = np.all(np.linalg.eigvalsh(D) > 0)
            if ok:
                Dinv_g = np.linalg.solve(D, gi[..., None])[..., 0]
                Dinv_H = np.linalg.solve(D, np.swapaxes(H0i, -1, -2))    # D_i^-1 H_i0
                S = H00 + lam * I6 - np.einsum("npq,nqr->pr", H0i, Dinv_H)
                if np.all(np.linalg.eigvalsh(S) > 0):
                    x0 = np.linalg.solve(S, g0 - np.einsum("npq,nq->p", H0i, Dinv_g))
                    xi = Dinv_g - np.einsum("nqp,p->nq", Dinv_H, x0)
                    trial = w - np.vstack([x0[None], xi])
                    lt = loss(trial)
                    if lt <= hist[-1]:
                        break
            lam = max(2.0 * lam, 1e-12 * max(1.0, float(np.max(np.abs(Hii)))))
            if lam > 1e30:
                return w, hist
        w = trial
        hist.append(lt)
        lam *= 0.1
        if abs(hist[-2] - hist[-1]) <= tol * max(1.0, abs(hist[-1])):
            break
    return w, hist


def second_order_modes(a, b, M: int, w0, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 (second-order training, c = 1) for the paper's layout: Newton-Raphson on the
    weights w = [w_0; w_1 .. w_n] with gradient and Hessian of L = sum_k a_k v_k^2 - b_k v_k
    (v_k = w_0^2 + w_i^2 on the i-th mode of K_M, w_0^2 elsewhere) from the features.  The
    Hessian is an arrow matrix (the bypass couples to every mode): each step is an O(n) solve by
    its Schur complement.  A step that does not lower the loss is damped (Levenberg-Marquardt).
    Returns (w [1 + n_modes, 1], loss history without the constant delta)."""
    shape = a.shape[:2] + (2 * (a.shape[2] - 1),)
    i1, i2, i3 = _mode_index(shape, M)
    ak, bk = a[i1, i2, i3], b[i1, i2, i3]
    a_rest = a.sum() - ak.sum()
    b_rest = b.sum() - bk.sum()
    w = np.asarray(w0, dtype=np.float64).reshape(-1).copy()

    def loss(x):
        beta = x[0] ** 2
        v = beta + x[1:] ** 2
        return float(a_rest * beta * beta - b_rest * beta + np.sum(ak * v * v - bk * v))

    hist = [loss(w)]
    lam = 0.0
    for _ in range(iters):
        wb, wm = w[0], w[1:]
        beta = wb * wb
        v = beta + wm * wm
        gk = 2.0 * ak * v - bk                    # dL/dv on the modes of K_M
        g_rest = 2.0 * a_rest * beta - b_rest     # summed over all other modes
        gb = 2.0 * wb * (g_rest + gk.sum())
        gm = 2.0 * wm * gk
        hbb = 8.0 * wb * wb * (a_rest + ak.sum()) + 2.0 * (g_rest + gk.sum())
        hmm = 8.0 * ak * wm * wm + 2.0 * gk
        hbm = 8.0 * ak * wb * wm
        while True:
            D = hmm + lam
            if np.all(D > 0):
                schur = hbb + lam - np.sum(hbm * hbm / D)
                if schur > 0:
                    xb = (gb - np.sum(hbm * gm / D)) / schur
                    xm = (gm - hbm * xb) / D
                    trial = w - np.concatenate(([xb], xm))
                    lt = loss(trial)
                    if lt <= hist[-1]:
                        break
            lam = max(2.0 * lam, 1e-12 * max(1.0, float(np.max(np.abs(hmm)))))
            if lam > 1e30:
                return w.reshape(-1, 1), hist
        w = trial
        hist.append(lt)
        lam *= 0.1 if lam > 0 else 0.0
        if abs(hist[-2] - hist[-1]) <= tol * max(1.0, abs(hist[-1])):
            break
    return w.reshape(-1, 1), hist


def _hess_2d(a):
    """Hessian in the entries per mode (Sec. 5.4): 2a for c = 1; the printed 3 x 3 for c = 2."""
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


def _psi_jac_2d(w, c: int):
    """v = entries(psi(w)) and J = dv/dw, and the constant d^2 v / dw^2 [C, P, P]."""
    if c == 1:
        return w ** 2, (2.0 * w)[..., None], np.full((1, 1, 1), 2.0)
    w1, w2, w3 = w[..., 0], w[..., 1], w[..., 2]
    v = np.stack([w1 * w1, w2 * w2 + w3 * w3, w1 * w3], axis=-1)
    z = np.zeros_like(w1)
    J = np.stack([np.stack([2 * w1, z, z], -1),
                  np.stack([z, 2 * w2, 2 * w3], -1),
                  np.stack([w3, z, w1], -1)], axis=-2)     # [..., entry, param]
    D2 = np.zeros((3, 3, 3))
    D2[0, 0, 0] = 2.0
    D2[1, 1, 1] = D2[1, 2, 2] = 2.0
    D2[2, 0, 2] = D2[2, 2, 0] = 1.0
    return v, J, D2


def second_order_modes_2d(a, b, M: int, w0, c: int, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 for 2D problems (c = 1, c = 2) on the paper's weight layout with the 2D mode
    set: Newton-Raphson on w = [w_0; w_1 .. w_n] for L = sum_k (1/2) v_k^T H_k v_k - b_k . v_k
    (H_k the Hessian in the entries of Sec. 5.4), v = psi(w_0) + psi(w_i) on the i-th mode of
    K_M and psi(w_0) elsewhere; gradient and Hessian by the chain rule through psi, an arrow of
    C x C blocks solved by its Schur complement (O(n) per step), Levenberg-Marquardt damping
    when a step does not lower the loss.  ``a, b``: features on the 2D half grid
    [N1, N2/2+1, C] with multiplicities (``features_2d``).  Returns (w [1 + n, C], loss history
    without delta)."""
    N1 = a.shape[0]
    C = a.shape[-1]
    ms = mode_set_2d(M)
    i1 = np.array([k1 % N1 for k1, _ in ms])
    i2 = np.array([k2 for _, k2 in ms])
    # the line k2 = 0 of the half grid holds (k1, 0) and (-k1, 0) with multiplicity 1 each;
    # the other columns carry the conjugates through multiplicity 2
    ak, bk = a[i1, i2], b[i1, i2]
    a_rest = a.reshape(-1, C).sum(axis=0) - ak.sum(axis=0)
    b_rest = b.reshape(-1, C).sum(axis=0) - bk.sum(axis=0)
    Hk = _hess_2d(ak)
    Hr = _hess_2d(a_rest)
    w = np.asarray(w0, dtype=np.float64).reshape(-1, C).copy()
    I = np.eye(C)

    def loss(x):
        v0, _, _ = _psi_jac_2d(x[0], c)
        vi = v0 + _psi_jac_2d(x[1:], c)[0]
        return float(0.5 * v0 @ Hr @ v0 - b_rest @ v0
                     + np.sum(0.5 * np.einsum("ne,nef,nf->n", vi, Hk, vi) - np.sum(bk * vi, axis=1)))

    hist = [loss(w)]
    lam = 0.0
    for _ in range(iters):
        v0, J0, D2 = _psi_jac_2d(w[0], c)
        u, Ji, _ = _psi_jac_2d(w[1:], c)
        vi = v0 + u
        Gi = np.einsum("nef,nf->ne", Hk, vi) - bk
        Gall = Hr @ v0 - b_rest + Gi.sum(axis=0)
        g0 = J0.T @ Gall
        gi = np.einsum("nep,ne->np", Ji, Gi)
        H00 = J0.T @ (Hr + Hk.sum(axis=0)) @ J0 + np.einsum("e,epq->pq", Gall, D2)
        H0i = np.einsum("ep,nef,nfq->npq", J0, Hk, Ji)
        Hii = np.einsum("nep,nef,nfq->npq", Ji, Hk, Ji) + np.einsum("ne,epq->npq", Gi, D2)
        while True:
            Dm = Hii + lam * I
            if np.all(np.linalg.eigvalsh(Dm) > 0):
                Dinv_g = np.linalg.solve(Dm, gi[..., None])[..., 0]
                Dinv_H = np.linalg.solve(Dm, np.swapaxes(H0i, -1, -2))
                S = H00 + lam * I - np.einsum("npq,nqr->pr", H0i, Dinv_H)
                if np.all(np.linalg.eigvalsh(S) > 0):
                    x0 = np.linalg.solve(S, g0 - np.einsum("npq,nq->p", H0i, Dinv_g))
                    xi = Dinv_g - np.einsum("nqp,p->nq", Dinv_H, x0)
                    trial = w - np.vstack([x0[None], xi])
                    lt = loss(trial)
                    if lt <= hist[-1]:
                        break
            lam = max(2.0 * lam, 1e-12 * max(1.0, float(np.max(np.abs(Hii)))))
            if lam > 1e30:
                return w, hist
        w = trial
        hist.append(lt)
        lam *= 0.1
        if abs(hist[-2] - hist[-1]) <= tol * max(1.0, abs(hist[-1])):
            break
    return w, hist
