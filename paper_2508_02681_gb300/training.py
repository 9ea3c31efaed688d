"""Training of the UNO preconditioner on solver-generated data (Sec. 5.3, Algorithm 3).

Data: pairs (f_j, u_j) with K_j u_j = f_j (Sec. 5.3: the right-hand sides and solutions that
occur in the solver), produced by batched UNO-CG solves of this library.  Model: s = P_theta f
with P_theta = T^H Q(psi(theta)) T on the full half grid.  Loss: the MSE of Eq. (fnocg-loss) over
a minibatch.  Gradients: the library's backward kernels through ``solver.uno_function``;
optimizer: Adam (torch).
"""
from __future__ import annotations

import numpy as np

from . import _lib, api
from .solver import Homogenization, uno_function


def generate_data(phases, props, load, shape, tol: float = 1e-8, chunk: int = 64):
    """Solve K_j u_j = f_j for every instance (one macroscopic load); returns device float32
    tensors ``f, u`` of shape ``[n, 1, N1, N2, N3]`` and the iteration counts."""
    import torch

    n = len(phases)
    f = torch.empty((n, 1) + tuple(shape), dtype=torch.float32, device="cuda")
    u = torch.empty_like(f)
    iters = []
    tmp = torch.empty((1,) + tuple(shape), dtype=torch.float64, device="cuda")
    for s0 in range(0, n, chunk):
        B = min(chunk, n - s0)
        h = Homogenization(_lib.THERMAL, shape, batch=B)
        api.unocg_set_stream(h.ctx, torch.cuda.current_stream())
        h.set_microstructure(np.stack(phases[s0:s0 + B]), 2)
        h.set_phase_properties(np.stack(props[s0:s0 + B]))
        h.set_macro_load(np.atleast_2d(load))
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        info = h.solve(tol=tol, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
        iters.extend(int(x) for x in info.iters)
        for b in range(B):
            api.unocg_rhs_dev(h.ctx, b, 0, tmp)
            f[s0 + b].copy_(tmp)
            api.unocg_get_fluctuation_dev(h.ctx, b, 0, tmp)
            u[s0 + b].copy_(tmp)
        torch.cuda.synchronize()
        h.close()
    return f, u, iters


def reference_theta(shape, kappa_ref: float) -> np.ndarray:
    """theta with psi(theta) = the reference-medium weights Q_ref (theta = sqrt(Q)), an
    initialization inside the convex region of the loss."""
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(np.zeros(shape, np.uint8), 1)
    h.set_phase_properties(np.array([kappa_ref]))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    nh = shape[0] * shape[1] * (shape[2] // 2 + 1)
    q = api.unocg_get_uno_weights(h.ctx, 0, nh, 1)
    h.close()
    q = np.maximum(q, 0.0)
    return np.sqrt(q).reshape(shape[0], shape[1], shape[2] // 2 + 1, 1)


def mode_set(M: int):
    """Modes of K_M = [-M, M]^2 x [0, M] without k = 0, in the weight order of the library
    (k1 slowest from -M, then k2 from -M, then k3 from 0)."""
    return [(k1, k2, k3) for k1 in range(-M, M + 1) for k2 in range(-M, M + 1) for k3 in range(M + 1)
            if (k1, k2, k3) != (0, 0, 0)]


def reference_modes(shape, M: int, kappa_ref: float) -> np.ndarray:
    """Weights ``[1 + n_modes, 1]`` of the paper's layout that reproduce the reference-medium
    operator on K_M: the bypass is the smallest reference weight (its value at the highest
    frequencies), each mode adds the rest of its reference weight."""
    q = reference_theta(shape, kappa_ref)[..., 0] ** 2
    qb = float(q.reshape(-1)[1:].min())
    w = np.zeros((1 + len(mode_set(M)), 1))
    w[0, 0] = np.sqrt(qb)
    for i, (k1, k2, k3) in enumerate(mode_set(M)):
        w[1 + i, 0] = np.sqrt(max(q[k1 % shape[0], k2 % shape[1], k3] - qb, 0.0))
    return w


# unique entries of a symmetric 3 x 3 block in the paper's order (App. B.2)
_ORDER3 = ((0, 0), (1, 1), (0, 1), (2, 2), (1, 2), (0, 2))
# psi for c = 3 (Eq. (local-param-3)): Q = L L^T, L lower triangular with
# L00 = w1, L11 = w2, L10 = w3, L22 = w4, L21 = w5, L20 = w6
_L3 = ((0, 0), (1, 1), (1, 0), (2, 2), (2, 1), (2, 0))


def psi(w, c: int) -> np.ndarray:
    """Local SPD parametrization (Sec. 5.2.2) on the host: weights ``[..., C]`` -> blocks
    ``[..., c, c]`` (``w^2`` for c = 1, ``L L^T`` for c = 3)."""
    w = np.asarray(w, dtype=np.float64)
    if c == 1:
        return (w[..., 0] ** 2)[..., None, None]
    L = np.zeros(w.shape[:-1] + (3, 3))
    for i, (r, q) in enumerate(_L3):
        L[..., r, q] = w[..., i]
    return L @ np.swapaxes(L, -1, -2)


def psi_inverse(Q) -> np.ndarray:
    """Weights w with psi(w) = Q for symmetric positive semi-definite blocks ``[..., c, c]``
    (square root for c = 1, the Cholesky factor with a non-negative diagonal for c = 3; a
    semi-definite block is factored after shifting it by 1e-14 of its trace)."""
    Q = np.asarray(Q, dtype=np.float64)
    c = Q.shape[-1]
    if c == 1:
        return np.sqrt(np.maximum(Q[..., 0, :], 0.0))
    shift = 1e-14 * np.trace(Q, axis1=-2, axis2=-1)[..., None, None] * np.eye(3)
    L = np.linalg.cholesky(Q + shift)
    return np.stack([L[..., r, q] for (r, q) in _L3], axis=-1)


def reference_modes_blocks(physics: int, shape, M: int, ref_props) -> np.ndarray:
    """Weights ``[1 + n_modes, C]`` of the paper's layout from the reference-medium weights of
    a homogeneous phase ``ref_props`` (kappa, or (E, nu)): the bypass is lambda I with lambda
    the smallest eigenvalue of Q_ref(k) over k != 0, each mode of K_M adds
    Q_ref(k) - lambda I.  For c = 1 this is ``reference_modes``."""
    c = 1 if physics == _lib.THERMAL else 3
    C = c * (c + 1) // 2
    h = Homogenization(physics, shape)
    h.set_microstructure(np.zeros(shape, np.uint8), 1)
    h.set_phase_properties(np.atleast_2d(np.asarray(ref_props, dtype=np.float64)).reshape(1, -1)
                           if c == 3 else np.array([float(ref_props)]))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    nh = shape[0] * shape[1] * (shape[2] // 2 + 1)
    v = api.unocg_get_uno_weights(h.ctx, 0, nh, C).reshape(shape[0], shape[1], -1, C)
    h.close()
    Q = np.zeros(v.shape[:3] + (c, c))
    if c == 1:
        Q[..., 0, 0] = v[..., 0]
    else:
        for i, (r, q) in enumerate(_ORDER3):
            Q[..., r, q] = Q[..., q, r] = v[..., i]
    lam = float(np.linalg.eigvalsh(Q.reshape(-1, c, c)[1:]).min())
    w = np.zeros((1 + len(mode_set(M)), C))
    w[0] = psi_inverse(lam * np.eye(c))
    i1, i2, i3 = _mode_index(shape, M)
    w[1:] = psi_inverse(Q[i1, i2, i3] - lam * np.eye(c))
    return w


def save_checkpoint(path: str, theta, optimizer=None, **meta):
    """Training checkpoint: the weights (theta or the paper's layout), the optimizer state (Adam
    moments and step counts) and free-form metadata (epoch, losses, M, ...)."""
    import torch
    torch.save({"theta": theta.detach().cpu(), "optimizer": optimizer.state_dict() if optimizer is not None else None,
                "meta": meta}, path)


def load_checkpoint(path: str, device="cuda"):
    """Returns (theta tensor on ``device`` with requires_grad, optimizer state dict or None, meta);
    resume with ``torch.optim.Adam([theta]).load_state_dict(state)``."""
    import torch
    ck = torch.load(path, map_location="cpu", weights_only=False)
    theta = ck["theta"].to(device).requires_grad_(True)
    return theta, ck["optimizer"], ck["meta"]


def train(f, u, theta0, epochs: int, batch: int = 64, lr: float = 1e-2, seed: int = 0,
          modes_M: int | None = None, checkpoint: str | None = None, resume: str | None = None):
    """Adam on the MSE loss; returns (theta tensor, per-epoch mean losses).  With ``modes_M``
    theta0 is in the paper's layout ``[1 + n_modes, 1]`` (see ``reference_modes``).  With
    ``checkpoint`` the weights, Adam state, shuffling state and losses are saved after every
    epoch; ``resume`` continues from such a file (epochs counts the total)."""
    import torch

    shape = tuple(f.shape[2:])
    op = api.unocg_uno_create(1, *shape)
    Fn = uno_function(modes_M)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    start = 0
    if resume is not None:
        theta, state, meta = load_checkpoint(resume)
        opt = torch.optim.Adam([theta], lr=lr)
        if state is not None:
            opt.load_state_dict(state)
        losses = list(meta.get("losses", []))
        start = int(meta.get("epoch", 0))
        if "rng" in meta:
            g.set_state(meta["rng"])
    else:
        theta = torch.tensor(theta0, dtype=torch.float32, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([theta], lr=lr)
    n = f.shape[0]
    for ep in range(start, epochs):
        perm = torch.randperm(n, generator=g)
        tot = 0.0
        for s0 in range(0, n, batch):
            idx = perm[s0:s0 + batch].to("cuda")
            fb, ub = f.index_select(0, idx), u.index_select(0, idx)
            opt.zero_grad()
            s = Fn.apply(fb, theta, op)
            loss = ((s - ub) ** 2).sum() / fb.shape[0]
            loss.backward()
            opt.step()
            tot += float(loss.detach()) * fb.shape[0]
        losses.append(tot / n)
        if checkpoint is not None:
            save_checkpoint(checkpoint, theta, opt, epoch=ep + 1, losses=losses, rng=g.get_state(), modes_M=modes_M)
    api.unocg_uno_destroy(op)
    return theta.detach(), losses


def features(f, u, chunk: int = 64):
    """Features a, b of Sec. 5.4 on the half grid from training data f, u (torch float32
    [N_s, c, N1, N2, N3] on the GPU): c = 1 (Eq. (features-c-1)) returns numpy float64 arrays
    [N1, N2, N3/2+1]; c = 3 (App. C) returns [N1, N2, N3/2+1, 6] in the paper's entry order
    (a_1..a_6 and b_1..b_6).  Every sample is transformed once."""
    import torch

    shape = tuple(f.shape[2:])
    c = int(f.shape[1])
    C = 1 if c == 1 else 6
    nh = shape[0] * shape[1] * (shape[2] // 2 + 1)
    op = api.unocg_uno_create(c, *shape)
    ab = torch.zeros(2 * nh * C, dtype=torch.float32, device=f.device)
    n = f.shape[0]
    for s0 in range(0, n, chunk):
        fb = f[s0:s0 + chunk].contiguous()
        ub = u[s0:s0 + chunk].contiguous()
        api.unocg_uno_features_dev(op, fb.shape[0], fb, ub, ab, accumulate=s0 > 0)
    torch.cuda.synchronize()
    api.unocg_uno_destroy(op)
    abh = ab.cpu().numpy().astype(np.float64).reshape(2, shape[0], shape[1], shape[2] // 2 + 1, C)
    if c == 1:
        abh = abh[..., 0]
    return abh[0] / n, 2.0 * abh[1] / n


def _mode_index(shape, M: int):
    N1, N2, _ = shape
    ms = mode_set(M)
    return (np.array([k1 % N1 for k1, _, _ in ms]), np.array([k2 % N2 for _, k2, _ in ms]),
            np.array([k3 for _, _, k3 in ms]))


def _gather(a, b, M: int, shape3, C: int):
    """Features at the modes of K_M (``_mode_index`` order) and their sums over all other modes of
    the half grid (multiplicities included)."""
    i1, i2, i3 = _mode_index(shape3, M)
    ak, bk = a[i1, i2, i3].reshape(-1, C), b[i1, i2, i3].reshape(-1, C)
    a_rest = a.reshape(-1, C).sum(axis=0) - ak.sum(axis=0)
    b_rest = b.reshape(-1, C).sum(axis=0) - bk.sum(axis=0)
    return ak, bk, a_rest, b_rest


def second_order_modes(a, b, M: int, w0, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 (second-order training, c = 1) for the paper's layout, on the device
    (``unocg_newton_*``): Newton-Raphson on w = [w_0; w_1 .. w_n] for L = sum_k a_k v_k^2 - b_k v_k
    (v_k = w_0^2 + w_i^2 on the i-th mode of K_M, w_0^2 elsewhere) from the features a, b
    [N1, N2, N3/2+1]; the arrow-shaped Hessian solved by its Schur complement, Levenberg-Marquardt
    damping.  Returns (w [1 + n_modes, 1], loss history without the constant delta)."""
    shape = a.shape[:2] + (2 * (a.shape[2] - 1),)
    ak, bk, ar, br = _gather(a, b, M, shape, 1)
    return api.unocg_newton_run(1, ak, bk, ar, br, np.asarray(w0).reshape(-1, 1), iters, tol)


def second_order_modes_c3(a, b, M: int, w0, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 for c = 3 (App. C) on the paper's weight layout, on the device: Newton-Raphson
    on w = [w_0; w_1 .. w_n] (six psi parameters each, Q = L L^T) from the features a, b
    [N1, N2, N3/2+1, 6].  Returns (w [1 + n_modes, 6], loss history without delta)."""
    shape = a.shape[:2] + (2 * (a.shape[2] - 1),)
    ak, bk, ar, br = _gather(a, b, M, shape, 6)
    return api.unocg_newton_run(3, ak, bk, ar, br, np.asarray(w0).reshape(-1, 6), iters, tol)


# ---------------------------------------------------------------------------------------------
# 2D problems (Sec. 6 with d = 2), c = 1 (thermal) and c = 2 (plane strain, Eq. (local-param-2)).
# The library solves a 2D cell as the x1-invariant 3D problem on `layers` voxels along a
# periodic axis 1 (solver.Homogenization2D: 2D axes 1, 2 are 3D axes 2, 3; 2D components x, y
# are 3D components 2, 3).  Every field of such a solve has Fourier content only at k1 = 0,
# where the unitary 3D transform is sqrt(layers) times the 2D one; the 2D UNO is therefore the
# 3D operator whose blocks at (0, k1', k2') are the 2D blocks (embedded, with the extrusion
# component decoupled) and whose other blocks are the embedded bypass.

_L2 = ((0, 0), (1, 1), (1, 0))   # positions of w1, w2, w3 in L (Eq. (local-param-2))
_ORDER2 = ((0, 0), (1, 1), (0, 1))  # entries v1 = Q_xx, v2 = Q_yy, v3 = Q_xy (Sec. 5.4)


def mode_set_2d(M: int):
    """Learned modes of the periodic row of Table (fnocg-mode-selection-2d), d = 2:
    [-M, M] x [0, M] minus {0}, ordered k1 (from -M), then k2."""
    return [(k1, k2) for k1 in range(-M, M + 1) for k2 in range(0, M + 1) if (k1, k2) != (0, 0)]


def psi2(w, c: int) -> np.ndarray:
    """Local parametrization for c = 1 (w^2) and c = 2 (L L^T, L = [[w1, 0], [w3, w2]])."""
    w = np.asarray(w, dtype=np.float64)
    if c == 1:
        return (w[..., 0] ** 2)[..., None, None]
    L = np.zeros(w.shape[:-1] + (2, 2))
    for i, (r, q) in enumerate(_L2):
        L[..., r, q] = w[..., i]
    return L @ np.swapaxes(L, -1, -2)


def _blocks_2d_full(w, M: int, shape2, c: int) -> np.ndarray:
    """2D blocks [N1, N2, c, c] of the bypass-plus-modes weights on the full grid: modes with
    k2 > 0 give their block to the conjugate (-k1, -k2); on the line k2 = 0 the blocks of
    (k1, 0) and (-k1, 0) are averaged so that the operator is real."""
    N1, N2 = shape2
    if not (2 * M < N1 and 2 * M < N2):
        raise ValueError("mode set larger than the 2D grid")
    C = 1 if c == 1 else 3
    w = np.asarray(w, dtype=np.float64).reshape(-1, C)
    B0 = psi2(w[0], c)
    Q = np.broadcast_to(B0, (N1, N2, c, c)).copy()
    ms = mode_set_2d(M)
    if len(ms) != w.shape[0] - 1:
        raise ValueError("weights do not match the mode set")
    for i, (k1, k2) in enumerate(ms):
        B = B0 + psi2(w[1 + i], c)
        Q[k1 % N1, k2] = B
        if k2 > 0:
            Q[(-k1) % N1, (-k2) % N2] = B
    line = Q[:, 0].copy()
    Q[:, 0] = 0.5 * (line + line[(-np.arange(N1)) % N1])
    return Q


def modes2d_blocks3d(w, M: int, shape2, layers: int, c: int, extrusion_weight=None) -> np.ndarray:
    """Block entries [layers, N1, N2/2+1, C3] (C3 = 1 or 6, the 3D paper order) of the extruded
    3D operator carrying the 2D bypass-plus-modes weights ``w`` (for ``unocg_set_uno_weights``
    with BLOCKS_HALFGRID on the extruded context).  c = 2: the extrusion component gets the
    diagonal entry ``extrusion_weight`` (default: half the trace of the 2D bypass block) and no
    coupling; plane-strain residuals have no such component, so it never acts."""
    N1, N2 = shape2
    n3h = N2 // 2 + 1
    Q2 = _blocks_2d_full(w, M, shape2, c)
    C = 1 if c == 1 else 3
    B0 = psi2(np.asarray(w, dtype=np.float64).reshape(-1, C)[0], c)
    if c == 1:
        out = np.broadcast_to(B0[0, 0], (layers, N1, n3h)).copy()
        out[0] = Q2[:, :n3h, 0, 0]
        return out[..., None]
    qe = 0.5 * float(np.trace(B0)) if extrusion_weight is None else float(extrusion_weight)
    Q3 = np.zeros((layers, N1, n3h, 3, 3))
    Q3[..., 0, 0] = qe
    Q3[..., 1:, 1:] = B0
    Q3[0, :, :, 1:, 1:] = Q2[:, :n3h]
    return np.stack([Q3[..., i, j] for (i, j) in _ORDER3], axis=-1)


def features_2d(f3, u3, layers: int, c: int, chunk: int = 64):
    """Features of Eq. (features-c-1) / Eq. (features-c-2) of 2D training data given as extruded
    3D fields (torch float32 [N_s, 1 or 3, layers, N1, N2] on the GPU, x1-invariant), from the
    GPU transform passes: the 3D features at k1 = 0, restricted to the in-plane entries and
    divided by `layers`.  Returns a, b [N1, N2/2+1, C] on the 2D half grid (multiplicity of the
    conjugate modes included: summing over it sums over the full 2D grid)."""
    a3, b3 = features(f3, u3, chunk=chunk)
    if c == 1:
        return a3[0][..., None] / layers, b3[0][..., None] / layers
    sel = [_ORDER3.index((1, 1)), _ORDER3.index((2, 2)), _ORDER3.index((1, 2))]
    return a3[0][..., sel] / layers, b3[0][..., sel] / layers


def second_order_modes_2d(a, b, M: int, w0, c: int, iters: int = 100, tol: float = 1e-12):
    """Algorithm 4 for 2D problems (c = 1, c = 2) on the paper's weight layout with the 2D mode
    set, on the device (``unocg_newton_*``).  ``a, b``: features on the 2D half grid
    [N1, N2/2+1, C] with multiplicities (``features_2d``).  The line k2 = 0 of the half grid
    holds (k1, 0) and (-k1, 0) with multiplicity 1 each; the other columns carry the conjugates
    through multiplicity 2.  Returns (w [1 + n, C], loss history without delta)."""
    N1 = a.shape[0]
    C = a.shape[-1]
    ms = mode_set_2d(M)
    i1 = np.array([k1 % N1 for k1, _ in ms], dtype=np.int64)
    i2 = np.array([k2 for _, k2 in ms], dtype=np.int64)
    ak, bk = a[i1, i2].reshape(-1, C), b[i1, i2].reshape(-1, C)
    ar = a.reshape(-1, C).sum(axis=0) - ak.sum(axis=0)
    br = b.reshape(-1, C).sum(axis=0) - bk.sum(axis=0)
    return api.unocg_newton_run(c, ak, bk, ar, br, np.asarray(w0).reshape(-1, C), iters, tol)


def reference_modes_2d(physics: int, props, shape2, M: int, layers: int = 4) -> np.ndarray:
    """Start weights for 2D training: the bypass from the smallest reference-medium block of the
    extruded grid's in-plane entries over k != 0 (c = 1: the smallest weight; c = 2: lambda I with
    lambda the smallest eigenvalue), each mode of K_M the rest of its reference block through the
    inverse of psi (Cholesky)."""
    h = reference_blocks_extruded(physics, props, shape2, layers)
    c = 1 if physics == _lib.THERMAL else 2
    N1, N2 = shape2
    ms = mode_set_2d(M)
    if c == 1:
        q = h[0, :, :, 0].copy()                # [N1, N2h] at k_ext = 0
        q[0, 0] = np.inf
        qmin = float(np.min(q))
        w = [np.sqrt(qmin)]
        for (k1, k2) in ms:
            w.append(np.sqrt(max(q[k1 % N1, k2] - qmin, 0.0)))
        return np.array(w)[:, None]
    Q = np.zeros(h.shape[:3] + (3, 3))
    for e, (i, j) in enumerate(_ORDER3):
        Q[..., i, j] = Q[..., j, i] = h[..., e]
    B = Q[0][..., 1:, 1:]                        # [N1, N2h, 2, 2] in-plane blocks at k_ext = 0
    ev = np.linalg.eigvalsh(B.reshape(-1, 2, 2))[1:]
    lam = float(ev.min())
    out = [[np.sqrt(lam), np.sqrt(lam), 0.0]]
    for (k1, k2) in ms:
        R = B[k1 % N1, k2] - lam * np.eye(2)
        R = 0.5 * (R + R.T) + 1e-300 * np.eye(2)
        ev2, V = np.linalg.eigh(R)
        R = (V * np.maximum(ev2, 0.0)) @ V.T + 1e-14 * lam * np.eye(2)
        L = np.linalg.cholesky(R)
        out.append([L[0, 0], L[1, 1], L[1, 0]])
    return np.array(out)


def reference_blocks_extruded(physics: int, props, shape2, layers: int = 4) -> np.ndarray:
    """Reference-medium block entries [layers, N1, N2/2+1, C3] of the extruded grid of a 2D cell
    (arithmetic-mean medium of the phase properties), read back from the library."""
    from .solver import Homogenization2D
    h = Homogenization2D(physics, shape2, layers=layers)
    h.set_microstructure(np.zeros(shape2, dtype=np.uint8), 1)
    p = np.asarray(props, dtype=np.float64)
    if physics == _lib.THERMAL:
        h.set_phase_properties(np.array([float(np.mean(p))]))
    else:
        # the arithmetic means of the Lame constants, as (E, nu) of one phase
        lam = np.mean([E * nu / ((1 + nu) * (1 - 2 * nu)) for E, nu in p])
        mu = np.mean([E / (2 * (1 + nu)) for E, nu in p])
        h.set_phase_properties(np.array([[mu * (3 * lam + 2 * mu) / (lam + mu), lam / (2 * (lam + mu))]]))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    C3 = 1 if physics == _lib.THERMAL else 6
    n3h = shape2[1] // 2 + 1
    out = api.unocg_get_uno_weights(h.h.ctx, 0, layers * shape2[0] * n3h, C3)
    h.close()
    return np.asarray(out).reshape(layers, shape2[0], n3h, C3)
