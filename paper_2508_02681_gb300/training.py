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


def train(f, u, theta0, epochs: int, batch: int = 64, lr: float = 1e-2, seed: int = 0,
          modes_M: int | None = None):
    """Adam on the MSE loss; returns (theta tensor, per-epoch mean losses).  With ``modes_M``
    theta0 is in the paper's layout ``[1 + n_modes, 1]`` (see ``reference_modes``)."""
    import torch

    shape = tuple(f.shape[2:])
    op = api.unocg_uno_create(1, *shape)
    Fn = uno_function(modes_M)
    theta = torch.tensor(theta0, dtype=torch.float32, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = f.shape[0]
    for _ in range(epochs):
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
    api.unocg_uno_destroy(op)
    return theta.detach(), losses
