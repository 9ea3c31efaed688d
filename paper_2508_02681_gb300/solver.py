"""Convenience wrappers over the C ABI: a homogenization solver object and the UNO operator as a
``torch.autograd.Function`` (forward and backward both run in the library's kernels)."""
from __future__ import annotations

import numpy as np

from . import _lib, api


def _tuning_cache(path, key, measure, apply):
    """Autotune cache (a JSON file of key -> chosen setting): apply the stored setting for
    ``key``, else ``measure()`` -> (setting, table), store and apply it.  Returns (setting,
    table or None)."""
    import json
    import os
    cache = {}
    if path and os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
    if key in cache:
        apply(cache[key])
        return cache[key], None
    setting, table = measure()
    apply(setting)
    if path:
        cache[key] = setting
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return setting, table


class Homogenization:
    """One context: ``batch`` instances of an ``n1 x n2 x n3`` periodic voxel problem.

    ``physics``: ``_lib.THERMAL`` (kappa per phase) or ``_lib.ELASTIC`` ((E, nu) per phase).
    """

    def __init__(self, physics: int, shape, batch: int = 1, L0: float = 1.0):
        self.physics = physics
        self.c = 1 if physics == _lib.THERMAL else 3
        self.dim = 3 if physics == _lib.THERMAL else 6
        self.shape = tuple(int(s) for s in shape)
        self.batch = batch
        self.n = int(np.prod(self.shape))
        self.ctx = api.unocg_create(physics, batch, *self.shape, L0)
        self.n_loads = 0
        self.n_phases = 0

    def close(self):
        if self.ctx is not None:
            api.unocg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_microstructure(self, phase, n_phases: int):
        api.unocg_set_microstructure(self.ctx, phase, n_phases)
        self.n_phases = n_phases

    def set_phase_properties(self, props):
        api.unocg_set_phase_properties(self.ctx, props)

    def set_macro_load(self, loads):
        loads = np.atleast_2d(np.asarray(loads, dtype=np.float64))
        api.unocg_set_macro_load(self.ctx, loads)
        self.n_loads = loads.shape[0]

    def set_uno_weights(self, kind=_lib.W_REFERENCE_MEDIUM, w=None, spd_eps: float = 0.0):
        api.unocg_set_uno_weights(self.ctx, kind, w, spd_eps)

    def set_uno_modes(self, M: int, w, spd_eps: float = 0.0):
        """The paper's weight layout: bypass ``w[0]`` plus ``w[1 + i]`` on the i-th mode of K_M."""
        api.unocg_set_uno_modes(self.ctx, M, w, spd_eps)

    def solve(self, raise_on_error: bool = True, **opts) -> api.Info:
        return api.unocg_solve(self.ctx, api.make_opts(**opts), self.batch * self.n_loads, raise_on_error)

    def autotune(self, cache: str | None = None, reps: int = 3, **opts):
        """Radix order of the Stockham plans and loop driver (``use_graph=3`` then takes it),
        measured on this context's inputs or read from the JSON ``cache``."""
        o = api.make_opts(**opts)
        key = f"periodic:{self.physics}:{list(self.shape)}:{self.batch}x{self.n_loads}:{o.precision}:{o.precond}"

        def measure():
            t = api.unocg_autotune(self.ctx, o, reps)
            i = int(np.nanargmin(t))
            return [i // 2, i % 2 + 1], t

        return _tuning_cache(cache, key, measure, lambda s: api.unocg_set_tuning(self.ctx, int(s[0]), int(s[1])))

    def fluctuation(self, instance: int = 0, load: int = 0) -> np.ndarray:
        """Zero-mean fluctuation, interleaved ``[n * c]`` (the paper's DOF order)."""
        return api.unocg_get_fluctuation(self.ctx, instance, load, self.n * self.c)

    def effective_tensor(self) -> np.ndarray:
        return api.unocg_get_effective_tensor(self.ctx, self.batch, self.dim, self.n_loads)

    def sensitivity(self) -> np.ndarray:
        n_props = self.n_phases * (1 if self.physics == _lib.THERMAL else 2)
        return api.unocg_get_sensitivity(self.ctx, self.batch, n_props, self.n_loads)



class DirichletHomogenization:
    """One context of the Dirichlet problem (fluctuation zero on the boundary, sine transform):
    ``batch`` instances of an ``n1 x n2 x n3`` voxel grid with ``(n1-1)(n2-1)(n3-1)`` free nodes.
    ``bc`` (per axis 1 = Dirichlet faces, 0 = periodic) selects mixed boundary conditions."""

    def __init__(self, physics: int, shape, batch: int = 1, L0: float = 1.0, bc=(1, 1, 1)):
        self.physics = physics
        self.c = 1 if physics == _lib.THERMAL else 3
        self.dim = 3 if physics == _lib.THERMAL else 6
        self.shape = tuple(int(s) for s in shape)
        self.bc = tuple(int(b) for b in bc)
        self.free_shape = tuple(s - b for s, b in zip(self.shape, self.bc))
        self.nf = int(np.prod(self.free_shape))
        self.batch = batch
        self.ctx = api.unocg_dir_create(physics, batch, *self.shape, L0, bc=self.bc)
        self.n_loads = 0

    def close(self):
        if self.ctx is not None:
            api.unocg_dir_destroy(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def set_microstructure(self, phase, n_phases: int):
        api.unocg_dir_set_microstructure(self.ctx, phase, n_phases)

    def set_phase_properties(self, props):
        api.unocg_dir_set_phase_properties(self.ctx, props)

    def set_macro_load(self, loads):
        loads = np.atleast_2d(np.asarray(loads, dtype=np.float64))
        api.unocg_dir_set_macro_load(self.ctx, loads)
        self.n_loads = loads.shape[0]

    def set_uno_weights(self, kind=_lib.W_REFERENCE_MEDIUM, w=None, spd_eps: float = 0.0):
        api.unocg_dir_set_uno_weights(self.ctx, kind, w, spd_eps)

    def set_uno_modes(self, M: int, w, spd_eps: float = 0.0):
        """Bypass ``w[0]`` plus ``w[1 + i]`` on the i-th mode of [0, 2M]^3."""
        api.unocg_dir_set_uno_modes(self.ctx, M, w, spd_eps)

    def uno_weights(self, instance: int = 0) -> np.ndarray:
        C_ = 1 if self.c == 1 else 6
        return api.unocg_dir_get_uno_weights(self.ctx, instance, self.nf, C_).reshape(self.free_shape + (C_,))

    def solve(self, raise_on_error: bool = True, **opts) -> api.Info:
        opts.setdefault("flexible", 0)
        return api.unocg_dir_solve(self.ctx, api.make_opts(**opts), self.batch * self.n_loads, raise_on_error)

    def autotune(self, cache: str | None = None, reps: int = 3, **opts):
        """Pass engines (register / shared-memory plane / separate passes; register or
        shared-memory axis-1 pass) for the solve's precision, measured or read from ``cache``."""
        opts.setdefault("flexible", 0)
        o = api.make_opts(**opts)
        key = (f"dirichlet:{self.physics}:{list(self.shape)}:{list(self.bc)}:{self.batch}x{self.n_loads}:"
               f"{o.precision}:{o.precond}")

        def measure():
            t = api.unocg_dir_autotune(self.ctx, o, reps)
            i = int(np.nanargmin(t))
            return [i // 2, i % 2], t

        return _tuning_cache(cache, key, measure,
                             lambda s: api.unocg_dir_set_tuning(self.ctx, o.precision, int(s[0]), int(s[1])))

    def fluctuation(self, instance: int = 0, load: int = 0) -> np.ndarray:
        """Fluctuation on the free nodes, interleaved ``[nf * c]``."""
        return api.unocg_dir_get_fluctuation(self.ctx, instance, load, self.nf * self.c)

    def effective_tensor(self) -> np.ndarray:
        return api.unocg_dir_get_effective_tensor(self.ctx, self.batch, self.dim, self.n_loads)



class Homogenization2D:
    """2D cells (Sec. 6 with d = 2: thermal, or plane-strain elasticity with (E, nu) per phase)
    solved as the x3-invariant 3D problem: the cell becomes axes 2 and 3 of a 3D grid with
    ``layers`` voxels along a periodic axis 1.  By uniqueness the 3D solution does not vary
    along that axis, equals the bilinear 2D solution on every layer (plane strain: u along the
    extrusion vanishes), and the in-plane averages are the 2D ones; the UNO restricted to the
    x3-invariant fields (Fourier mode 0 along the extrusion) is the 2D one.

    ``bc``: per 2D axis 1 (Dirichlet faces) or 0 (periodic).  Loads: thermal (g1, g2); elastic
    Mandel (eps11, eps22, sqrt2 eps12).  Microstructures [batch][N1][N2]."""

    def __init__(self, physics: int, shape, batch: int = 1, L0: float = 1.0, bc=(0, 0), layers=None):
        self.physics = physics
        self.shape2 = tuple(int(s) for s in shape)
        self.bc2 = tuple(int(b) for b in bc)
        self.c2 = 1 if physics == _lib.THERMAL else 2
        self.dim2 = 2 if physics == _lib.THERMAL else 3
        self.batch = batch
        periodic = not any(self.bc2)
        self.layers = layers or (4 if periodic else 2)
        shape3 = (self.layers,) + self.shape2
        # the voxel edge follows the 2D axis 1 (axis 2 of the 3D grid): h = L0 / N1
        L03 = L0 * self.layers / self.shape2[0]
        if periodic:
            self.h = Homogenization(physics, shape3, batch=batch, L0=L03)
        else:
            self.h = DirichletHomogenization(physics, shape3, batch=batch, L0=L03, bc=(0,) + self.bc2)
        self.free2 = tuple(n - b for n, b in zip(self.shape2, self.bc2))
        # 2D components / Mandel rows inside the 3D ones (axes 2 and 3)
        self._comp = [0] if self.c2 == 1 else [1, 2]
        self._rows = [1, 2] if self.c2 == 1 else [1, 2, 5]

    def close(self):
        self.h.close()

    def set_microstructure(self, phase, n_phases: int):
        ph = np.asarray(phase, dtype=np.uint8).reshape((self.batch,) + self.shape2)
        self.h.set_microstructure(np.repeat(ph[:, None], self.layers, axis=1), n_phases)

    def set_phase_properties(self, props):
        self.h.set_phase_properties(props)

    def set_macro_load(self, loads):
        loads = np.atleast_2d(np.asarray(loads, dtype=np.float64))
        l3 = np.zeros((loads.shape[0], 3 if self.c2 == 1 else 6))
        l3[:, self._rows] = loads
        self.h.set_macro_load(l3)
        self.n_loads = loads.shape[0]

    def set_uno_weights(self, kind=_lib.W_REFERENCE_MEDIUM, w=None, spd_eps: float = 0.0):
        self.h.set_uno_weights(kind, w, spd_eps)

    def solve(self, raise_on_error: bool = True, **opts) -> api.Info:
        return self.h.solve(raise_on_error=raise_on_error, **opts)

    def fluctuation(self, instance: int = 0, load: int = 0) -> np.ndarray:
        """2D fluctuation on the free nodes (layer 0), interleaved ``[n2d * c]``."""
        u = self.h.fluctuation(instance, load)
        c3 = 1 if self.c2 == 1 else 3
        free3 = (self.layers,) + self.free2
        return np.ascontiguousarray(u.reshape(free3 + (c3,))[0][..., self._comp]).ravel()

    def effective_tensor(self) -> np.ndarray:
        """``[batch][dim2][n_loads]`` in-plane averaged flux / stress."""
        return self.h.effective_tensor()[:, self._rows, :]


class UnevenBatch:
    """Many instances of possibly different grid sizes (the serving-style batch): the instances
    of one size share a batched context (per-(instance, load) convergence masks), and the
    contexts of all sizes are solved together by ``unocg_batch_solve``."""

    def __init__(self, physics: int, phases, props, loads, n_phases: int = 2):
        self.physics = physics
        self.loads = np.atleast_2d(np.asarray(loads, dtype=np.float64))
        groups: dict[tuple, list[int]] = {}
        for i, ph in enumerate(phases):
            groups.setdefault(tuple(ph.shape), []).append(i)
        self.n = len(phases)
        self.groups = []
        for shape, idx in sorted(groups.items()):
            h = Homogenization(physics, shape, batch=len(idx))
            h.set_microstructure(np.stack([np.asarray(phases[i], dtype=np.uint8) for i in idx]), n_phases)
            h.set_phase_properties(np.stack([np.asarray(props[i], dtype=np.float64) for i in idx]))
            h.set_macro_load(self.loads)
            h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
            self.groups.append((idx, h))

    def solve(self, **opts):
        """Returns per-instance (iterations [L], true relative residuals [L], status)."""
        hs = [h for _, h in self.groups]
        infos = api.unocg_batch_solve([h.ctx for h in hs], api.make_opts(**opts),
                                      [h.batch * self.loads.shape[0] for h in hs])
        L = self.loads.shape[0]
        out = [None] * self.n
        for (idx, _), info in zip(self.groups, infos):
            for j, i in enumerate(idx):
                out[i] = (info.iters[j * L:(j + 1) * L].copy(), info.true_rel_res[j * L:(j + 1) * L].copy(),
                          info.load_status[j * L:(j + 1) * L].copy())
        return out

    def effective_tensors(self) -> np.ndarray:
        res = [None] * self.n
        for idx, h in self.groups:
            C = h.effective_tensor()
            for j, i in enumerate(idx):
                res[i] = C[j]
        return np.stack(res)

    def close(self):
        for _, h in self.groups:
            h.close()
        self.groups = []


def uno_function(modes_M: int | None = None):
    """``torch.autograd.Function`` for ``s = P_theta r`` on a batch ``[B, c, N1, N2, N3]``.
    theta: per-mode parameters ``[N1, N2, N3/2+1, C]``, or with ``modes_M`` the paper's layout
    ``[1 + n_modes, C]`` (bypass, then the modes of K_M)."""
    import torch

    def set_weights(op, theta):
        if modes_M is None:
            api.unocg_uno_set_theta_dev(op, theta)
        else:
            api.unocg_uno_set_modes_dev(op, modes_M, theta)

    class UnoApply(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r, theta, op):
            r = r.contiguous()
            set_weights(op, theta)
            s = torch.empty_like(r)
            api.unocg_uno_apply_dev(op, r.shape[0], r, s)
            ctx.save_for_backward(r, theta)
            ctx.op = op
            return s

        @staticmethod
        def backward(ctx, gs):
            r, theta = ctx.saved_tensors
            gs = gs.contiguous()
            gr = torch.empty_like(r) if ctx.needs_input_grad[0] else None
            gt = torch.empty_like(theta) if ctx.needs_input_grad[1] else None
            set_weights(ctx.op, theta)
            api.unocg_uno_backward_dev(ctx.op, r.shape[0], r, gs, gr, gt)
            return gr, gt, None

    return UnoApply
