"""Python entry points with the names of the C ABI (``include/unocg.h``).

Host arrays are NumPy arrays; device arrays are torch CUDA tensors (PyTorch supplies device
memory and streams only).  Every function marshals its arguments and calls the library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import SolveInfo, SolveOpts, UnocgError


def _check(ctx, rc):
    if rc != _lib.OK:
        lib = _lib.load()
        msg = lib.unocg_last_error(ctx).decode() if ctx else ""
        raise UnocgError(rc, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# values per field of each live periodic context (c * N1 * N2 * N3), for the checks of the
# device-pointer entry points
_FIELD_VALUES: dict[int, int] = {}


def _device_field(ctx, t, name: str):
    """Raise ValueError unless ``t`` is a contiguous float64 CUDA tensor of one field of ``ctx``
    (c * N1 * N2 * N3 values): the library reads and writes exactly that many values."""
    need = _FIELD_VALUES.get(ctx.value)
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: a CUDA tensor is required")
    import torch
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: float64 required, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if need is not None and t.numel() != need:
        raise ValueError(f"{name}: {t.numel()} values, the context's field has {need}")
    return C.c_void_p(t.data_ptr())


def unocg_create(physics: int, batch: int, n1: int, n2: int, n3: int, L0: float = 1.0):
    lib = _lib.load()
    h = C.c_void_p()
    rc = lib.unocg_create(C.byref(h), physics, batch, n1, n2, n3, L0)
    if rc != _lib.OK:
        msg = lib.unocg_last_error(h).decode() if h.value else "invalid arguments or unsupported grid"
        if h.value:
            lib.unocg_destroy(h)
        raise UnocgError(rc, msg)
    _FIELD_VALUES[h.value] = (1 if physics == _lib.THERMAL else 3) * n1 * n2 * n3
    return h


def unocg_destroy(ctx):
    _FIELD_VALUES.pop(ctx.value, None)
    _lib.load().unocg_destroy(ctx)


def unocg_set_wait_limit(ctx, seconds: float):
    _check(ctx, _lib.load().unocg_set_wait_limit(ctx, seconds))


def unocg_set_stream(ctx, stream=None):
    _check(ctx, _lib.load().unocg_set_stream(ctx, _stream(stream) if stream is not None else None))


def unocg_set_microstructure(ctx, phase: np.ndarray, n_phases: int):
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    _check(ctx, _lib.load().unocg_set_microstructure(ctx, _ptr(ph), n_phases))


def unocg_set_microstructure_dev(ctx, phase_dev, n_phases: int, stream=None):
    _check(ctx, _lib.load().unocg_set_microstructure_dev(ctx, C.c_void_p(phase_dev.data_ptr()), n_phases, _stream(stream)))


def unocg_set_phase_properties(ctx, props: np.ndarray):
    p = np.ascontiguousarray(props, dtype=np.float64)
    _check(ctx, _lib.load().unocg_set_phase_properties(ctx, _ptr(p)))


def unocg_set_macro_load(ctx, loads: np.ndarray):
    l2 = np.ascontiguousarray(np.atleast_2d(loads), dtype=np.float64)
    _check(ctx, _lib.load().unocg_set_macro_load(ctx, l2.shape[0], _ptr(l2)))


def unocg_set_uno_weights(ctx, kind: int, w: np.ndarray | None = None, spd_eps: float = 0.0):
    if w is None:
        _check(ctx, _lib.load().unocg_set_uno_weights(ctx, kind, None, _lib.DTYPE_F64, spd_eps))
        return
    a = np.ascontiguousarray(w)
    dt = _lib.DTYPE_F64 if a.dtype == np.float64 else _lib.DTYPE_F32
    if dt == _lib.DTYPE_F32:
        a = a.astype(np.float32)
    _check(ctx, _lib.load().unocg_set_uno_weights(ctx, kind, _ptr(a), dt, spd_eps))


def unocg_set_uno_modes(ctx, M: int, w: np.ndarray, spd_eps: float = 0.0):
    a = np.ascontiguousarray(w)
    dt = _lib.DTYPE_F64 if a.dtype == np.float64 else _lib.DTYPE_F32
    if dt == _lib.DTYPE_F32:
        a = a.astype(np.float32)
    _check(ctx, _lib.load().unocg_set_uno_modes(ctx, M, _ptr(a), dt, spd_eps))


def unocg_get_uno_weights(ctx, instance: int, n_modes: int, C_: int) -> np.ndarray:
    out = np.empty(n_modes * C_, dtype=np.float64)
    _check(ctx, _lib.load().unocg_get_uno_weights(ctx, instance, _ptr(out)))
    return out


def make_opts(tol=1e-6, max_iter=10000, precond=_lib.PRECOND_UNO, precision=_lib.FP64,
              replace_every=50, flexible=None, use_graph=3, replace_drop=1e-3) -> SolveOpts:
    if flexible is None:
        flexible = 1 if precision == _lib.MIXED else 0
    return SolveOpts(tol, max_iter, precond, precision, replace_every, flexible, use_graph, replace_drop)


class Info:
    """Per-(instance, load) results of a solve."""

    def __init__(self, n: int):
        self.iters = np.zeros(n, dtype=np.int32)
        self.rel_res = np.zeros(n)
        self.true_rel_res = np.zeros(n)
        self.load_status = np.zeros(n, dtype=np.int32)
        self.c = SolveInfo(0, 0, self.iters.ctypes.data_as(C.POINTER(C.c_int)),
                           self.rel_res.ctypes.data_as(C.POINTER(C.c_double)),
                           self.true_rel_res.ctypes.data_as(C.POINTER(C.c_double)),
                           self.load_status.ctypes.data_as(C.POINTER(C.c_int)), 0, 0)

    @property
    def status(self):
        return self.c.status

    @property
    def checks(self):
        return self.c.checks

    @property
    def replacements(self):
        return self.c.replacements


def unocg_solve(ctx, opts: SolveOpts, n_results: int, raise_on_error: bool = True) -> Info:
    info = Info(n_results)
    rc = _lib.load().unocg_solve(ctx, C.byref(opts), C.byref(info.c))
    if raise_on_error:
        _check(ctx, rc)
    return info


def unocg_solve_async(ctx, opts: SolveOpts):
    _check(ctx, _lib.load().unocg_solve_async(ctx, C.byref(opts)))


def unocg_solve_wait(ctx, n_results: int, raise_on_error: bool = True) -> Info:
    info = Info(n_results)
    rc = _lib.load().unocg_solve_wait(ctx, C.byref(info.c))
    if raise_on_error:
        _check(ctx, rc)
    return info


def unocg_get_fluctuation(ctx, instance: int, load: int, n_values: int) -> np.ndarray:
    out = np.empty(n_values, dtype=np.float64)
    _check(ctx, _lib.load().unocg_get_fluctuation(ctx, instance, load, _ptr(out)))
    return out


def unocg_get_fluctuation_dev(ctx, instance: int, load: int, out_dev, stream=None):
    out = _device_field(ctx, out_dev, "out_dev")
    _check(ctx, _lib.load().unocg_get_fluctuation_dev(ctx, instance, load, out, _stream(stream)))


def unocg_get_effective_tensor(ctx, batch: int, dim: int, n_loads: int) -> np.ndarray:
    out = np.empty((batch, dim, n_loads), dtype=np.float64)
    _check(ctx, _lib.load().unocg_get_effective_tensor(ctx, _ptr(out)))
    return out


def unocg_get_sensitivity(ctx, batch: int, n_props: int, n_loads: int) -> np.ndarray:
    out = np.empty((batch, n_props, n_loads, n_loads), dtype=np.float64)
    _check(ctx, _lib.load().unocg_get_sensitivity(ctx, _ptr(out)))
    return out


def unocg_batch_solve(ctxs, opts: SolveOpts, n_results=None):
    """Solve several contexts together; with ``n_results`` (results per context) returns their
    ``Info`` objects."""
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    infos = None
    carr = None
    if n_results is not None:
        infos = [Info(n) for n in n_results]
        carr = (SolveInfo * len(ctxs))(*[i.c for i in infos])
    rc = _lib.load().unocg_batch_solve(len(ctxs), arr, C.byref(opts), carr)
    if rc != _lib.OK:
        raise UnocgError(rc, "batch solve failed")
    if infos is not None:
        for i, ci in zip(infos, carr):
            i.c = ci
    return infos


def unocg_apply_K_dev(ctx, instance: int, d_dev, p_dev, stream=None):
    d = _device_field(ctx, d_dev, "d_dev")
    p = _device_field(ctx, p_dev, "p_dev")
    _check(ctx, _lib.load().unocg_apply_K_dev(ctx, instance, d, p, _stream(stream)))


def _device_field32(ctx, t, name: str):
    """As ``_device_field`` for float32 fields."""
    import torch
    if not getattr(t, "is_cuda", False) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous float32 CUDA tensor is required")
    need = _FIELD_VALUES.get(ctx.value)
    if need is not None and t.numel() != need:
        raise ValueError(f"{name}: {t.numel()} values, the context's field has {need}")
    return C.c_void_p(t.data_ptr())


def unocg_apply_K32_dev(ctx, instance: int, d_dev, p_dev, stream=None):
    d = _device_field32(ctx, d_dev, "d_dev")
    p = _device_field32(ctx, p_dev, "p_dev")
    _check(ctx, _lib.load().unocg_apply_K32_dev(ctx, instance, d, p, _stream(stream)))


def unocg_set_ku_tile(ctx, tile: int):
    _check(ctx, _lib.load().unocg_set_ku_tile(ctx, tile))


def unocg_get_ku_tile(ctx) -> int:
    out = C.c_int(0)
    _check(ctx, _lib.load().unocg_get_ku_tile(ctx, C.byref(out)))
    return out.value


def unocg_autotune_ku(ctx, reps: int = 20):
    """Times of the K d candidates (index 0: the earlier kernels, 1..8: TMA tile shapes, 9..16:
    vector-march shapes; NaN where unavailable) and the index kept."""
    times = np.zeros(17)
    best = C.c_int(0)
    _check(ctx, _lib.load().unocg_autotune_ku(ctx, reps, _ptr(times), C.byref(best)))
    return times, best.value


def unocg_apply_uno_dev(ctx, instance: int, r_dev, s_dev, stream=None):
    r = _device_field(ctx, r_dev, "r_dev")
    s = _device_field(ctx, s_dev, "s_dev")
    _check(ctx, _lib.load().unocg_apply_uno_dev(ctx, instance, r, s, _stream(stream)))


def unocg_apply_uno_dev_noalloc(ctx, instance: int, r_dev, s_dev, stream=None):
    r = _device_field(ctx, r_dev, "r_dev")
    s = _device_field(ctx, s_dev, "s_dev")
    _check(ctx, _lib.load().unocg_apply_uno_dev_noalloc(ctx, instance, r, s, _stream(stream)))


def unocg_rhs_dev(ctx, instance: int, load: int, f_dev, stream=None):
    f = _device_field(ctx, f_dev, "f_dev")
    _check(ctx, _lib.load().unocg_rhs_dev(ctx, instance, load, f, _stream(stream)))


def unocg_profile_iteration(ctx, opts: SolveOpts, reps: int = 10) -> np.ndarray:
    out = np.zeros(4)
    _check(ctx, _lib.load().unocg_profile_iteration(ctx, C.byref(opts), reps, _ptr(out), 4))
    return out


# ---------------------------------------------------------------- standalone UNO operator
def _ucheck(op, rc):
    if rc != _lib.OK:
        raise UnocgError(rc, _lib.load().unocg_uno_last_error(op).decode() if op else "")


def unocg_uno_create(c: int, n1: int, n2: int, n3: int):
    h = C.c_void_p()
    _ucheck(None, _lib.load().unocg_uno_create(C.byref(h), c, n1, n2, n3))
    return h


def unocg_uno_destroy(op):
    _lib.load().unocg_uno_destroy(op)


def unocg_uno_set_theta_dev(op, theta_dev, stream=None):
    _ucheck(op, _lib.load().unocg_uno_set_theta_dev(op, C.c_void_p(theta_dev.data_ptr()), _stream(stream)))


def unocg_uno_set_modes_dev(op, M: int, w_dev, stream=None):
    _ucheck(op, _lib.load().unocg_uno_set_modes_dev(op, M, C.c_void_p(w_dev.data_ptr()), _stream(stream)))


def unocg_uno_features_dev(op, batch: int, f_dev, u_dev, ab_dev, accumulate: bool = False, stream=None):
    _ucheck(op, _lib.load().unocg_uno_features_dev(op, batch, C.c_void_p(f_dev.data_ptr()),
                                                   C.c_void_p(u_dev.data_ptr()), C.c_void_p(ab_dev.data_ptr()),
                                                   1 if accumulate else 0, _stream(stream)))


def unocg_uno_apply_dev(op, batch: int, r_dev, s_dev, stream=None):
    _ucheck(op, _lib.load().unocg_uno_apply_dev(op, batch, C.c_void_p(r_dev.data_ptr()),
                                                C.c_void_p(s_dev.data_ptr()), _stream(stream)))


def unocg_uno_backward_dev(op, batch: int, r_dev, gs_dev, gr_dev, gtheta_dev, stream=None):
    _ucheck(op, _lib.load().unocg_uno_backward_dev(
        op, batch, C.c_void_p(r_dev.data_ptr()), C.c_void_p(gs_dev.data_ptr()),
        C.c_void_p(gr_dev.data_ptr()) if gr_dev is not None else None,
        C.c_void_p(gtheta_dev.data_ptr()) if gtheta_dev is not None else None, _stream(stream)))


# ---------------------------------------------------------------- Dirichlet boundary conditions
def _dcheck(ctx, rc):
    if rc != _lib.OK:
        lib = _lib.load()
        msg = lib.unocg_dir_last_error(ctx).decode() if ctx else ""
        raise UnocgError(rc, msg)


def unocg_dir_create(physics: int, batch: int, n1: int, n2: int, n3: int, L0: float = 1.0, bc=None):
    """``bc``: per axis 1 (Dirichlet faces) or 0 (periodic); None = Dirichlet on every axis."""
    lib = _lib.load()
    h = C.c_void_p()
    if bc is None:
        rc = lib.unocg_dir_create(C.byref(h), physics, batch, n1, n2, n3, L0)
    else:
        b = np.ascontiguousarray([int(x) for x in bc], dtype=np.int32)
        rc = lib.unocg_dir_create_bc(C.byref(h), physics, batch, n1, n2, n3, L0, _ptr(b))
    if rc != _lib.OK:
        msg = lib.unocg_dir_last_error(h).decode() if h.value else "invalid arguments or unsupported grid"
        if h.value:
            lib.unocg_dir_destroy(h)
        raise UnocgError(rc, msg)
    return h


def unocg_dir_destroy(ctx):
    _lib.load().unocg_dir_destroy(ctx)


def unocg_dir_set_stream(ctx, stream):
    _dcheck(ctx, _lib.load().unocg_dir_set_stream(ctx, _stream(stream)))


def unocg_dir_set_microstructure(ctx, phase: np.ndarray, n_phases: int):
    a = np.ascontiguousarray(phase, dtype=np.uint8)
    _dcheck(ctx, _lib.load().unocg_dir_set_microstructure(ctx, _ptr(a), n_phases))


def unocg_dir_set_phase_properties(ctx, props: np.ndarray):
    a = np.ascontiguousarray(props, dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_set_phase_properties(ctx, _ptr(a)))


def unocg_dir_set_macro_load(ctx, loads: np.ndarray):
    a = np.ascontiguousarray(np.atleast_2d(loads), dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_set_macro_load(ctx, a.shape[0], _ptr(a)))


def unocg_dir_set_uno_weights(ctx, kind: int, w=None, spd_eps: float = 0.0):
    if w is None:
        _dcheck(ctx, _lib.load().unocg_dir_set_uno_weights(ctx, kind, None, _lib.DTYPE_F64, spd_eps))
        return
    a = np.ascontiguousarray(w, dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_set_uno_weights(ctx, kind, _ptr(a), _lib.DTYPE_F64, spd_eps))


def unocg_dir_set_uno_modes(ctx, M: int, w, spd_eps: float = 0.0):
    a = np.ascontiguousarray(w, dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_set_uno_modes(ctx, M, _ptr(a), _lib.DTYPE_F64, spd_eps))


def unocg_dir_get_uno_weights(ctx, instance: int, n_modes: int, C_: int) -> np.ndarray:
    out = np.empty(n_modes * C_, dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_get_uno_weights(ctx, instance, _ptr(out)))
    return out


def unocg_dir_solve(ctx, opts: SolveOpts, n_results: int, raise_on_error: bool = True) -> Info:
    info = Info(n_results)
    rc = _lib.load().unocg_dir_solve(ctx, C.byref(opts), C.byref(info.c))
    if raise_on_error:
        _dcheck(ctx, rc)
    return info


def unocg_dir_solve_async(ctx, opts: SolveOpts):
    _dcheck(ctx, _lib.load().unocg_dir_solve_async(ctx, C.byref(opts)))


def unocg_dir_solve_wait(ctx, n_results: int, raise_on_error: bool = True) -> Info:
    info = Info(n_results)
    rc = _lib.load().unocg_dir_solve_wait(ctx, C.byref(info.c))
    if raise_on_error:
        _dcheck(ctx, rc)
    return info


def unocg_dir_get_fluctuation(ctx, instance: int, load: int, n_values: int) -> np.ndarray:
    out = np.empty(n_values, dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_get_fluctuation(ctx, instance, load, _ptr(out)))
    return out


def unocg_dir_get_fluctuation_dev(ctx, instance: int, load: int, out_dev, stream=None):
    _dcheck(ctx, _lib.load().unocg_dir_get_fluctuation_dev(ctx, instance, load, C.c_void_p(out_dev.data_ptr()),
                                                           _stream(stream)))


def unocg_dir_get_effective_tensor(ctx, batch: int, dim: int, n_loads: int) -> np.ndarray:
    out = np.empty((batch, dim, n_loads), dtype=np.float64)
    _dcheck(ctx, _lib.load().unocg_dir_get_effective_tensor(ctx, _ptr(out)))
    return out


def unocg_dir_apply_K_dev(ctx, instance: int, p_dev, q_dev, stream=None):
    _dcheck(ctx, _lib.load().unocg_dir_apply_K_dev(ctx, instance, C.c_void_p(p_dev.data_ptr()),
                                                   C.c_void_p(q_dev.data_ptr()), _stream(stream)))


def unocg_dir_apply_uno_dev(ctx, instance: int, r_dev, s_dev, stream=None):
    _dcheck(ctx, _lib.load().unocg_dir_apply_uno_dev(ctx, instance, C.c_void_p(r_dev.data_ptr()),
                                                     C.c_void_p(s_dev.data_ptr()), _stream(stream)))


# ---------------------------------------------------------------- tuning
def unocg_set_tuning(ctx, radix_order: int, path: int):
    _check(ctx, _lib.load().unocg_set_tuning(ctx, radix_order, path))


def unocg_autotune(ctx, opts: SolveOpts, reps: int = 3) -> np.ndarray:
    """Mean ms per solve for [radix_order][driver] (driver 0 graph, 1 persistent; NaN: n/a)."""
    out = np.zeros(6)
    _check(ctx, _lib.load().unocg_autotune(ctx, C.byref(opts), reps, _ptr(out)))
    return out.reshape(3, 2)


def unocg_dir_set_tuning(ctx, precision: int, plane_engine: int, line_engine: int):
    _dcheck(ctx, _lib.load().unocg_dir_set_tuning(ctx, precision, plane_engine, line_engine))


def unocg_dir_autotune(ctx, opts: SolveOpts, reps: int = 3) -> np.ndarray:
    """Mean ms per solve for [plane_engine][line_engine] (NaN: not applicable)."""
    out = np.zeros(6)
    _dcheck(ctx, _lib.load().unocg_dir_autotune(ctx, C.byref(opts), reps, _ptr(out)))
    return out.reshape(3, 2)


# ---------------------------------------------------------------- second-order training (device)
def unocg_newton_run(c: int, a_k, b_k, a_rest, b_rest, w0, max_steps: int = 100, tol: float = 1e-12):
    """Algorithm 4 on the device (``unocg_newton_*``): features at the learned modes ``a_k, b_k``
    ``[n, C]``, sums over the other modes ``a_rest, b_rest`` ``[C]``, start weights ``w0``
    ``[1 + n, C]``.  Returns (weights [1 + n, C], loss history without delta)."""
    lib = _lib.load()
    C_ = c * (c + 1) // 2
    ak = np.ascontiguousarray(a_k, dtype=np.float64).reshape(-1, C_)
    bk = np.ascontiguousarray(b_k, dtype=np.float64).reshape(-1, C_)
    ar = np.ascontiguousarray(a_rest, dtype=np.float64).reshape(C_)
    br = np.ascontiguousarray(b_rest, dtype=np.float64).reshape(C_)
    w = np.ascontiguousarray(w0, dtype=np.float64).reshape(-1, C_)
    n = ak.shape[0]
    if bk.shape[0] != n or w.shape[0] != n + 1:
        raise ValueError("features and weights do not match")
    h = C.c_void_p()
    rc = lib.unocg_newton_create(C.byref(h), c, n)
    if rc != _lib.OK:
        msg = lib.unocg_newton_last_error(h).decode() if h.value else "invalid arguments"
        if h.value:
            lib.unocg_newton_destroy(h)
        raise UnocgError(rc, msg)
    try:
        rc = lib.unocg_newton_set_features(h, _ptr(ak), _ptr(bk), _ptr(ar), _ptr(br))
        if rc != _lib.OK:
            raise UnocgError(rc, lib.unocg_newton_last_error(h).decode())
        out = np.empty_like(w)
        hist = np.empty(max_steps + 1)
        nh = C.c_int(hist.size)
        rc = lib.unocg_newton_run(h, _ptr(w), max_steps, tol, _ptr(out), _ptr(hist), C.byref(nh))
        if rc != _lib.OK:
            raise UnocgError(rc, lib.unocg_newton_last_error(h).decode())
        return out, [float(x) for x in hist[:nh.value]]
    finally:
        lib.unocg_newton_destroy(h)
