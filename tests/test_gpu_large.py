"""Planes too large for one shared-memory block: the row pass (axis 3 on chunks of rows) plus the
axis-2 column pass.  FP64 takes this path from 128^2 planes on, FP32 from 256^2 planes; the
256^3 elastic instance of the uneven-batch workload runs on it."""
import numpy as np
import pytest

from oracle import fem, uno
from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("physics,shape", [(1, (4, 128, 128)), (3, (3, 128, 128)), (1, (2, 256, 256)),
                                           (3, (2, 256, 192))])
def test_fp64_apply_on_row_path_matches_oracle(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=1)
    props = np.array([1.0, 7.0]) if physics == 1 else np.array([[1.0, 0.3], [7.0, 0.2]])
    ctx = api.unocg_create(physics, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 2)
    api.unocg_set_phase_properties(ctx, props)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    r = random_field((c,) + shape, seed=2)
    rr = torch.tensor(r, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_apply_uno_dev(ctx, 0, rr, ss)
    torch.cuda.synchronize()
    Q = uno.reference_medium_Q(physics, props, shape)
    # The oracle forms S(k) by transforming the stencil: its absolute rounding error (about
    # eps times the stencil's absolute sum) is relative to S ~ theta^2 at the lowest
    # frequency, so the oracle's own error grows like (N / 2 pi)^2.
    tol = 1e-12 * max(1.0, (max(shape) / 64.0) ** 2)
    assert rel(ss.cpu().numpy(), uno.uno_apply(Q, r)) < tol
    api.unocg_destroy(ctx)


def _theta(shape, c, seed):
    rng = np.random.default_rng(seed)
    th = rng.standard_normal((shape[0], shape[1], shape[2] // 2 + 1, c * (c + 1) // 2)) * 0.3
    th[..., 0] += 1.0
    if c == 3:
        th[..., 1] += 1.0
        th[..., 3] += 1.0
    return th


@pytest.mark.parametrize("c,shape", [(1, (2, 256, 256)), (3, (2, 256, 192)), (1, (4, 512, 64))])
def test_fp32_operator_on_row_path_matches_oracle(c, shape):
    """The FP32 training operator on planes of 256^2 and 512 x 33 (row pass + column pass):
    apply and the input gradient of the backward against the FP64 oracle."""
    import torch
    from paper_2508_02681_gb300 import api
    th = _theta(shape, c, 1).astype(np.float32).astype(np.float64)
    B = 2
    r = np.stack([random_field((c,) + shape, seed=10 + b) for b in range(B)])
    g = np.stack([random_field((c,) + shape, seed=30 + b) for b in range(B)])
    op = api.unocg_uno_create(c, *shape)
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    api.unocg_uno_set_theta_dev(op, tt)
    rr = torch.tensor(r, dtype=torch.float32, device="cuda")
    gg = torch.tensor(g, dtype=torch.float32, device="cuda")
    ss = torch.empty_like(rr)
    gr = torch.empty_like(rr)
    api.unocg_uno_apply_dev(op, B, rr, ss)
    api.unocg_uno_backward_dev(op, B, rr, gg, gr, None)
    torch.cuda.synchronize()
    Q = uno.symmetrize_half(uno.psi(th, c), shape[2])
    for b in range(B):
        assert rel(ss[b].cpu().numpy().astype(np.float64), uno.uno_apply(Q, r[b])) < 2e-5
        assert rel(gr[b].cpu().numpy().astype(np.float64), uno.uno_apply(Q, g[b])) < 2e-5
    api.unocg_uno_destroy(op)


def _solver(physics, phase, props, loads):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(physics, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


@pytest.mark.parametrize("shape", [(16, 128, 128), (8, 256, 256)])
def test_row_path_solves_agree_across_precisions(shape):
    """FP64 on the row path against mixed precision (whole planes at 128^2, rows at 256^2).  A
    wrong transform would still converge, more slowly: the iteration counts must agree too."""
    from paper_2508_02681_gb300 import _lib
    phase, _ = rsa_spheres(shape, 5.0, 0.2, seed=3)
    props = np.array([1.0, 20.0])
    h = _solver(_lib.THERMAL, phase, props, unit_loads(1))
    i64 = h.solve(tol=1e-6, max_iter=3000, precision=_lib.FP64)
    C64 = h.effective_tensor()[0]
    imx = h.solve(tol=1e-6, max_iter=3000, precision=_lib.MIXED)
    Cmx = h.effective_tensor()[0]
    assert i64.status == _lib.OK and imx.status == _lib.OK
    assert np.all(i64.true_rel_res <= 1e-6) and np.all(imx.true_rel_res <= 1e-6)
    assert rel(Cmx, C64) < 1e-6
    it64, itmx = np.asarray(i64.iters), np.asarray(imx.iters)
    assert np.all(itmx <= 1.1 * it64 + 3) and np.all(it64 <= 1.1 * itmx + 3)
    h.close()


def _interface_nodes(phase, count, rng):
    """Nodes whose eight adjacent elements are not all of one phase (there f = -B^T C E != 0)."""
    mixed = np.zeros(phase.shape, bool)
    for o in fem.CORNERS:
        mixed |= np.roll(phase, shift=tuple(int(x) for x in o), axis=(0, 1, 2)) != phase
    idx = np.argwhere(mixed)
    pick = idx[rng.choice(len(idx), size=count, replace=False)]
    return [tuple(int(x) for x in p) for p in pick]


def test_elastic_256_mixed_single_instance():
    """The 256^3 elastic instance (contrast 100, six Mandel loads, mixed precision, 1e-6)."""
    from paper_2508_02681_gb300 import _lib
    shape = (256, 256, 256)
    phase, vf = rsa_spheres(shape, 24.0, 0.3, seed=2508002681 + 5999)
    props = np.array([[1.0, 0.3], [100.0, 0.2]])
    loads = unit_loads(3)
    h = _solver(_lib.ELASTIC, phase, props, loads)
    info = h.solve(tol=1e-6, max_iter=3000, precision=_lib.MIXED)
    assert info.status == _lib.OK
    assert np.all(info.true_rel_res <= 1e-6)
    C = h.effective_tensor()[0]
    assert np.max(np.abs(C - C.T)) < 1e-5 * np.max(np.abs(C))
    Ds = [fem.material_matrix(3, p) for p in props]
    voigt = (1 - vf) * Ds[0] + vf * Ds[1]
    reuss = np.linalg.inv((1 - vf) * np.linalg.inv(Ds[0]) + vf * np.linalg.inv(Ds[1]))
    Cs = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(voigt - Cs).min() > -1e-6
    assert np.linalg.eigvalsh(Cs - reuss).min() > -1e-6
    # oracle, node by node: the residual at random and at interface nodes is below the tolerance
    # times the largest |f| seen at interface nodes (a lower bound of ||f||_inf)
    rng = np.random.default_rng(8)
    nodes = [tuple(int(x) for x in rng.integers(0, 256, size=3)) for _ in range(16)]
    nodes += _interface_nodes(phase, 64, rng)
    for l in (0, 3):
        u = h.fluctuation(0, l)
        f0 = fem.residual_at_nodes(phase, props, 3, np.zeros_like(u), loads[l], nodes)
        res = fem.residual_at_nodes(phase, props, 3, u, loads[l], nodes)
        assert np.max(np.abs(f0)) > 0
        assert np.max(np.abs(res)) <= 3e-6 * np.max(np.abs(f0))
    h.close()
