"""Planes too large for one shared-memory block: the row pass + axis-2 column pass path.
FP64 switches to it at 128^2 planes, FP32 at 256^2 planes; the 256^3 elastic instance of the
uneven-batch workload runs on it."""
import numpy as np
import pytest

from oracle import fem, uno
from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("physics", [1, 3])
def test_fp64_apply_on_row_path_matches_oracle(physics):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    shape = (4, 128, 128)
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
    assert rel(ss.cpu().numpy(), uno.uno_apply(Q, r)) < 1e-12
    api.unocg_destroy(ctx)


def test_fp32_row_path_solve_agrees_with_fp64():
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (8, 256, 256)
    phase, _ = rsa_spheres(shape, 5.0, 0.2, seed=3)
    props = np.array([1.0, 20.0])
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    i64 = h.solve(tol=1e-8, max_iter=3000, precision=_lib.FP64)
    C64 = h.effective_tensor()[0]
    imx = h.solve(tol=1e-6, max_iter=3000, precision=_lib.MIXED)
    Cmx = h.effective_tensor()[0]
    assert np.all(i64.true_rel_res <= 1e-8) and np.all(imx.true_rel_res <= 1e-6)
    assert rel(Cmx, C64) < 1e-6
    h.close()


def test_elastic_256_mixed_single_instance():
    """The 256^3 elastic instance (contrast 100, 6 Mandel loads, mixed precision, 1e-6)."""
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (256, 256, 256)
    phase, vf = rsa_spheres(shape, 24.0, 0.3, seed=2508002681 + 5000 + 999)
    props = np.array([[1.0, 0.3], [100.0, 0.2]])
    loads = unit_loads(3)
    h = Homogenization(_lib.ELASTIC, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=3000, precision=_lib.MIXED)
    assert info.status == _lib.OK
    assert np.all(info.true_rel_res <= 1e-6)
    C = h.effective_tensor()[0]
    assert np.max(np.abs(C - C.T)) < 1e-4 * np.max(np.abs(C))
    Ds = [fem.material_matrix(3, p) for p in props]
    voigt = (1 - vf) * Ds[0] + vf * Ds[1]
    reuss = np.linalg.inv((1 - vf) * np.linalg.inv(Ds[0]) + vf * np.linalg.inv(Ds[1]))
    Cs = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(voigt - Cs).min() > -1e-6
    assert np.linalg.eigvalsh(Cs - reuss).min() > -1e-6
    # residual at sampled nodes, by the oracle one node at a time
    rng = np.random.default_rng(8)
    nodes = [tuple(int(x) for x in rng.integers(0, 256, size=3)) for _ in range(16)]
    u = h.fluctuation(0, 3)
    f0 = fem.residual_at_nodes(phase, props, 3, np.zeros_like(u), loads[3], nodes)
    res = fem.residual_at_nodes(phase, props, 3, u, loads[3], nodes)
    # ||f||_inf bounds every sampled |f| from above; the GPU reported the global ratio
    assert np.max(np.abs(res)) <= 1e-6 * max(np.max(np.abs(f0)), 1e-300) * 50
    h.close()
