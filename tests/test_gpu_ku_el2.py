"""The FP32 elastic K d with element pairs in packed FP32x2 arithmetic (Sec. 4.1, element forces in
the Walsh basis, two elements of a row per thread) against the assembled K of the oracle: grids of
one and several node tiles along every axis, ragged tiles (N3 not a multiple of 32, N2 not a
multiple of 8, N1 not a multiple of the plane chunk of 8, 16 or 32 planes), two- and four-node
periodic axes (the halo element pairs wrap onto the tile itself), several phases; and a
mixed-precision elastic solve with it against the oracle's flexible PCG."""
import numpy as np
import pytest

from oracle import fem
from oracle import homogenize as hz
from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

SHAPES = [(2, 16, 32), (3, 9, 64), (18, 8, 36), (4, 2, 4), (9, 3, 6), (6, 20, 96), (10, 24, 40)]
TOL32 = 2e-6   # FP32 element forces of about 190 operations, relative to the largest |p|


def _props():
    return np.array([[1.0, 0.3], [10.0, 0.2], [3.0, 0.45]])


@pytest.mark.parametrize("cz", ["", "8", "32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_K32_elastic_pairs_match_assembled_K(shape, cz, monkeypatch):
    """`cz`: node planes per block (default: 16 below 10^6 nodes per field; 8 and 32 as set by
    UNOCG_KE2_CZ, 32 being the default of large grids)."""
    import torch
    from paper_2508_02681_gb300 import api
    phase = random_phase(shape, 3, seed=sum(shape) + 1)
    props = _props()
    ctx = api.unocg_create(3, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 3)
    api.unocg_set_phase_properties(ctx, props)
    d = random_field((3,) + shape, seed=13).astype(np.float32)
    K = fem.assemble_K(phase, props, 3)
    p_ref = fem.to_soa(K @ fem.from_soa(d.astype(np.float64)), 3, shape)
    dd = torch.tensor(d, device="cuda")
    if cz:
        monkeypatch.setenv("UNOCG_KE2_CZ", cz)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("UNOCG_KU_EL2", flag)
        pp = torch.full_like(dd, float("nan"))
        api.unocg_apply_K32_dev(ctx, 0, dd, pp)
        torch.cuda.synchronize()
        p = pp.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(p)), flag
        assert rel(p, p_ref) < TOL32, (flag, rel(p, p_ref))
        out[flag] = p
    assert rel(out["1"], out["0"]) < TOL32
    api.unocg_destroy(ctx)


def test_elastic_mixed_solve_with_pairs_matches_oracle(monkeypatch):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    monkeypatch.setenv("UNOCG_KU_EL2", "1")
    shape = (16, 16, 20)
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=21)
    props = np.array([[1.0, 0.3], [10.0, 0.2]])
    loads = unit_loads(3)[[0, 4]]
    ref = hz.solve(phase, props, 3, loads, precond="uno", tol=1e-9, flexible=True)
    C_ref = hz.effective_tensor(phase, props, 3, ref["u"], loads)
    h = Homogenization(_lib.ELASTIC, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1)
    assert info.status == _lib.OK
    assert np.all(info.true_rel_res <= 1e-6)
    assert np.all(info.iters <= np.array(ref["iters"]) + 8)
    assert rel(h.effective_tensor()[0], C_ref) < 1e-6
    h.close()
