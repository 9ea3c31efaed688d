"""The FP32 thermal K d of the mixed-precision loop on TMA-staged tiles, against the assembled K
of the oracle (Sec. 4.1): every tile shape the grid allows, grids of one and several tiles along
i2 and i1, ragged plane chunks, two- and three-node periodic axes (the halo planes and rows wrap
onto the tile itself), 32 to 256 nodes along i3 (a row in one warp, or across warps), batches."""
import numpy as np
import pytest

from oracle import fem
from synth import random_field, random_phase
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

# (16, 2, 32): no tile shape divides N2 = 2, only the earlier kernel runs
SHAPES = [(2, 16, 32), (3, 16, 64), (15, 16, 64), (25, 32, 128), (9, 8, 256), (16, 2, 32), (30, 64, 64),
          (5, 8, 192), (4, 12, 96), (6, 16, 160)]
TOL32 = 4e-6   # FP32 stencil of 21 terms, relative to the largest |p|


def _ctx(shape, phase, props, batch=1):
    from paper_2508_02681_gb300 import api
    ctx = api.unocg_create(1, batch, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 4)
    api.unocg_set_phase_properties(ctx, props)
    return ctx


@pytest.mark.parametrize("shape", SHAPES)
def test_K32_every_tile_matches_assembled_K(shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    phase = random_phase(shape, 4, seed=sum(shape))
    props = np.array([1.0, 7.5, 0.3, 42.0])
    ctx = _ctx(shape, phase, props)
    d = random_field((1,) + shape, seed=11).astype(np.float32)
    K = fem.assemble_K(phase, props, 1)
    p_ref = fem.to_soa(K @ fem.from_soa(d.astype(np.float64)), 1, shape)
    dd = torch.tensor(d, device="cuda")
    ran = []
    for tile in range(17):
        try:
            api.unocg_set_ku_tile(ctx, tile)
        except _lib.UnocgError as err:
            assert tile > 0 and err.code == _lib.ERR_INVALID_ARG
            continue
        pp = torch.full_like(dd, float("nan"))
        api.unocg_apply_K32_dev(ctx, 0, dd, pp)
        torch.cuda.synchronize()
        p = pp.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(p)), tile
        assert rel(p, p_ref) < TOL32, (tile, rel(p, p_ref))
        ran.append(tile)
    assert 0 in ran and (any(t > 0 for t in ran) or shape[1] == 2), ran
    api.unocg_destroy(ctx)


def test_K32_batch_instances_and_default_tile():
    """Instances of a batch take their own phase labels and conductivities (TMA tile (4, 12))."""
    import torch
    from paper_2508_02681_gb300 import api
    shape, B = (12, 16, 128), 3
    phases = np.stack([random_phase(shape, 4, seed=40 + b) for b in range(B)])
    props = np.stack([np.array([1.0, 3.0, 10.0, 0.5]) * (b + 1) for b in range(B)])
    ctx = _ctx(shape, phases, props, batch=B)
    # too few blocks for the vector march: the automatic choice keeps the column march; take a
    # TMA tile explicitly
    assert api.unocg_get_ku_tile(ctx) == 0
    api.unocg_set_ku_tile(ctx, 1)
    assert api.unocg_get_ku_tile(ctx) == 1
    for b in range(B):
        d = random_field((1,) + shape, seed=60 + b).astype(np.float32)
        K = fem.assemble_K(phases[b], props[b], 1)
        p_ref = fem.to_soa(K @ fem.from_soa(d.astype(np.float64)), 1, shape)
        dd = torch.tensor(d, device="cuda")
        pp = torch.empty_like(dd)
        api.unocg_apply_K32_dev(ctx, b, dd, pp)
        torch.cuda.synchronize()
        assert rel(pp.cpu().numpy().astype(np.float64), p_ref) < TOL32
    api.unocg_destroy(ctx)


def test_ku_autotune_keeps_the_fastest_and_solves_match():
    """The stencil autotuner times every candidate on the context's own fields and keeps the
    fastest; mixed-precision solves with the earlier kernel and with the tuned tile reach the
    tolerance with the same effective tensor (to the 1e-6 of mixed precision)."""
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import rsa_spheres, unit_loads
    phase, _ = rsa_spheres((32, 32, 64), 4.0, 0.3, seed=5)
    h = Homogenization(_lib.THERMAL, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([1.0, 100.0]))
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    times, best = api.unocg_autotune_ku(h.ctx, reps=5)
    assert np.isfinite(times[0]) and np.isfinite(times[best])
    assert times[best] == np.nanmin(times)
    assert api.unocg_get_ku_tile(h.ctx) == best
    Cs = []
    for tile in (0, best):
        api.unocg_set_ku_tile(h.ctx, tile)
        info = h.solve(tol=1e-6, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED)
        assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
        Cs.append(h.effective_tensor()[0])
    assert rel(Cs[1], Cs[0]) < 1e-6
    h.close()


# tile shapes (node rows, node planes), in the order of the library's table (indices 1..8; the
# vector march takes 9..16 for the same shapes)
TILE_SHAPES = [(4, 12), (8, 12), (2, 12), (8, 24), (16, 6), (4, 24), (16, 12), (8, 6)]


def _vec_supported(shape, rows):
    n1, n2, n3 = shape
    th = rows * (n3 // 4)
    return n3 % 32 == 0 and n3 <= 512 and th % 32 == 0 and 64 <= th <= 512 and n2 % rows == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_K32_vector_march_tiles_available(shape):
    """The vector-march tiles (9..16) the library accepts are those of the stated rule."""
    from paper_2508_02681_gb300 import _lib, api
    phase = random_phase(shape, 4, seed=3)
    ctx = _ctx(shape, phase, np.array([1.0, 2.0, 3.0, 4.0]))
    for k, (rows, planes) in enumerate(TILE_SHAPES, start=1):
        ok = True
        try:
            api.unocg_set_ku_tile(ctx, 8 + k)
        except _lib.UnocgError as err:
            assert err.code == _lib.ERR_INVALID_ARG
            ok = False
        assert ok == _vec_supported(shape, rows), (k, rows)
        if ok:
            assert api.unocg_get_ku_tile(ctx) == 8 + k
    api.unocg_destroy(ctx)


def test_vector_march_solve_matches_oracle():
    """The vector march (tile 14: shape (4, 24)) inside the mixed loop, 16 x 256 x 256, against
    the oracle's flexible PCG."""
    from oracle import homogenize as hz
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import rsa_spheres, unit_loads
    shape = (16, 256, 256)
    phase, _ = rsa_spheres(shape, 5.0, 0.3, seed=21)
    props = np.array([1.0, 20.0])
    loads = unit_loads(1)[:1]
    ref = hz.solve(phase, props, 1, loads, precond="uno", tol=1e-8, flexible=True)
    C_ref = hz.effective_tensor(phase, props, 1, ref["u"], loads)
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    api.unocg_set_ku_tile(h.ctx, 14)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1)
    assert api.unocg_get_ku_tile(h.ctx) == 14
    assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
    assert np.all(info.iters <= np.array(ref["iters"]) + 8)
    assert rel(h.effective_tensor()[0], C_ref) < 1e-6
    h.close()


def test_auto_choice_takes_the_vector_march_on_large_grids():
    """Three loads: 256^3 takes the vector march with shape (4, 24) (tile 14); 192^3 the one with
    shape (2, 12) (tile 11: 15 warps per SM against 12 for (4, 24)); 64^3, below 10^6 nodes per
    field, the one with shape (8, 6) (tile 16, at least one block per SM); a grid too small for
    one block per SM the column march (tile 0)."""
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import unit_loads
    for shape, want in (((256, 256, 256), 14), ((192, 192, 192), 11), ((64, 64, 64), 16), ((24, 16, 32), 0)):
        h = Homogenization(_lib.THERMAL, shape)
        h.set_microstructure(np.zeros(shape, dtype=np.uint8), 2)
        h.set_phase_properties(np.array([1.0, 2.0]))
        h.set_macro_load(unit_loads(1))
        assert api.unocg_get_ku_tile(h.ctx) == want, shape
        h.close()
