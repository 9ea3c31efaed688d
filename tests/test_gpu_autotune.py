"""Autotuners of the batched / repeated solves (radix plans and loop driver of the periodic
solver; pass engines of the Dirichlet / mixed-BC solver): every candidate solves to the same
result, the table marks what does not apply, the choice is kept and cached."""
import numpy as np
import pytest

from synth import rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 20, 30)])
def test_periodic_autotune(shape, tmp_path):
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    phase, _ = rsa_spheres(shape, shape[0] / 5.0, 0.25, seed=3)
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([1.0, 10.0]))
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    kw = dict(tol=1e-10, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.FP64, flexible=0)
    h.solve(**kw)
    C0 = h.effective_tensor()[0]
    cache = str(tmp_path / "tune.json")
    setting, table = h.autotune(cache=cache, reps=2, **kw)
    assert table.shape == (3, 2) and np.all(np.isfinite(table[:, 0])) and np.all(table[np.isfinite(table)] > 0)
    assert table[setting[0], setting[1] - 1] == np.nanmin(table)
    for order in range(3):
        for path in (1, 2):
            if not np.isfinite(table[order, path - 1]):
                continue
            api.unocg_set_tuning(h.ctx, order, path)
            h.solve(use_graph=3, **kw)
            assert rel(h.effective_tensor()[0], C0) < 1e-12
    s2, t2 = h.autotune(cache=cache, reps=2, **kw)
    assert s2 == setting and t2 is None
    h.close()


@pytest.mark.parametrize("shape,bc,physics", [((16, 16, 16), (1, 1, 1), 1), ((12, 10, 18), (1, 1, 1), 3),
                                              ((16, 12, 16), (0, 1, 0), 1)])
def test_dirichlet_autotune(shape, bc, physics):
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import DirichletHomogenization
    phase, _ = rsa_spheres(shape, shape[0] / 5.0, 0.25, seed=4)
    props = np.array([1.0, 10.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])
    h = DirichletHomogenization(physics, shape, bc=bc)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(unit_loads(physics)[:2])
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    for prec in (_lib.FP64, _lib.MIXED):
        kw = dict(tol=1e-10 if prec == _lib.FP64 else 1e-6, max_iter=3000, precond=_lib.PRECOND_UNO, precision=prec)
        h.solve(**kw)
        C0 = h.effective_tensor()[0]
        setting, table = h.autotune(reps=2, **kw)
        assert table.shape == (3, 2)
        assert np.isfinite(table[2, 1])                      # separate passes, shared-memory axis 1
        if physics == 3 or bc != (1, 1, 1):
            assert np.all(np.isnan(table[:, 0]))             # register axis-1 pass: c = 1, Dirichlet only
        if bc != (1, 1, 1) or shape[1] != shape[2]:
            assert np.all(np.isnan(table[0]))                # register planes: Dirichlet, N2 = N3
        assert table[setting[0], setting[1]] == np.nanmin(table)
        for pe in range(3):
            for le in range(2):
                if not np.isfinite(table[pe, le]):
                    continue
                api.unocg_dir_set_tuning(h.ctx, prec, pe, le)
                h.solve(**kw)
                assert rel(h.effective_tensor()[0], C0) < (1e-12 if prec == _lib.FP64 else 1e-6)
    h.close()
