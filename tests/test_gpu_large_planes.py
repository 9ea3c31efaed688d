"""Flexible (Polak-Ribiere) UNO-CG on grids whose (axis-2, axis-3) planes are too large for one
block: the forward and inverse transforms then run as a row pass plus a separate axis-2 pass (for
256 x 256 FP32 planes both in registers), or, for 256 x 256 FP32 planes, as one pass on a cluster
of two blocks.
The r . s_old term of the flexible coefficient reads the previous s_hat, so the inverse axis-2
pass must leave it intact.  FP64 against the oracle's flexible PCG on the same inputs (fields
1e-9, effective tensor 1e-10); mixed precision to the effective tensor (1e-6) with the true
residual at the tolerance and no more iterations than the oracle needs plus a small slack."""
import numpy as np
import pytest

from oracle import homogenize as hz
from synth import rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

PROPS = np.array([1.0, 20.0])


def _case(shape):
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=5)
    loads = unit_loads(1)[:2]
    r = hz.solve(phase, PROPS, 1, loads, precond="uno", tol=1e-9, flexible=True)
    r["C"] = hz.effective_tensor(phase, PROPS, 1, r["u"], loads)
    return phase, loads, r


@pytest.fixture(scope="module")
def fp64_case():
    return _case((6, 120, 120))   # FP64 planes of 120 x 61 complex exceed one block's shared memory


@pytest.fixture(scope="module")
def f32_case():
    return _case((6, 180, 180))   # FP32 planes of 180 x 91 complex exceed one block's shared memory


def _solver(phase, loads):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(_lib.THERMAL, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(PROPS)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


@pytest.mark.parametrize("use_graph", [1, 0])
def test_flexible_fp64_row_passes_match_oracle(fp64_case, use_graph):
    from paper_2508_02681_gb300 import _lib
    phase, loads, ref = fp64_case
    h = _solver(phase, loads)
    info = h.solve(tol=1e-9, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64, flexible=1,
                   use_graph=use_graph)
    for l in range(2):
        assert abs(int(info.iters[l]) - ref["iters"][l]) <= 1
        assert rel(h.fluctuation(0, l), ref["u"][l]) < 1e-9
    assert rel(h.effective_tensor()[0], ref["C"]) < 1e-10
    h.close()


def test_flexible_mixed_row_passes_converge(f32_case):
    from paper_2508_02681_gb300 import _lib
    phase, loads, ref = f32_case
    h = _solver(phase, loads)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1,
                   replace_every=50)
    assert info.status == _lib.OK
    assert np.all(info.true_rel_res <= 1e-6)
    assert np.all(info.iters <= np.array(ref["iters"]) + 8)
    assert rel(h.effective_tensor()[0], ref["C"]) < 1e-6
    h.close()


@pytest.fixture(scope="module")
def cluster_case():
    return _case((4, 256, 256))   # FP32 256 x 256 planes: one pass on two-CTA clusters


@pytest.mark.parametrize("use_graph,passes,cols_reg", [(1, 1, 1), (0, 1, 1), (1, 3, 1), (0, 3, 1), (1, 0, 1),
                                                      (0, 0, 1), (1, 0, 0), (1, 2, 0)])
def test_cluster_plane_passes_mixed_match_oracle(cluster_case, use_graph, passes, cols_reg, monkeypatch):
    """256 x 256 planes in the mixed loop against the oracle's flexible PCG: plane passes on
    two-CTA clusters (values exchanged through distributed shared memory; `passes` masks which:
    1 forward, 2 inverse) or as row pass plus column pass (the register column pass, two columns
    a warp, or with `cols_reg` 0 the shared-memory one)."""
    from paper_2508_02681_gb300 import _lib
    monkeypatch.setenv("UNOCG_PLANE_CL", str(passes))
    monkeypatch.setenv("UNOCG_COLS_REG", str(cols_reg))
    phase, loads, ref = cluster_case
    h = _solver(phase, loads)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1,
                   replace_every=50, use_graph=use_graph)
    assert info.status == _lib.OK
    assert np.all(info.true_rel_res <= 1e-6)
    assert np.all(info.iters <= np.array(ref["iters"]) + 8)
    assert rel(h.effective_tensor()[0], ref["C"]) < 1e-6
    h.close()


@pytest.mark.parametrize("passes", [0, 1, 3])
def test_cluster_plane_passes_elastic_mixed_match_oracle(passes, monkeypatch):
    """The same for three components per node (each component's plane is its own cluster)."""
    from paper_2508_02681_gb300 import _lib
    monkeypatch.setenv("UNOCG_PLANE_CL", str(passes))
    from paper_2508_02681_gb300.solver import Homogenization
    phase, _ = rsa_spheres((2, 256, 256), 3.0, 0.25, seed=6)
    props = np.array([[1.0, 0.3], [10.0, 0.2]])
    loads = unit_loads(3)[[0, 3]]
    ref = hz.solve(phase, props, 3, loads, precond="uno", tol=1e-9, flexible=True)
    Cref = hz.effective_tensor(phase, props, 3, ref["u"], loads)
    h = Homogenization(_lib.ELASTIC, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1)
    assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
    assert rel(h.effective_tensor()[0], Cref) < 1e-6
    h.close()
