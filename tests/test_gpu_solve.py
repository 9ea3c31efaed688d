"""GPU UNO-CG / Jac-CG solves against the FP64 oracle on the same seeded inputs.

Bars: FP64 path fields within 1e-9 relative and effective tensors within 1e-10; mixed path
(FP32 fields, BF16 weights, FP64 reductions, residual replacement, flexible CG) effective
tensors within 1e-6 relative with a true FP64 residual of at most the tolerance."""
import numpy as np
import pytest

from oracle import homogenize as hz
from synth import random_phase, rsa_spheres, unit_loads, workload
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _solver(physics, phase, props, loads, n_phases=None):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(physics, phase.shape)
    h.set_microstructure(phase, n_phases or int(phase.max()) + 1)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


@pytest.fixture(scope="module")
def config1():
    w = workload(1)
    ref = {}
    for pc in ("jacobi", "uno"):
        r = hz.solve(w["phase"], w["props"], 1, w["loads"], precond=pc, tol=w["tol"])
        r["C"] = hz.effective_tensor(w["phase"], w["props"], 1, r["u"], w["loads"])
        ref[pc] = r
    return w, ref


@pytest.mark.parametrize("pc", ["jacobi", "uno"])
@pytest.mark.parametrize("use_graph", [1, 0, 2])
def test_config1_fp64_matches_oracle(config1, pc, use_graph):
    from paper_2508_02681_gb300 import _lib
    w, ref = config1
    if use_graph == 2 and pc == "jacobi":
        pytest.skip("the persistent loop runs the UNO preconditioner")
    h = _solver(1, w["phase"], w["props"], w["loads"])
    precond = _lib.PRECOND_UNO if pc == "uno" else _lib.PRECOND_JACOBI
    info = h.solve(tol=w["tol"], max_iter=2000, precond=precond, precision=_lib.FP64, use_graph=use_graph)
    r = ref[pc]
    for l in range(3):
        assert abs(int(info.iters[l]) - r["iters"][l]) <= 1
        assert rel(h.fluctuation(0, l), r["u"][l]) < 1e-9
    C = h.effective_tensor()[0]
    assert rel(C, r["C"]) < 1e-10
    assert np.all(info.true_rel_res <= 10 * w["tol"])
    h.close()


@pytest.mark.parametrize("use_graph", [1, 0, 2])
def test_config1_mixed_matches_oracle(config1, use_graph):
    from paper_2508_02681_gb300 import _lib
    w, ref = config1
    h = _solver(1, w["phase"], w["props"], w["loads"])
    info = h.solve(tol=1e-6, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED,
                   replace_every=50, use_graph=use_graph)
    C = h.effective_tensor()[0]
    assert rel(C, ref["uno"]["C"]) < 1e-6
    assert np.all(info.true_rel_res <= 1e-6)
    h.close()


@pytest.mark.parametrize("use_graph", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_elastic_small_matches_oracle(precision, use_graph):
    from paper_2508_02681_gb300 import _lib
    phase, _ = rsa_spheres((8, 8, 8), 2.0, 0.3, seed=77)
    props = np.array([[1.0, 0.3], [10.0, 0.2]])
    loads = unit_loads(3)
    tol = 1e-8 if precision == 0 else 1e-6
    ref = hz.solve(phase, props, 3, loads, precond="uno", tol=1e-12)
    Cref = hz.effective_tensor(phase, props, 3, ref["u"], loads)
    h = _solver(3, phase, props, loads)
    info = h.solve(tol=tol, max_iter=2000, precond=_lib.PRECOND_UNO, precision=precision, use_graph=use_graph)
    C = h.effective_tensor()[0]
    assert rel(C, Cref) < (1e-9 if precision == 0 else 1e-6)
    if precision == 0:
        ref8 = hz.solve(phase, props, 3, loads, precond="uno", tol=tol)
        for l in range(6):
            assert rel(h.fluctuation(0, l), ref8["u"][l]) < 1e-9
    assert np.all(info.true_rel_res <= tol)
    h.close()


def test_paths_agree_bitwise_on_fp64():
    """The graph, host-driven and persistent loops run the same kernels in the same order of
    reductions, so their FP64 iterates agree exactly."""
    from paper_2508_02681_gb300 import _lib
    phase, _ = rsa_spheres((16, 16, 16), 3.0, 0.25, seed=5)
    props = np.array([1.0, 10.0])
    h = _solver(1, phase, props, unit_loads(1))
    out = []
    for ug in (0, 1, 2):
        info = h.solve(tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64, use_graph=ug)
        out.append((list(info.iters), h.fluctuation(0, 1), h.effective_tensor()[0]))
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert np.array_equal(o[1], out[0][1])
        assert np.array_equal(o[2], out[0][2])
    h.close()


def test_device_wait_limit_reports_timeout_and_context_recovers():
    """A grid-barrier wait that expires makes the persistent loop return DEVICE_TIMEOUT (no GPU
    fault, no hang); with the default limit the same context solves normally afterwards."""
    from paper_2508_02681_gb300 import _lib, api
    phase, _ = rsa_spheres((16, 16, 16), 3.0, 0.25, seed=6)
    props = np.array([1.0, 10.0])
    h = _solver(1, phase, props, unit_loads(1))
    api.unocg_set_wait_limit(h.ctx, 0.0)  # one clock cycle: every early block gives up
    info = h.solve(raise_on_error=False, tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO,
                   precision=_lib.FP64, use_graph=2)
    assert info.status == _lib.ERR_DEVICE_TIMEOUT
    api.unocg_set_wait_limit(h.ctx, 1.0)
    info = h.solve(tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64, use_graph=2)
    assert info.status == _lib.OK
    h.close()
