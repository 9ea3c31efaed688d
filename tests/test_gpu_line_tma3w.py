"""The three-component axis-1 pass of the mixed-precision elastic loop on long axes (96, 128, 192
and 256 points: only the r_hat tiles staged by the TMA, the previous s_hat and the 3 x 3 block
entries read by each thread from global memory, each line's tile column as its exchange slots)
against the oracle's flexible and plain PCG: effective stiffness within 1e-6, true FP64 residual
at the tolerance, iterations within a small slack, and within rounding of the shared-memory
Stockham pass (UNOCG_LINE_TMA=0) on the same inputs."""
import numpy as np
import pytest

from oracle import homogenize as hz
from synth import rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

PROPS = np.array([[1.0, 0.3], [10.0, 0.2]])


@pytest.fixture(scope="module", params=[(96, 8, 8), (128, 8, 10), (192, 6, 6), (256, 8, 8)])
def case(request):
    shape = request.param
    phase, _ = rsa_spheres(shape, 2.5, 0.25, seed=23)
    loads = unit_loads(3)[[0, 3]]
    out = {}
    for flexible in (True, False):
        ref = hz.solve(phase, PROPS, 3, loads, precond="uno", tol=1e-9, flexible=flexible)
        out[flexible] = (ref, hz.effective_tensor(phase, PROPS, 3, ref["u"], loads))
    return phase, loads, out


def _mixed(phase, loads, flexible):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(_lib.ELASTIC, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(PROPS)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED,
                   flexible=1 if flexible else 0)
    C = h.effective_tensor()[0]
    h.close()
    return info, C


@pytest.mark.parametrize("flexible", [True, False])
def test_long_axis_c3_tma_pass_matches_oracle(case, flexible, monkeypatch):
    from paper_2508_02681_gb300 import _lib
    phase, loads, out = case
    ref, C_ref = out[flexible]
    res = {}
    for tma in (1, 0):
        monkeypatch.setenv("UNOCG_LINE_TMA", str(tma))
        info, C = _mixed(phase, loads, flexible)
        assert info.status == _lib.OK, tma
        assert np.all(info.true_rel_res <= 1e-6), tma
        assert np.all(info.iters <= np.array(ref["iters"]) + 8), (tma, info.iters, ref["iters"])
        assert rel(C, C_ref) < 1e-6, tma
        res[tma] = C
    assert rel(res[1], res[0]) < 1e-6
