"""The axis-1 pass of the mixed-precision loop for c = 1 as a persistent pipeline of TMA tiles
(UNOCG_LINE_TP=1, off by default; a ring of shared-memory stages refilled by one producer thread while the
consumer warps transform) against the oracle's flexible and plain PCG: effective tensor within
1e-6, true FP64 residual at the tolerance, iterations within a small slack.  The grid is capped
(UNOCG_LINE_TP_BLOCKS) so that each block walks many tiles: the ring wraps, stages are stored and
reloaded, the tiles of a load that converged first are skipped, the last tile of a pair is
partial; the result matches the one-tile-per-block pass within rounding."""
import numpy as np
import pytest

from oracle import homogenize as hz
from synth import rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

PROPS = np.array([1.0, 20.0])


@pytest.fixture(scope="module", params=[(64, 16, 30), (128, 24, 30), (256, 16, 30)])
def case(request):
    shape = request.param
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=17)
    loads = unit_loads(1)[:2]
    out = {}
    for flexible in (True, False):
        ref = hz.solve(phase, PROPS, 1, loads, precond="uno", tol=1e-9, flexible=flexible)
        out[flexible] = (ref, hz.effective_tensor(phase, PROPS, 1, ref["u"], loads))
    return phase, loads, out


def _mixed(phase, loads, flexible):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(_lib.THERMAL, phase.shape)
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
def test_line_pipeline_matches_oracle(case, flexible, monkeypatch):
    from paper_2508_02681_gb300 import _lib
    phase, loads, out = case
    ref, C_ref = out[flexible]
    res = {}
    for tp, blocks in ((1, 1), (1, 3), (1, 0), (0, 0)):
        monkeypatch.setenv("UNOCG_LINE_TP", str(tp))
        monkeypatch.setenv("UNOCG_LINE_TP_BLOCKS", str(blocks))
        info, C = _mixed(phase, loads, flexible)
        assert info.status == _lib.OK, (tp, blocks)
        assert np.all(info.true_rel_res <= 1e-6), (tp, blocks)
        assert np.all(info.iters <= np.array(ref["iters"]) + 8), (tp, blocks, info.iters, ref["iters"])
        assert rel(C, C_ref) < 1e-6, (tp, blocks)
        res[(tp, blocks)] = C
    for key, C in res.items():
        assert rel(C, res[(0, 0)]) < 1e-6, key
