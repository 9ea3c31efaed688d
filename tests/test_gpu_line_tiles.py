"""The TMA-staged axis-1 pass of the mixed-precision loop in both tile widths (16 positions per
block with the 128-byte swizzle, 8 with the 64-byte swizzle; UNOCG_LINE_P selects one, read at
every launch) on long axis-1 lines, against the oracle's flexible PCG: effective tensor within
1e-6 and the true FP64 residual at the tolerance, both widths within rounding of each other."""
import numpy as np
import pytest

from oracle import homogenize as hz
from synth import rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

PROPS = np.array([1.0, 20.0])


@pytest.fixture(scope="module", params=[(256, 16, 16), (128, 24, 24), (64, 20, 20)])
def case(request):
    shape = request.param
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=11)
    loads = unit_loads(1)[:2]
    ref = hz.solve(phase, PROPS, 1, loads, precond="uno", tol=1e-9, flexible=True)
    C = hz.effective_tensor(phase, PROPS, 1, ref["u"], loads)
    return phase, loads, ref, C


def _mixed(phase, loads):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    h = Homogenization(_lib.THERMAL, phase.shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(PROPS)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=1)
    C = h.effective_tensor()[0]
    h.close()
    return info, C


def test_line_tile_widths_match_oracle(case, monkeypatch):
    from paper_2508_02681_gb300 import _lib
    phase, loads, ref, C_ref = case
    out = {}
    for p in (16, 8):
        monkeypatch.setenv("UNOCG_LINE_P", str(p))
        info, C = _mixed(phase, loads)
        assert info.status == _lib.OK
        assert np.all(info.true_rel_res <= 1e-6)
        assert np.all(info.iters <= np.array(ref["iters"]) + 8)
        assert rel(C, C_ref) < 1e-6
        out[p] = (info, C)
    assert rel(out[16][1], out[8][1]) < 1e-6
