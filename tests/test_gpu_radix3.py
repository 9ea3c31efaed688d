"""Register-FFT passes on axes of 3 x 2^k points (48, 96, 192: 12- and 24-point DFTs in
registers, radix 3 x 4 and 3 x 8, with 2, 4 or 8 threads per line) against the oracle, which
transforms by the DFT's definition.

The UNO apply in FP64 covers the register plane passes of 48^2 and 96^2 planes and the register
axis-1 pass of 48 points; the solves cover the FP32 plane passes of 48^2, 96^2 and 192^2 planes
and the TMA axis-1 pass of 48, 96 and 192 points (mixed precision), with the FP64 loop on the
same inputs.  Bars as for the other solves: FP64 effective tensors within 1e-7 of the oracle's
at the tolerance 1e-6 (CG iterates differ by rounding there, see test_gpu_fullsize), mixed
effective tensors within 1e-6 with a true FP64 residual at the tolerance."""
import numpy as np
import pytest

from oracle import homogenize as hz
from oracle import uno
from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _props(physics):
    return np.array([1.0, 20.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", [(48, 48, 48), (8, 96, 96), (48, 16, 20), (6, 48, 48)])
def test_uno_apply_radix3_axes(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=8)
    props = _props(physics)
    ctx = api.unocg_create(physics, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 2)
    api.unocg_set_phase_properties(ctx, props)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    r = random_field((c,) + shape, seed=12)
    s_ref = uno.uno_apply(uno.reference_medium_Q(physics, props, shape), r)
    rr = torch.tensor(r, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_apply_uno_dev(ctx, 0, rr, ss)
    torch.cuda.synchronize()
    assert rel(ss.cpu().numpy(), s_ref) < 1e-12 * max(1.0, (max(shape) / 64.0) ** 2)
    api.unocg_destroy(ctx)


def _solve_pair(physics, shape, radius, nloads):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    phase, _ = rsa_spheres(shape, radius, 0.25, seed=9)
    props = _props(physics)
    loads = unit_loads(physics)[:nloads]
    ref = hz.solve(phase, props, physics, loads, precond="uno", tol=TOL)
    C_ref = hz.effective_tensor(phase, props, physics, ref["u"], loads)
    out = {}
    for prec in (_lib.FP64, _lib.MIXED):
        h = Homogenization(physics, shape)
        h.set_microstructure(phase, 2)
        h.set_phase_properties(props)
        h.set_macro_load(loads)
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        info = h.solve(tol=TOL, max_iter=2000, precond=_lib.PRECOND_UNO, precision=prec)
        assert info.status == _lib.OK
        assert np.all(info.true_rel_res <= TOL)
        out[prec] = (info, h.effective_tensor()[0])
        h.close()
    info64, C64 = out[_lib.FP64]
    for l in range(nloads):
        assert abs(int(info64.iters[l]) - ref["iters"][l]) <= 1, (l, int(info64.iters[l]), ref["iters"][l])
    assert rel(C64, C_ref) < 1e-7
    assert rel(out[_lib.MIXED][1], C_ref) < 1e-6


@pytest.mark.parametrize("shape,radius", [((48, 48, 48), 4.5), ((192, 32, 32), 4.0), ((96, 96, 96), 9.0),
                                          ((4, 192, 192), 3.0)])
def test_thermal_solve_radix3_axes(shape, radius):
    _solve_pair(1, shape, radius, 1 if max(shape) >= 96 else 2)


def test_elastic_solve_radix3_axes():
    _solve_pair(3, (48, 48, 48), 4.5, 2)
