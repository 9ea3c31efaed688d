"""GPU parity of single hot-path steps against the oracle: K d, the right-hand side and the UNO
apply P r (reference-medium and psi(theta) weights), on grids that span several tiles, odd
(3- and 5-smooth) lengths and ragged tails."""
import numpy as np
import pytest

from oracle import fem, uno
from synth import random_field, random_phase
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4), (6, 5, 8), (9, 10, 12), (16, 12, 20), (27, 25, 30)]


def _ctx(physics, shape, phase, props, loads=None):
    from paper_2508_02681_gb300 import api
    ctx = api.unocg_create(physics, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, int(np.max(phase)) + 1 if phase.size else 1)
    api.unocg_set_phase_properties(ctx, props)
    if loads is not None:
        api.unocg_set_macro_load(ctx, loads)
    return ctx


def _props(physics, n_ph, seed):
    rng = np.random.default_rng(seed)
    if physics == 1:
        return rng.uniform(0.5, 20.0, size=n_ph)
    return np.stack([rng.uniform(0.5, 20.0, size=n_ph), rng.uniform(0.05, 0.45, size=n_ph)], axis=1)


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_Ku_matches_assembled_K(physics, shape):
    import torch
    from paper_2508_02681_gb300 import api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 3, seed=sum(shape))
    phase[0, 0, 0] = 2
    props = _props(physics, 3, 1)
    ctx = _ctx(physics, shape, phase, props)
    d = random_field((c,) + shape, seed=7)
    K = fem.assemble_K(phase, props, physics)
    p_ref = fem.to_soa(K @ fem.from_soa(d), c, shape)
    dd = torch.tensor(d, device="cuda")
    pp = torch.empty_like(dd)
    api.unocg_apply_K_dev(ctx, 0, dd, pp)
    torch.cuda.synchronize()
    assert rel(pp.cpu().numpy(), p_ref) < 1e-13
    api.unocg_destroy(ctx)


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", SHAPES[:4])
def test_rhs_matches_oracle(physics, shape):
    import torch
    from paper_2508_02681_gb300 import api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=3)
    props = _props(physics, 2, 2)
    rng = np.random.default_rng(4)
    loads = rng.standard_normal((2, 3 if physics == 1 else 6))
    ctx = _ctx(physics, shape, phase, props, loads)
    for l in range(2):
        f_ref = fem.to_soa(fem.assemble_f(phase, props, physics, loads[l]), c, shape)
        f = torch.empty((c,) + shape, dtype=torch.float64, device="cuda")
        api.unocg_rhs_dev(ctx, 0, l, f)
        torch.cuda.synchronize()
        assert rel(f.cpu().numpy(), f_ref) < 1e-13
    api.unocg_destroy(ctx)


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_uno_apply_reference_medium(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=5)
    props = _props(physics, 2, 3)
    ctx = _ctx(physics, shape, phase, props)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    r = random_field((c,) + shape, seed=9)
    Q = uno.reference_medium_Q(physics, props, shape)
    s_ref = uno.uno_apply(Q, r)
    rr = torch.tensor(r, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_apply_uno_dev(ctx, 0, rr, ss)
    torch.cuda.synchronize()
    assert rel(ss.cpu().numpy(), s_ref) < 1e-12
    api.unocg_destroy(ctx)


# power-of-two axes: the register-FFT passes (square planes of 32..128, axis 1 of 16..256)
REG_SHAPES = [(16, 32, 32), (32, 64, 64), (2, 128, 128), (64, 16, 20), (128, 8, 6), (256, 4, 4)]


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", REG_SHAPES)
def test_uno_apply_power_of_two_axes(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=6)
    props = _props(physics, 2, 4)
    ctx = _ctx(physics, shape, phase, props)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    r = random_field((c,) + shape, seed=10)
    Q = uno.reference_medium_Q(physics, props, shape)
    s_ref = uno.uno_apply(Q, r)
    rr = torch.tensor(r, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_apply_uno_dev(ctx, 0, rr, ss)
    torch.cuda.synchronize()
    # the oracle's symbol carries a rounding error ~ eps / theta_min^2 (see test_gpu_large)
    assert rel(ss.cpu().numpy(), s_ref) < 1e-12 * max(1.0, (max(shape) / 64.0) ** 2)
    api.unocg_destroy(ctx)


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("shape", [(4, 6, 8), (10, 9, 12), (16, 16, 16)])
def test_uno_apply_theta_weights(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    C = c * (c + 1) // 2
    phase = random_phase(shape, 2, seed=5)
    props = _props(physics, 2, 3)
    ctx = _ctx(physics, shape, phase, props)
    rng = np.random.default_rng(11)
    theta = rng.standard_normal((shape[0], shape[1], shape[2] // 2 + 1, C)) + 2.0
    api.unocg_set_uno_weights(ctx, _lib.W_THETA, theta, 1e-12)
    Q = uno.symmetrize_half(uno.psi(theta, c), shape[2])
    r = random_field((c,) + shape, seed=10)
    s_ref = uno.uno_apply(Q, r)
    rr = torch.tensor(r, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_apply_uno_dev(ctx, 0, rr, ss)
    torch.cuda.synchronize()
    assert rel(ss.cpu().numpy(), s_ref) < 1e-12
    api.unocg_destroy(ctx)


def test_weights_safety_check_rejects_non_spd():
    from paper_2508_02681_gb300 import _lib, api
    shape = (4, 4, 8)
    phase = random_phase(shape, 2, seed=5)
    ctx = _ctx(1, shape, phase, np.array([1.0, 2.0]))
    v = np.ones((4, 4, 5, 1))
    v[1, 2, 3, 0] = -0.5
    with pytest.raises(_lib.UnocgError) as e:
        api.unocg_set_uno_weights(ctx, _lib.W_BLOCKS, v, 1e-12)
    assert e.value.code == _lib.ERR_NOT_SPD
    api.unocg_destroy(ctx)
