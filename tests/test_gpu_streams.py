"""Stream order at the C ABI.  The contexts run on their own non-blocking stream; entry points
that read device results on the host must wait for it, and `_dev` entry points, which enqueue
on the caller's stream (NULL: the legacy default stream, PyTorch's default), must run after the
context's earlier work and before its later work."""
import numpy as np
import pytest

from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def test_weights_read_right_after_they_are_built():
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (96, 96, 96)
    h = Homogenization(_lib.ELASTIC, shape)
    h.set_microstructure(random_phase(shape, 2, seed=4), 2)
    h.set_phase_properties(np.array([[1.0, 0.3], [20.0, 0.2]]))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    nh = shape[0] * shape[1] * (shape[2] // 2 + 1)
    first = api.unocg_get_uno_weights(h.ctx, 0, nh, 6)   # builds the weights, then reads them
    again = api.unocg_get_uno_weights(h.ctx, 0, nh, 6)
    assert np.array_equal(first, again)
    assert np.all(np.isfinite(first))
    h.close()


def test_dev_results_on_the_default_stream():
    import torch
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (48, 48, 48)
    phase, _ = rsa_spheres(shape, 5.0, 0.3, seed=8)
    h = Homogenization(_lib.ELASTIC, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([[1.0, 0.3], [10.0, 0.2]]))
    h.set_macro_load(unit_loads(3))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    h.solve(tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
    ref_u = [h.fluctuation(0, l) for l in range(6)]
    assert torch.cuda.current_stream().cuda_stream == 0   # the legacy default stream
    tmp = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    got = torch.empty((6, 3) + shape, dtype=torch.float32, device="cuda")
    for l in range(6):
        api.unocg_get_fluctuation_dev(h.ctx, 0, l, tmp)   # enqueued on the default stream
        got[l].copy_(tmp)                                  # torch work on the same stream
    out = got.cpu().numpy().astype(np.float64)
    for l in range(6):
        u = ref_u[l].reshape(shape + (3,)).transpose(3, 0, 1, 2)
        assert rel(out[l], u) < 1e-6
    # K d on the default stream reads the context's device inputs written on its own stream
    h.set_phase_properties(np.array([[2.0, 0.3], [20.0, 0.2]]))
    d = torch.tensor(random_field((3,) + shape, seed=9), device="cuda")
    p = torch.empty_like(d)
    api.unocg_apply_K_dev(h.ctx, 0, d, p)
    p2 = torch.empty_like(d)
    torch.cuda.synchronize()
    api.unocg_apply_K_dev(h.ctx, 0, d, p2)
    torch.cuda.synchronize()
    assert torch.equal(p, p2)
    h.close()


def test_dev_apply_on_a_side_stream_orders_against_the_context():
    import torch
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (64, 64, 64)
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(random_phase(shape, 2, seed=5), 2)
    h.set_phase_properties(np.array([1.0, 30.0]))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    r = torch.tensor(random_field((1,) + shape, seed=6), device="cuda")
    side = torch.cuda.Stream()
    s1 = torch.empty_like(r)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        api.unocg_apply_uno_dev(h.ctx, 0, r, s1, stream=side)
    side.synchronize()
    s2 = torch.empty_like(r)
    api.unocg_apply_uno_dev(h.ctx, 0, r, s2)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    h.close()
