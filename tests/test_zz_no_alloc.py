"""The allocation-free UNO apply (static device scratch) against the allocating entry point.

Collected last so that it also runs after every other GPU test of the session."""
import numpy as np
import pytest

from synth import random_field, random_phase

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("physics,shape", [(1, (16, 12, 20)), (3, (8, 10, 12)), (3, (64, 64, 64)),
                                           (1, (2, 256, 256))])
def test_noalloc_apply_matches_allocating_apply(physics, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=4)
    props = np.array([1.0, 9.0]) if physics == 1 else np.array([[1.0, 0.3], [9.0, 0.2]])
    ctx = api.unocg_create(physics, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 2)
    api.unocg_set_phase_properties(ctx, props)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    for call in range(2):  # two calls in a row on the same scratch
        r = torch.tensor(random_field((c,) + shape, seed=50 + call), device="cuda")
        s_ref = torch.empty_like(r)
        s_na = torch.full_like(r, float("nan"))
        api.unocg_apply_uno_dev(ctx, 0, r, s_ref)
        api.unocg_apply_uno_dev_noalloc(ctx, 0, r, s_na)
        torch.cuda.synchronize()
        a, b = s_na.cpu().numpy(), s_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    api.unocg_destroy(ctx)


def test_noalloc_rejects_grids_beyond_the_scratch():
    import torch
    from paper_2508_02681_gb300 import _lib, api
    shape = (128, 128, 128)  # 128 * 128 * 65 = 1064960 complex values > 524288
    ctx = api.unocg_create(1, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, np.zeros(shape, np.uint8), 1)
    api.unocg_set_phase_properties(ctx, np.array([1.0]))
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    r = torch.zeros((1,) + shape, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(r)
    with pytest.raises(_lib.UnocgError) as ei:
        api.unocg_apply_uno_dev_noalloc(ctx, 0, r, s)
    assert ei.value.code == _lib.ERR_INVALID_ARG and "static scratch" in str(ei.value)
    api.unocg_destroy(ctx)


def test_noalloc_needs_prepared_weights():
    import torch
    from paper_2508_02681_gb300 import _lib, api
    shape = (8, 8, 8)
    ctx = api.unocg_create(1, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, np.zeros(shape, np.uint8), 1)
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)  # no properties yet: not prepared
    r = torch.zeros((1,) + shape, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.UnocgError) as ei:
        api.unocg_apply_uno_dev_noalloc(ctx, 0, r, torch.zeros_like(r))
    assert ei.value.code == _lib.ERR_STATE
    api.unocg_destroy(ctx)


def test_noalloc_back_to_back_on_a_side_stream():
    """Two allocation-free applies with different inputs, enqueued back to back on a side stream
    with no synchronisation between them: the second reuses the scratch after the first in
    stream order, and both results match the allocating apply."""
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c, shape = 3, (16, 16, 24)
    phase = random_phase(shape, 2, seed=8)
    ctx = api.unocg_create(3, 1, *shape, 1.0)
    api.unocg_set_microstructure(ctx, phase, 2)
    api.unocg_set_phase_properties(ctx, np.array([[1.0, 0.3], [20.0, 0.2]]))
    api.unocg_set_uno_weights(ctx, _lib.W_REFERENCE_MEDIUM)
    rs = [torch.tensor(random_field((c,) + shape, seed=70 + k), device="cuda") for k in range(2)]
    outs = [torch.full_like(r, float("nan")) for r in rs]
    refs = [torch.empty_like(r) for r in rs]
    for r, ref in zip(rs, refs):
        api.unocg_apply_uno_dev(ctx, 0, r, ref)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # inputs written before the side stream reads them
    for r, out in zip(rs, outs):
        api.unocg_apply_uno_dev_noalloc(ctx, 0, r, out, stream=side)
    side.synchronize()
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    api.unocg_destroy(ctx)
