"""Edge cases of the Dirichlet / mixed-BC path against the oracle: one free node, single-point
and two-point lines, odd and even pair counts, the largest axis the passes accept (512), a
homogeneous cell with zero right-hand side, and batches whose instances converge at
different iterations."""
import numpy as np
import pytest

from oracle import fem, mixedbc as mb
from synth import random_field, random_phase, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _ctx(physics, phase, props, bc, loads=None, batch=1):
    from paper_2508_02681_gb300.solver import DirichletHomogenization
    h = DirichletHomogenization(physics, phase.shape[-3:], batch=batch, bc=bc)
    h.set_microstructure(phase, int(phase.max()) + 1)
    h.set_phase_properties(props)
    if loads is not None:
        h.set_macro_load(loads)
    return h


@pytest.mark.parametrize("shape,bc", [((2, 2, 2), (1, 1, 1)), ((3, 2, 4), (1, 1, 1)), ((2, 3, 4), (0, 1, 0)),
                                      ((4, 2, 3), (1, 0, 1)), ((5, 3, 2), (0, 0, 1)), ((4, 4, 512), (1, 1, 1)),
                                      ((3, 512, 4), (0, 1, 0))])
@pytest.mark.parametrize("physics", [1, 3])
def test_operators_on_degenerate_and_large_axes(shape, bc, physics):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    props = np.array([1.0, 5.0]) if physics == 1 else np.array([[1.0, 0.3], [5.0, 0.2]])
    phase = random_phase(shape, 2, seed=2)
    h = _ctx(physics, phase, props, bc)
    bcb = tuple(bool(b) for b in bc)
    Ms = mb.free_shape(shape, bcb)
    p = random_field((c,) + Ms, seed=3)
    pd = torch.tensor(p, device="cuda")
    qd = torch.empty_like(pd)
    api.unocg_dir_apply_K_dev(h.ctx, 0, pd, qd)
    torch.cuda.synchronize()
    K = mb.assemble_K(phase, props, physics, bcb)
    assert rel(qd.cpu().numpy(), fem.to_soa(K @ fem.from_soa(p), c, Ms)) < 1e-12
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    Q = mb.reference_Q(physics, props, shape, bcb)
    api.unocg_dir_apply_uno_dev(h.ctx, 0, pd, qd)
    torch.cuda.synchronize()
    # the long transforms of the 512-point axis: rounding grows with the transform length and the
    # spread of the reference weights (as for the periodic FFT, 1e-12 x (N / 64)^2)
    tol = 1e-12 * max(1.0, (max(shape) / 64.0) ** 2)
    assert rel(qd.cpu().numpy(), mb.uno_apply(Q, p, shape, bcb)) < tol
    loads = unit_loads(physics)[:2]
    h.set_macro_load(loads)
    ref = mb.solve(phase, props, physics, bcb, loads, tol=1e-10)
    info = h.solve(tol=1e-10, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
    assert info.status == _lib.OK
    for l in range(2):
        assert rel(h.fluctuation(0, l), ref["u"][l]) < 1e-9
    assert rel(h.effective_tensor()[0], mb.effective_tensor(phase, props, physics, bcb, ref["u"], loads)) < 1e-10
    h.close()


@pytest.mark.parametrize("bc", [(1, 1, 1), (0, 1, 0)])
def test_homogeneous_cell_zero_rhs(bc):
    """A homogeneous cell: the right-hand side vanishes up to rounding (exactly for the normal
    strains), the solver stops at once or iterates on rounding noise relative to it, and the
    averaged stress is the material's."""
    from paper_2508_02681_gb300 import _lib
    shape = (8, 8, 8)
    h = _ctx(3, np.zeros(shape, np.uint8), np.array([[2.0, 0.25]]), bc, unit_loads(3))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    for prec in (_lib.FP64, _lib.MIXED):
        info = h.solve(tol=1e-8, max_iter=100, precond=_lib.PRECOND_UNO, precision=prec)
        assert info.status == _lib.OK and np.all(info.iters <= 30)
        assert rel(h.effective_tensor()[0], fem.material_matrix(3, (2.0, 0.25))) < 1e-14
        for l in range(6):
            assert np.max(np.abs(h.fluctuation(0, l))) < 1e-12
    h.close()


def test_batch_with_instances_converging_at_different_iterations():
    """Masks: an instance that converged stays frozen while the others iterate."""
    from paper_2508_02681_gb300 import _lib
    shape = (12, 12, 12)
    ph = np.stack([np.zeros(shape, np.uint8), random_phase(shape, 2, seed=5), random_phase(shape, 2, seed=6)])
    props = np.array([[1.0, 1.0], [1.0, 50.0], [1.0, 5.0]])
    loads = unit_loads(1)[:1]
    h = _ctx(1, ph, props, (1, 1, 1), loads, batch=3)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-10, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
    assert info.status == _lib.OK
    assert info.iters[0] <= 2 and info.iters[1] > info.iters[2] > info.iters[0]
    C = h.effective_tensor()
    for b in range(3):
        ref = mb.solve(ph[b], props[b], 1, (True, True, True), loads, tol=1e-10)
        if b == 0:   # homogeneous: zero fluctuation up to rounding
            assert np.max(np.abs(h.fluctuation(b, 0))) < 1e-14
        else:
            assert abs(ref["iters"][0] - info.iters[b]) <= 1
            assert rel(h.fluctuation(b, 0), ref["u"][0]) < 1e-9
        assert rel(C[b], mb.effective_tensor(ph[b], props[b], 1, (True, True, True), ref["u"], loads)) < 1e-10
    h.close()
