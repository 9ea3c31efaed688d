"""Failure detection without a GPU fault (host-side injections): invalid arguments, corrupted
weights, NaN in the inputs, exhausted iteration budgets; every failure is a status code and the
context stays usable for the next solve."""
import numpy as np
import pytest

from synth import rsa_spheres, unit_loads

pytestmark = pytest.mark.gpu


def _periodic(shape=(16, 16, 16)):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=8)
    h = Homogenization(_lib.THERMAL, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([1.0, 10.0]))
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


def _dirichlet(shape=(16, 16, 16), bc=(1, 1, 1)):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import DirichletHomogenization
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=8)
    h = DirichletHomogenization(_lib.THERMAL, shape, bc=bc)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([1.0, 10.0]))
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


@pytest.mark.parametrize("make", [_periodic, _dirichlet])
def test_non_finite_load_is_rejected_and_the_context_stays_usable(make):
    """A NaN in a load would make every entry of that right-hand side NaN; the max-norm
    reduction (fmax drops NaN) would read it as zero and the stopping test as converged, so
    the load is rejected on the host."""
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300._lib import UnocgError
    h = make()
    good = h.solve(tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64, flexible=0)
    C0 = h.effective_tensor()[0]
    for v in (np.nan, np.inf):
        bad = unit_loads(1).copy()
        bad[1, 2] = v
        with pytest.raises(UnocgError) as e:
            h.set_macro_load(bad)
        assert e.value.code == _lib.ERR_INVALID_ARG
    info = h.solve(tol=1e-8, max_iter=500, precond=_lib.PRECOND_UNO, precision=_lib.FP64, flexible=0)
    assert info.status == _lib.OK and np.array_equal(info.iters, good.iters)
    assert np.max(np.abs(h.effective_tensor()[0] - C0)) < 1e-14 * np.max(np.abs(C0))
    h.close()


@pytest.mark.parametrize("make", [_periodic, _dirichlet])
def test_iteration_budget_and_recovery(make):
    from paper_2508_02681_gb300 import _lib
    h = make()
    info = h.solve(raise_on_error=False, tol=1e-12, max_iter=3, precond=_lib.PRECOND_JACOBI, precision=_lib.FP64,
                   flexible=0)
    assert info.status == _lib.ERR_NOT_CONVERGED and np.all(info.iters == 3)
    info = h.solve(tol=1e-8, max_iter=2000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED, flexible=0)
    assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-8)
    h.close()


def test_invalid_inputs_are_rejected_before_any_launch():
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300._lib import UnocgError
    h = _periodic()
    for props in (np.array([1.0, np.nan]), np.array([1.0, -2.0]), np.array([np.inf, 1.0])):
        with pytest.raises(UnocgError) as e:
            h.set_phase_properties(props)
        assert e.value.code == _lib.ERR_INVALID_ARG
    with pytest.raises(UnocgError):
        h.set_microstructure(np.full((16, 16, 16), 5, np.uint8), 2)  # label out of range
    nh = 16 * 16 * 9
    with pytest.raises(UnocgError) as e:
        h.set_uno_weights(_lib.W_BLOCKS, np.full(nh, np.nan))          # corrupted weights
    assert e.value.code == _lib.ERR_NOT_SPD
    with pytest.raises(UnocgError) as e:
        h.solve(tol=-1.0, precond=_lib.PRECOND_UNO)
    assert e.value.code == _lib.ERR_INVALID_ARG
    h.close()
    d = _dirichlet()
    with pytest.raises(UnocgError):
        d.set_phase_properties(np.array([np.nan, 1.0]))
    with pytest.raises(UnocgError) as e:
        d.set_uno_weights(_lib.W_BLOCKS, np.full(15 ** 3, np.nan))
    assert e.value.code == _lib.ERR_NOT_SPD
    with pytest.raises(UnocgError):
        d.solve(flexible=1, precond=_lib.PRECOND_UNO)
    d.close()
