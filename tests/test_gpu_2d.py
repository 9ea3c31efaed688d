"""2D problems (Sec. 6 with d = 2: thermal and plane-strain elasticity, periodic / Dirichlet /
mixed BC) through the 3D path as x3-invariant problems on an extruded grid, against the
bilinear 2D oracle (``oracle/fem2d.py``).  The x3-invariant 3D solution equals the 2D one on
every layer, and CG takes the same iterations (pinned on the oracle side in
``tests/test_oracle_fem2d.py``)."""
import numpy as np
import pytest

from oracle import fem2d as f2
from synth import rsa_disks
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _props(physics):
    return np.array([1.0, 10.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])


@pytest.mark.parametrize("bc", [(0, 0), (0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("physics,shape", [(1, (12, 10)), (3, (10, 12)), (1, (32, 48))])
def test_2d_solves_match_oracle(bc, physics, shape):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization2D
    phase, _ = rsa_disks(shape, shape[0] / 6.0, 0.3, seed=5)
    props = _props(physics)
    dim = 2 if physics == 1 else 3
    loads = np.eye(dim)
    bcb = tuple(bool(b) for b in bc)
    ref = f2.solve(phase, props, physics, bcb, loads, precond="uno", tol=1e-10)
    Cref = f2.effective_tensor(phase, props, physics, bcb, ref["u"], loads)
    h = Homogenization2D(physics, shape, bc=bc)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-10, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64, flexible=0)
    assert info.status == _lib.OK
    for l in range(dim):
        assert abs(int(info.iters[l]) - ref["iters"][l]) <= 1
        assert rel(h.fluctuation(0, l), ref["u"][l]) < 1e-9
    assert rel(h.effective_tensor()[0], Cref) < 1e-10
    info = h.solve(tol=1e-6, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED,
                   flexible=0 if any(bc) else 1)
    assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
    assert rel(h.effective_tensor()[0], Cref) < 1e-6
    h.close()


def test_table3_iterations_400():
    """Table 3's 2D thermal setting (400 x 400 pixels, kappa = 1 and 0.2, tolerance 1e-6) on a
    synthetic disk microstructure: the reference-medium UNO (the FANS fundamental solution,
    condition number at most 5) converges in about the paper's 14 iterations, Jacobi and plain
    CG in hundreds to about a thousand (paper: 895 and 1039 on its sample)."""
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization2D
    shape = (400, 400)
    phase, _ = rsa_disks(shape, 12.0, 0.3, seed=1)
    h = Homogenization2D(_lib.THERMAL, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(np.array([1.0, 0.2]))
    h.set_macro_load(np.eye(2)[:1])
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    its = {}
    for name, pc in (("fans", _lib.PRECOND_UNO), ("jacobi", _lib.PRECOND_JACOBI), ("cg", _lib.PRECOND_NONE)):
        info = h.solve(tol=1e-6, max_iter=20000, precond=pc, precision=_lib.FP64, flexible=0)
        assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
        its[name] = int(info.iters[0])
    print("2D 400^2 iterations", its)
    assert 8 <= its["fans"] <= 20
    assert its["jacobi"] > 20 * its["fans"] and its["cg"] > its["jacobi"] * 0.9
    h.close()
