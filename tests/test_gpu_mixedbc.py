"""Mixed boundary conditions (Sec. 6.2: Dirichlet faces on some axes, periodic across the others;
Table (fnocg-mode-selection-2d), mixed row) on the GPU against the FP64 oracle of per-axis BC
(``oracle/mixedbc.py``, Fourier transform along the periodic axes composed with the sine
transform).  The library applies the Fourier part through Hartley passes (with a conversion to
the two-dimensional Hartley spectrum when two axes are periodic); the tests check that the
operator is the paper's.  Bars as for the other boundary conditions."""
import numpy as np
import pytest

from oracle import fem, mixedbc as mb, uno
from synth import random_field, random_phase, rsa_spheres, unit_loads
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

PAPER = (0, 1, 0)  # Dirichlet faces on axis 2, periodic across axes 1 and 3 (Sec. 7, 3D mixed BC)
PATTERNS = [PAPER, (1, 1, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1)]
SHAPES = [(6, 5, 8), (8, 6, 10), (9, 10, 12), (16, 16, 16)]


def _ctx(physics, phase, props, bc, loads=None, batch=1):
    from paper_2508_02681_gb300.solver import DirichletHomogenization
    h = DirichletHomogenization(physics, phase.shape[-3:], batch=batch, bc=bc)
    h.set_microstructure(phase, int(phase.max()) + 1)
    h.set_phase_properties(props)
    if loads is not None:
        h.set_macro_load(loads)
    return h


def _props(physics):
    return np.array([1.0, 10.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])


def _bcb(bc):
    return tuple(bool(b) for b in bc)


@pytest.mark.parametrize("physics", [1, 3])
@pytest.mark.parametrize("bc", PATTERNS)
@pytest.mark.parametrize("shape", SHAPES)
def test_operators_and_reference_weights_match_oracle(physics, bc, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    c = 1 if physics == 1 else 3
    phase = random_phase(shape, 2, seed=3)
    props = _props(physics)
    h = _ctx(physics, phase, props, bc)
    Ms = mb.free_shape(shape, _bcb(bc))
    p = random_field((c,) + Ms, seed=5)
    pd = torch.tensor(p, device="cuda")
    qd = torch.empty_like(pd)
    api.unocg_dir_apply_K_dev(h.ctx, 0, pd, qd)
    torch.cuda.synchronize()
    K = mb.assemble_K(phase, props, physics, _bcb(bc))
    assert rel(qd.cpu().numpy(), fem.to_soa(K @ fem.from_soa(p), c, Ms)) < 1e-12
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    Qref = mb.reference_Q(physics, props, shape, _bcb(bc))
    assert rel(h.uno_weights(0), uno.entries_from_blocks(Qref)) < 1e-12
    api.unocg_dir_apply_uno_dev(h.ctx, 0, pd, qd)
    torch.cuda.synchronize()
    assert rel(qd.cpu().numpy(), mb.uno_apply(Qref, p, shape, _bcb(bc))) < 1e-12
    h.close()


@pytest.mark.parametrize("c,bc,shape", [(1, PAPER, (8, 6, 10)), (3, PAPER, (9, 10, 12)), (3, (0, 0, 1), (6, 8, 5)),
                                        (1, (1, 1, 0), (16, 16, 16))])
def test_theta_weights_are_made_even_and_match_oracle(c, bc, shape):
    import torch
    from paper_2508_02681_gb300 import _lib, api
    physics = 1 if c == 1 else 3
    h = _ctx(physics, random_phase(shape, 2, seed=6), _props(physics), bc)
    Ms = mb.free_shape(shape, _bcb(bc))
    rng = np.random.default_rng(8)
    th = rng.standard_normal(Ms + (uno.n_unique(c),)) * 0.3
    th[..., 0] += 1.0
    if c == 3:
        th[..., 1] += 1.0
        th[..., 3] += 1.0
    h.set_uno_weights(_lib.W_THETA, th)
    Q = mb.symmetrize(uno.psi(th, c), _bcb(bc))
    assert rel(h.uno_weights(0), uno.entries_from_blocks(Q)) < 1e-14
    r = random_field((c,) + Ms, seed=9)
    rd = torch.tensor(r, device="cuda")
    sd = torch.empty_like(rd)
    api.unocg_dir_apply_uno_dev(h.ctx, 0, rd, sd)
    torch.cuda.synchronize()
    assert rel(sd.cpu().numpy(), mb.uno_apply(Q, r, shape, _bcb(bc))) < 1e-12
    h.close()


@pytest.mark.parametrize("physics,shape,bc", [(1, (16, 16, 16), PAPER), (1, (12, 10, 18), PAPER), (3, (8, 10, 12), PAPER),
                                              (3, (16, 16, 16), (1, 0, 1)), (1, (10, 12, 9), (0, 0, 1))])
@pytest.mark.parametrize("precond", ["uno", "jacobi", "none"])
def test_fp64_solve_matches_oracle(physics, shape, bc, precond):
    from paper_2508_02681_gb300 import _lib
    phase, _ = rsa_spheres(shape, shape[0] / 5.0, 0.25, seed=12)
    props = _props(physics)
    loads = unit_loads(physics)[:2]
    tol = 1e-10
    ref = mb.solve(phase, props, physics, _bcb(bc), loads, precond=precond, tol=tol)
    Cref = mb.effective_tensor(phase, props, physics, _bcb(bc), ref["u"], loads)
    h = _ctx(physics, phase, props, bc, loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    pc = {"uno": _lib.PRECOND_UNO, "jacobi": _lib.PRECOND_JACOBI, "none": _lib.PRECOND_NONE}[precond]
    info = h.solve(tol=tol, max_iter=20000, precond=pc, precision=_lib.FP64)
    assert info.status == _lib.OK
    for l in range(2):
        # plain CG runs hundreds of iterations, where the summation order of the dot products
        # (GPU blocks vs NumPy) moves the threshold crossing by a few iterations
        slack = 1 if precond != "none" else max(1, int(0.03 * ref["iters"][l]))
        assert abs(int(info.iters[l]) - ref["iters"][l]) <= slack
        assert rel(h.fluctuation(0, l), ref["u"][l]) < 1e-9
        assert info.true_rel_res[l] <= 2 * tol
    assert rel(h.effective_tensor()[0], Cref) < 1e-10
    h.close()


@pytest.mark.parametrize("physics,shape,bc", [(1, (16, 16, 16), PAPER), (3, (16, 16, 16), PAPER), (1, (32, 32, 32), PAPER),
                                              (1, (24, 20, 30), (1, 0, 0))])
def test_mixed_precision_matches_oracle(physics, shape, bc):
    from paper_2508_02681_gb300 import _lib
    phase, _ = rsa_spheres(shape, shape[0] / 5.0, 0.25, seed=13)
    props = _props(physics)
    loads = unit_loads(physics)
    ref = mb.solve(phase, props, physics, _bcb(bc), loads, precond="uno", tol=1e-10)
    Cref = mb.effective_tensor(phase, props, physics, _bcb(bc), ref["u"], loads)
    h = _ctx(physics, phase, props, bc, loads)
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    info = h.solve(tol=1e-6, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED)
    assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
    assert rel(h.effective_tensor()[0], Cref) < 1e-6
    h.close()


def test_energy_between_periodic_and_dirichlet_on_gpu():
    """Nested fluctuation spaces (Dirichlet within mixed within periodic): the diagonal of the
    averaged-flux tensor orders the same way on the GPU."""
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (32, 32, 32)
    phase, _ = rsa_spheres(shape, 5.0, 0.3, seed=31)
    props = np.array([1.0, 20.0])
    C = {}
    for name, bc in (("mix", PAPER), ("dir", (1, 1, 1))):
        h = _ctx(1, phase, props, bc, unit_loads(1))
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        h.solve(tol=1e-10, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
        C[name] = h.effective_tensor()[0]
        h.close()
    hp = Homogenization(1, shape)
    hp.set_microstructure(phase, 2)
    hp.set_phase_properties(props)
    hp.set_macro_load(unit_loads(1))
    hp.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    hp.solve(tol=1e-10, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
    C["per"] = hp.effective_tensor()[0]
    hp.close()
    for i in range(3):
        assert C["per"][i, i] < C["mix"][i, i] < C["dir"][i, i]


def test_paper_mixed_bc_iterations_64():
    """Sec. 7 (3D mixed BC): the UNO with Fourier x sine transform cuts the Jac-CG iterations on
    the 64^3 thermal and elastic workloads, as for the other boundary conditions."""
    from paper_2508_02681_gb300 import _lib
    shape = (64, 64, 64)
    phase, _ = rsa_spheres(shape, 6.0, 0.3, seed=77)
    for physics, props, red in ((1, np.array([1.0, 100.0]), 3), (3, np.array([[1.0, 0.3], [10.0, 0.2]]), 3)):
        h = _ctx(physics, phase, props, PAPER, unit_loads(physics)[:1])
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        its = {}
        for name, pc in (("uno", _lib.PRECOND_UNO), ("jacobi", _lib.PRECOND_JACOBI)):
            for prec in (_lib.FP64, _lib.MIXED):
                info = h.solve(tol=1e-6, max_iter=20000, precond=pc, precision=prec)
                assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
                its[name, prec] = int(info.iters[0])
        assert its["uno", _lib.FP64] * red < its["jacobi", _lib.FP64]
        h.close()


def test_invalid_patterns():
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300._lib import UnocgError
    with pytest.raises(UnocgError):
        api.unocg_dir_create(1, 1, 8, 8, 8, bc=(0, 0, 0))  # all periodic: the periodic context
    with pytest.raises(UnocgError):
        api.unocg_dir_create(1, 1, 8, 8, 8, bc=(0, 2, 0))
    h = _ctx(1, np.zeros((8, 8, 8), np.uint8), np.array([1.0]), PAPER)
    with pytest.raises(UnocgError):
        h.set_uno_modes(1, np.ones((1 + 27, 1)))  # the mode layout needs Dirichlet faces everywhere
    h.close()
