"""Pins of the oracle for boundary conditions chosen per axis (Sec. 4.1, Sec. 6.2 mixed BC,
Table (fnocg-mode-selection-2d)): the all-Dirichlet and all-periodic cases reduce to the
separately pinned oracles, and the mixed case obeys the energy ordering of nested fluctuation
spaces, Hill's lemma and the direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dirichlet as dr, fem, homogenize as hz, mixedbc as mb, uno
from synth import random_phase, rsa_spheres

DIR = (True, True, True)
PER = (False, False, False)
MIX = (False, True, False)   # Dirichlet on the faces of axis 2, periodic across the others


@pytest.mark.parametrize("physics,props", [(1, [1.0, 6.0]), (3, [[1.0, 0.3], [5.0, 0.2]])])
def test_all_dirichlet_reduces_to_dirichlet_oracle(physics, props):
    shape = (5, 6, 4)
    phase = random_phase(shape, 2, seed=1)
    c = mb.n_comp(physics)
    K1 = mb.assemble_K(phase, props, physics, DIR).toarray()
    K2 = dr.assemble_K(phase, props, physics).toarray()
    assert np.max(np.abs(K1 - K2)) < 1e-14
    load = np.arange(1, 4 if c == 1 else 7) * 0.3
    assert np.max(np.abs(mb.assemble_f(phase, props, physics, DIR, load) - dr.assemble_f(phase, props, physics, load))) < 1e-14
    assert np.max(np.abs(mb.reference_Q(physics, props, shape, DIR) - dr.reference_Q(physics, props, shape))) < 1e-10
    r = np.random.default_rng(2).standard_normal((c,) + dr.free_shape(shape))
    Q = dr.reference_Q(physics, props, shape)
    assert np.max(np.abs(mb.uno_apply(Q, r, shape, DIR) - dr.uno_apply(Q, r))) < 1e-12


@pytest.mark.parametrize("physics,props", [(1, [1.0, 6.0]), (3, [[1.0, 0.3], [5.0, 0.2]])])
def test_all_periodic_reduces_to_periodic_oracle(physics, props):
    shape = (4, 6, 6)
    phase = random_phase(shape, 2, seed=3)
    c = mb.n_comp(physics)
    assert np.max(np.abs(mb.assemble_K(phase, props, physics, PER).toarray()
                         - fem.assemble_K(phase, props, physics).toarray())) < 1e-14
    load = np.arange(1, 4 if c == 1 else 7) * 0.3
    assert np.max(np.abs(mb.assemble_f(phase, props, physics, PER, load) - fem.assemble_f(phase, props, physics, load))) < 1e-14
    Qf = mb.reference_Q(physics, props, shape, PER)
    Qh = uno.reference_medium_Q(physics, props, shape)
    assert np.max(np.abs(Qf[:, :, : shape[2] // 2 + 1] - Qh)) < 1e-10 * np.max(np.abs(Qh))
    r = np.random.default_rng(4).standard_normal((c,) + shape)
    assert np.max(np.abs(mb.uno_apply(Qf, r, shape, PER) - uno.uno_apply(Qh, r))) < 1e-10
    loads = np.eye(3 if c == 1 else 6)[:2]
    a = mb.solve(phase, props, physics, PER, loads, tol=1e-11)
    b = hz.solve(phase, props, physics, loads, tol=1e-11)
    for l in range(2):
        assert np.max(np.abs(a["u"][l] - b["u"][l])) < 1e-9 * np.max(np.abs(b["u"][l]))


def test_conjugate_modes_needed_for_a_real_output():
    shape = (6, 5, 4)
    rng = np.random.default_rng(5)
    Q = rng.random(mb.free_shape(shape, MIX) + (1, 1)) + 0.5
    r = rng.standard_normal((1,) + mb.free_shape(shape, MIX))
    with pytest.raises(AssertionError):
        mb.uno_apply(Q, r, shape, MIX)
    Qs = mb.symmetrize(Q, MIX)
    s = mb.uno_apply(Qs, r, shape, MIX)
    assert np.sum(r * s) > 0
    # symmetrization is a projection
    assert np.max(np.abs(mb.symmetrize(Qs, MIX) - Qs)) < 1e-15


@pytest.mark.parametrize("physics", [1, 3])
def test_mixed_reference_weights_and_homogeneous_cell(physics):
    shape = (6, 5, 8)
    c = mb.n_comp(physics)
    props = [2.0] if physics == 1 else [[3.0, 0.25]]
    phase = np.zeros(shape, np.uint8)
    B = mb.transformed_blocks(physics, fem.material_matrix(physics, props[0]), shape, MIX)
    # brute force: the dense transform of the assembled homogeneous operator
    K = mb.assemble_K(phase, props, physics, MIX).toarray()
    Ms = mb.free_shape(shape, MIX)
    T = np.kron(np.kron(mb.axis_matrix(shape[0], False), mb.axis_matrix(shape[1], True)), mb.axis_matrix(shape[2], False))
    for a in range(c):
        for b in range(c):
            full = T.conj() @ K[a::c, b::c] @ T.T
            assert np.max(np.abs(np.diag(full).reshape(Ms) - B[..., a, b])) < 1e-13
            if physics == 1:
                assert np.max(np.abs(full - np.diag(np.diag(full)))) < 1e-13
    loads = np.eye(3 if c == 1 else 6)
    assert np.max(np.abs(mb.assemble_f(phase, props, physics, MIX, loads[0]))) < 1e-14
    out = mb.solve(phase, props, physics, MIX, loads, tol=1e-10)
    C = mb.effective_tensor(phase, props, physics, MIX, out["u"], loads)
    assert np.max(np.abs(C - fem.material_matrix(physics, props[0]))) < 1e-13


@pytest.mark.parametrize("physics,props,load", [
    (1, [1.0, 10.0], [0.4, -1.0, 0.7]),
    (3, [[1.0, 0.3], [10.0, 0.2]], [0.2, -0.5, 1.0, 0.3, -0.2, 0.6])])
def test_mixed_energy_between_periodic_and_dirichlet(physics, props, load):
    """Dirichlet fields (zero on all faces) are mixed fields, and mixed fields (zero on the
    axis-2 faces, periodic across the others) are periodic ones: W_per <= W_mix <= W_dir."""
    shape = (6, 6, 6)
    phase, _ = rsa_spheres(shape, 1.6, 0.3, seed=3)
    W = {}
    for name, bc in (("per", PER), ("mix", MIX), ("dir", DIR)):
        out = mb.solve(phase, props, physics, bc, [load], precond="uno", tol=1e-12)
        u = out["u"][0]
        ud = spla.spsolve(out["K"].tocsc(), out["f"][0])
        if name == "per":
            c = mb.n_comp(physics)
            v = ud.reshape(-1, c)
            ud = (v - v.mean(axis=0)).ravel()
        assert np.max(np.abs(u - ud)) < 1e-9 * np.max(np.abs(ud))
        C = mb.effective_tensor(phase, props, physics, bc, [u], [load])[:, 0]
        W[name] = float(C @ np.asarray(load))
        # mean gradient of the fluctuation vanishes (periodic faces cancel, Dirichlet faces are zero)
        eps = mb.element_mean_strain(u, shape, bc, physics)
        assert np.max(np.abs(eps.mean(axis=0))) < 1e-13
    assert W["per"] < W["mix"] < W["dir"]
