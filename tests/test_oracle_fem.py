"""Pins of the oracle's finite-element layer against closed forms and invariants."""
import numpy as np
import pytest

from oracle import fem, uno
from synth import random_phase, rsa_spheres


def test_thermal_element_matrix_by_corner_distance():
    # Trilinear brick Laplacian on the unit cube: 1/3 on the diagonal, 0 between edge
    # neighbours, -1/12 across face diagonals and the body diagonal.
    K = fem.element_stiffness(1, np.eye(3), 1.0)
    expect = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}
    for a in range(8):
        for b in range(8):
            dist = int(np.sum(fem.CORNERS[a] != fem.CORNERS[b]))
            assert K[a, b] == pytest.approx(expect[dist], abs=1e-15)


def test_elastic_element_rigid_modes_and_uniform_strain():
    lam, mu = 1.7, 0.6
    E = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    D = fem.material_matrix(3, (E, nu))
    h = 0.37
    K = fem.element_stiffness(3, D, h)
    ev = np.linalg.eigvalsh(K)
    # exactly six rigid-body modes (3 translations, 3 rotations)
    assert np.sum(np.abs(ev) < 1e-12 * ev.max()) == 6
    assert np.all(ev > -1e-12 * ev.max())
    x = fem.CORNERS * h
    rng = np.random.default_rng(3)
    W = rng.standard_normal((3, 3))
    W = W - W.T
    u_rot = (x @ W.T).ravel()
    assert np.max(np.abs(K @ u_rot)) < 1e-12
    # a uniform strain field u = eps x stores energy |V| eps:C:eps; Mandel eps = (11,22,33,
    # sqrt2*12, sqrt2*13, sqrt2*23)
    eps = rng.standard_normal((3, 3))
    eps = 0.5 * (eps + eps.T)
    u = (x @ eps.T).ravel()
    s2 = np.sqrt(2.0)
    em = np.array([eps[0, 0], eps[1, 1], eps[2, 2], s2 * eps[0, 1], s2 * eps[0, 2], s2 * eps[1, 2]])
    tr = np.trace(eps)
    energy = h ** 3 * (lam * tr * tr + 2 * mu * np.sum(eps * eps))
    assert u @ K @ u == pytest.approx(energy, rel=1e-12)
    assert em @ D @ em == pytest.approx(energy / h ** 3, rel=1e-12)


def test_assembled_homogeneous_thermal_stencil():
    shape = (5, 6, 7)
    kappa = 2.5
    phase = np.zeros(shape, dtype=np.uint8)
    K = fem.assemble_K(phase, [kappa], 1).toarray()
    h = 1.0 / shape[0]
    node = (2 * shape[1] + 3) * shape[2] + 4
    row = K[node].reshape(shape)
    for d1 in (-1, 0, 1):
        for d2 in (-1, 0, 1):
            for d3 in (-1, 0, 1):
                nz = abs(d1) + abs(d2) + abs(d3)
                val = row[2 + d1, 3 + d2, 4 + d3]
                exp = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[nz] * kappa * h
                assert val == pytest.approx(exp, abs=1e-14)
    assert np.count_nonzero(np.abs(row) > 1e-14) == 21


@pytest.mark.parametrize("physics", [1, 3])
def test_K_symmetric_with_constant_null_space(physics):
    shape = (4, 4, 4)
    phase = random_phase(shape, 2, seed=11)
    props = [1.0, 7.0] if physics == 1 else [[1.0, 0.3], [10.0, 0.2]]
    K = fem.assemble_K(phase, props, physics).toarray()
    c = 1 if physics == 1 else 3
    assert np.max(np.abs(K - K.T)) < 1e-14
    n = int(np.prod(shape))
    for j in range(c):
        t = np.zeros(c * n)
        t[j::c] = 1.0
        assert np.max(np.abs(K @ t)) < 1e-13
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10) == c  # null space = constants only
    assert ev.min() > -1e-12


def test_symbol_matches_tensor_product_closed_form():
    # Fourier symbol of the homogeneous stencil = sum_a K1(t_a) prod_{b!=a} M1(t_b) (thermal)
    # with the 1D FE stiffness/mass symbols K1 = 2 - 2cos, M1 = (2 + cos)/3.
    shape = (6, 5, 8)
    h = 1.0 / 6
    S = uno.reference_symbol(1, 2.0, shape)
    k = np.meshgrid(*[np.arange(s) for s in (6, 5, 5)], indexing="ij")
    t = [2 * np.pi * k[a] / shape[a] for a in range(3)]
    K1 = lambda x: 2 - 2 * np.cos(x)
    M1 = lambda x: (2 + np.cos(x)) / 3
    cf = 2.0 * h * (K1(t[0]) * M1(t[1]) * M1(t[2]) + M1(t[0]) * K1(t[1]) * M1(t[2])
                    + M1(t[0]) * M1(t[1]) * K1(t[2]))
    assert np.max(np.abs(S[..., 0, 0] - cf)) < 1e-14
    lam, mu = 1.3, 0.7
    S3 = uno.reference_symbol(3, (lam, mu), shape)
    for a in range(3):
        b_, c_ = (a + 1) % 3, (a + 2) % 3
        saa = (lam + 2 * mu) * K1(t[a]) * M1(t[b_]) * M1(t[c_]) + mu * (
            K1(t[b_]) * M1(t[a]) * M1(t[c_]) + K1(t[c_]) * M1(t[a]) * M1(t[b_]))
        assert np.max(np.abs(S3[..., a, a] - h * saa)) < 1e-14
        sab = (lam + mu) * np.sin(t[a]) * np.sin(t[b_]) * M1(t[c_])
        assert np.max(np.abs(S3[..., a, b_] - h * sab)) < 1e-14


def test_homogeneous_spectrum_and_jacobi_bound():
    # lambda_max(K) = 4 kappa h at theta = (pi, 0, 0); the Jacobi-preconditioned maximum is
    # 4 / (8/3) = 1.5, the value printed for Jac-CG in Table 3.
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table3_spectra.json")))
    shape = (6, 6, 6)
    kappa = 1.3
    K = fem.assemble_K(np.zeros(shape, np.uint8), [kappa], 1).toarray()
    h = 1.0 / 6
    ev = np.linalg.eigvalsh(K)
    assert ev.max() == pytest.approx(4 * kappa * h, rel=1e-12)
    d = np.diag(K)
    evj = np.linalg.eigvals(K / d[:, None]).real
    assert evj.max() == pytest.approx(gold["JacCG"]["lambda_max"], abs=0.5e-4)


def test_rhs_zero_for_homogeneous_and_in_range():
    shape = (5, 4, 6)
    for physics, props, load in [(1, [3.0], [0.3, -1.0, 2.0]),
                                 (3, [[2.0, 0.25]], [1.0, -0.5, 0.2, 0.3, 0.7, -1.1])]:
        f = fem.assemble_f(np.zeros(shape, np.uint8), props, physics, load)
        assert np.max(np.abs(f)) < 1e-14
    phase, _ = rsa_spheres((8, 8, 8), 2.0, 0.3, seed=5)
    f = fem.assemble_f(phase, [1.0, 10.0], 1, [1.0, 0.0, 0.0])
    assert abs(f.sum()) < 1e-13 and np.max(np.abs(f)) > 1e-3
    f3 = fem.assemble_f(phase, [[1.0, 0.3], [10.0, 0.2]], 3, [0, 0, 0, 1.0, 0, 0])
    assert np.max(np.abs(f3.reshape(-1, 3).sum(axis=0))) < 1e-13


def test_thermal_rhs_corner_signs():
    # f_a = -sum_{e contains a} kappa_e (h^2/4) s_a . g, with s_a = 2 o - 1 the corner signs
    shape = (4, 4, 4)
    phase = random_phase(shape, 2, seed=2)
    kap = np.array([1.0, 4.0])
    g = np.array([0.2, -1.0, 0.5])
    f = fem.assemble_f(phase, kap, 1, g)
    h = 0.25
    ref = np.zeros(shape)
    for i1 in range(4):
        for i2 in range(4):
            for i3 in range(4):
                for o in fem.CORNERS:
                    node = ((i1 + o[0]) % 4, (i2 + o[1]) % 4, (i3 + o[2]) % 4)
                    ref[node] -= kap[phase[i1, i2, i3]] * h * h / 4 * np.dot(2 * o - 1, g)
    assert np.max(np.abs(f - ref.ravel())) < 1e-15


@pytest.mark.parametrize("physics,props", [(1, [1.0, 4.0]), (3, [[1.0, 0.3], [4.0, 0.2]])])
def test_residual_at_nodes_matches_assembly(physics, props):
    shape = (4, 5, 6)
    phase = random_phase(shape, 2, seed=21)
    c = 1 if physics == 1 else 3
    rng = np.random.default_rng(3)
    u = rng.standard_normal(c * int(np.prod(shape)))
    load = rng.standard_normal(3 if physics == 1 else 6)
    K = fem.assemble_K(phase, props, physics)
    f = fem.assemble_f(phase, props, physics, load)
    full = (f - K @ u).reshape(-1, c)
    nodes = [(0, 0, 0), (3, 4, 5), (1, 2, 3), (2, 0, 5)]
    got = fem.residual_at_nodes(phase, props, physics, u, load, nodes)
    for q, nd in enumerate(nodes):
        flat = (nd[0] * shape[1] + nd[1]) * shape[2] + nd[2]
        assert np.max(np.abs(got[q] - full[flat])) < 1e-13
