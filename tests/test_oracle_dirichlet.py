"""Pins of the oracle's Dirichlet-BC layer (Sec. 4.1, Sec. 6, Dirichlet row of Table
(fnocg-mode-selection-2d)) against textbook facts, the periodic assembly and brute force."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dirichlet as dr, fem
from synth import random_phase, rsa_spheres


def test_dst_orthonormal_involution_and_1d_laplacian():
    for N in (2, 5, 8, 13):
        S = dr.dst_matrix(N)
        assert np.max(np.abs(S - S.T)) < 1e-15
        assert np.max(np.abs(S @ S - np.eye(N - 1))) < 1e-13
        # the 1D Dirichlet Laplacian tridiag(-1, 2, -1) has eigenvectors S[k] and eigenvalues
        # 2 - 2 cos(pi (k+1) / N)
        L = 2 * np.eye(N - 1) - np.eye(N - 1, k=1) - np.eye(N - 1, k=-1)
        lam = 2 - 2 * np.cos(np.pi * np.arange(1, N) / N)
        assert np.max(np.abs(S @ L @ S - np.diag(lam))) < 1e-13


@pytest.mark.parametrize("physics,props", [(1, [1.0, 7.0]), (3, [[1.0, 0.3], [6.0, 0.2]])])
def test_K_spd_and_interior_rows_match_periodic_assembly(physics, props):
    shape = (6, 7, 8)
    phase = random_phase(shape, 2, seed=4)
    c = dr.n_comp(physics)
    K = dr.assemble_K(phase, props, physics)
    Kd = K.toarray()
    assert np.max(np.abs(Kd - Kd.T)) < 1e-14
    assert np.linalg.eigvalsh(Kd).min() > 1e-6 * np.abs(Kd).max()  # no null space left
    # a field supported on free nodes 2..N-2 (full-grid index) sees the same stencil as in the
    # periodic assembly of the same voxels, on the rows of nodes 1..N-1
    rng = np.random.default_rng(0)
    M = dr.free_shape(shape)
    v = np.zeros((c,) + M)
    v[:, 1:-1, 1:-1, 1:-1] = rng.standard_normal((c,) + tuple(m - 2 for m in M))
    got = fem.to_soa(K @ fem.from_soa(v), c, M)
    vp = np.zeros((c,) + shape)
    vp[:, 1:, 1:, 1:] = v           # full-grid node i = free node i - 1; wrap never reached
    Kp = fem.assemble_K(phase, props, physics)
    ref = fem.to_soa(Kp @ fem.from_soa(vp), c, shape)[:, 1:, 1:, 1:]
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("physics", [1, 3])
def test_transformed_blocks_match_dense_transform(physics):
    shape = (4, 5, 6)
    c = dr.n_comp(physics)
    props = [2.0] if physics == 1 else [[3.0, 0.25]]
    D = fem.material_matrix(physics, props[0])
    B = dr.transformed_blocks(physics, D, shape)
    K = dr.assemble_K(np.zeros(shape, np.uint8), props, physics).toarray()
    M = dr.free_shape(shape)
    n = int(np.prod(M))
    T = np.kron(np.kron(dr.dst_matrix(shape[0]), dr.dst_matrix(shape[1])), dr.dst_matrix(shape[2]))
    for a in range(c):
        for b in range(c):
            Kab = K[a::c, b::c]
            full = T @ Kab @ T.T
            assert np.max(np.abs(np.diag(full).reshape(M) - B[..., a, b])) < 1e-13
            if a == b and physics == 1:
                # the sine transform diagonalizes the homogeneous thermal operator
                assert np.max(np.abs(full - np.diag(np.diag(full)))) < 1e-13
    if physics == 3:
        # couplings of different components have no diagonal in the sine basis
        for a in range(3):
            for b in range(3):
                if a != b:
                    assert np.max(np.abs(B[..., a, b])) < 1e-13


def test_reference_weights_invert_the_homogeneous_thermal_operator():
    shape = (6, 5, 7)
    phase = np.zeros(shape, np.uint8)
    K = dr.assemble_K(phase, [3.0], 1)
    Q = dr.reference_Q(1, [3.0], shape)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(dr.free_shape(shape))
    y = dr.uno_apply(Q, fem.to_soa(K @ x.ravel(), 1, dr.free_shape(shape)))
    assert np.max(np.abs(y[0] - x)) < 1e-12 * np.max(np.abs(x))
    # PCG with these weights converges in one iteration
    from oracle import pcg
    f = K @ rng.standard_normal(K.shape[0])
    M = dr.free_shape(shape)
    P = lambda r: dr.uno_apply(Q, r.reshape((1,) + M)).ravel()
    _, it, _ = pcg.pcg(lambda x: K @ x, f, P, 1e-10, 10)
    assert it == 1


@pytest.mark.parametrize("physics", [1, 3])
def test_uno_apply_identity_and_positive(physics):
    shape = (5, 6, 4)
    c = dr.n_comp(physics)
    M = dr.free_shape(shape)
    rng = np.random.default_rng(5)
    r = rng.standard_normal((c,) + M)
    I = np.broadcast_to(np.eye(c), M + (c, c))
    assert np.max(np.abs(dr.uno_apply(I, r) - r)) < 1e-13
    Q = dr.reference_Q(physics, [1.0] if c == 1 else [[1.0, 0.3]], shape)
    assert np.all(np.linalg.eigvalsh(Q) > 0)
    assert float(np.sum(r * dr.uno_apply(Q, r))) > 0


@pytest.mark.parametrize("physics,props,load", [
    (1, [1.0, 10.0], [0.4, -1.0, 0.7]),
    (3, [[1.0, 0.3], [10.0, 0.2]], [0.2, -0.5, 1.0, 0.3, -0.2, 0.6])])
def test_solution_energy_bounds_and_hill_lemma(physics, props, load):
    shape = (6, 6, 6)
    phase, _ = rsa_spheres(shape, 1.6, 0.3, seed=3)
    c = dr.n_comp(physics)
    out = dr.solve(phase, props, physics, [load], precond="uno", tol=1e-12)
    u = out["u"][0]
    K = out["K"]
    # PCG agrees with a direct sparse solve
    ud = spla.spsolve(K.tocsc(), out["f"][0])
    assert np.max(np.abs(u - ud)) < 1e-9 * np.max(np.abs(ud))
    # energy of the full field (affine macroscopic part + fluctuation) from the assembled
    # full-grid K: the nodal interpolant of eps_bar . x is exact for trilinear elements
    h = fem.spacing(shape)
    N = np.asarray(shape)
    X = np.stack(np.meshgrid(*[np.arange(n + 1) * h for n in N], indexing="ij"), axis=-1).reshape(-1, 3)
    if physics == 1:
        aff = X @ np.asarray(load)
    else:
        e = np.asarray(load)
        s2 = np.sqrt(2.0)
        E = np.array([[e[0], e[3] / s2, e[4] / s2], [e[3] / s2, e[1], e[5] / s2], [e[4] / s2, e[5] / s2, e[2]]])
        aff = (X @ E.T).ravel()
    w = aff + dr.extend_to_full(u, shape, c)
    Kf = dr.assemble_K_full(phase, props, physics)
    vol = float(np.prod(N * h))
    W = float(w @ (Kf @ w)) / vol
    C = dr.effective_tensor(phase, props, physics, [u], [load])[:, 0]
    # Hill's lemma for kinematic boundary conditions: <sigma> . eps_bar = <sigma . eps>
    assert float(C @ np.asarray(load)) == pytest.approx(W, rel=1e-9)
    # the fluctuation space of Dirichlet BC is a subspace of the periodic one: more energy
    # than with periodic BC, less than the Voigt bound
    from oracle import homogenize
    per = homogenize.solve(phase, props, physics, [load], precond="uno", tol=1e-12)
    Cp = homogenize.effective_tensor(phase, props, physics, per["u"], [load])[:, 0]
    Wp = float(Cp @ np.asarray(load))
    D = np.stack([fem.material_matrix(physics, p) for p in np.asarray(props, dtype=float)])
    Dv = np.einsum("eij->ij", D[phase.ravel()]) / phase.size
    Wv = float(np.asarray(load) @ Dv @ np.asarray(load))
    assert Wp < W < Wv
    # mean gradient of a field that vanishes on the boundary is zero
    eps = dr.element_mean_strain(u, shape, physics)
    assert np.max(np.abs(eps.mean(axis=0))) < 1e-13


def test_homogeneous_returns_its_own_tensor():
    shape = (5, 4, 6)
    for physics, props, dim in ((1, [2.5], 3), (3, [[4.0, 0.3]], 6)):
        phase = np.zeros(shape, np.uint8)
        loads = np.eye(dim)
        f = dr.assemble_f(phase, props, physics, loads[0])
        assert np.max(np.abs(f)) < 1e-14
        out = dr.solve(phase, props, physics, loads, tol=1e-10)
        C = dr.effective_tensor(phase, props, physics, out["u"], loads)
        assert np.max(np.abs(C - fem.material_matrix(physics, props[0]))) < 1e-13


def test_modes_layout_counts_and_bypass():
    # Table (fnocg-mode-selection-2d), Dirichlet row: (2M+1)^d learned modes, no conjugates;
    # off the mode set Q is the bypass, on it bypass plus mode block
    from oracle import uno
    shape = (8, 9, 10)
    for c in (1, 3):
        M = 2
        modes = dr.mode_list(M)
        assert len(modes) == (2 * M + 1) ** 3 and len(set(modes)) == len(modes)
        rng = np.random.default_rng(c)
        w = rng.standard_normal((1 + len(modes), uno.n_unique(c)))
        Q = dr.modes_Q(w, M, shape, c)
        W0 = uno.psi(w[0], c)
        assert np.max(np.abs(Q[5:, :, :] - W0)) == 0.0
        k = modes[17]
        assert np.max(np.abs(Q[k] - W0 - uno.psi(w[18], c))) < 1e-14
        assert np.all(np.linalg.eigvalsh(Q.reshape(-1, c, c)) > -1e-12)
