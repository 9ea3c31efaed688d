"""Pins of the 2D learned-UNO oracle (oracle/uno2d.py, c = 1 and c = 2, periodic BC) against
what the paper and the mathematics fix: the Cholesky-like parametrization of Eq. (local-param-2)
against numpy's Cholesky factor, the loss of Sec. 5.4 from the features of Eq. (features-c-1) /
Eq. (features-c-2) against the loss of Eq. (fnocg-loss) evaluated in real space, the printed
gradient against central differences of that real-space loss, the printed Hessian against
differences of the gradient, exact recovery of a generating operator, and the reduction of
c = 2 to two c = 1 problems when the components decouple.  Also the embedding of 2D weights in
the extruded 3D operator (the 2D cell as the x1-invariant 3D problem) against the oracle's 3D
UNO apply."""
import numpy as np
import pytest

from oracle import fem2d, uno, uno2d
from synth import random_field

SHAPE = (8, 6)


def _data(c, Ns, seed):
    f = np.stack([random_field((c,) + SHAPE, seed=seed + j) for j in range(Ns)])
    u = np.stack([random_field((c,) + SHAPE, seed=seed + 100 + j) for j in range(Ns)])
    return f, u


def _weights(c, M, seed):
    rng = np.random.default_rng(seed)
    n = len(uno2d.mode_list(M))
    return rng.normal(size=(1 + n, uno2d.n_entries(c))) * 0.7 + 0.5


def test_psi_c2_is_the_cholesky_like_product():
    rng = np.random.default_rng(0)
    for _ in range(20):
        B = rng.normal(size=(2, 2))
        A = B @ B.T + 0.1 * np.eye(2)
        L = np.linalg.cholesky(A)             # lower triangular, A = L L^T
        w = np.array([L[0, 0], L[1, 1], L[1, 0]])
        assert np.allclose(uno2d.psi(w, 2), A, rtol=0, atol=1e-14)
    assert np.allclose(uno2d.psi(np.array([1.0, 1.0, 0.0]), 2), np.eye(2))
    # any weights give a symmetric positive semi-definite block (signs of the diagonal free)
    W = rng.normal(size=(50, 3))
    ev = np.linalg.eigvalsh(uno2d.psi(W, 2))
    assert ev.min() >= -1e-14
    assert np.allclose(uno2d.psi(-W, 2), uno2d.psi(W, 2))


def test_mode_set_size_and_real_operator():
    for M in (1, 2, 3):
        ms = uno2d.mode_list(M)
        assert len(ms) == (2 * M + 1) * (M + 1) - 1 and len(set(ms)) == len(ms)
    # blocks on conjugate modes agree, so P r is real for real r (uno_apply asserts it)
    c, M = 2, 2
    Q = uno2d.modes_Q(_weights(c, M, 1), M, SHAPE, c)
    for k1 in range(SHAPE[0]):
        for k2 in range(SHAPE[1]):
            assert np.allclose(Q[k1, k2], Q[(-k1) % SHAPE[0], (-k2) % SHAPE[1]])
    fem2d.uno_apply(Q, random_field((c,) + SHAPE, seed=3), SHAPE, (False, False))


@pytest.mark.parametrize("c", [1, 2])
def test_loss_from_features_equals_loss_by_definition(c):
    M = 2
    f, u = _data(c, 5, 10)
    w = _weights(c, M, 2)
    Q = uno2d.modes_Q(w, M, SHAPE, c)
    a, b, delta = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    L_def = uno2d.loss_by_definition(Q, f, u)
    L_feat = uno2d.loss_from_features(uno2d.entries(Q), a, b, delta)
    assert abs(L_feat - L_def) <= 1e-12 * abs(L_def)


@pytest.mark.parametrize("c", [1, 2])
def test_gradient_matches_central_differences_of_the_real_space_loss(c):
    f, u = _data(c, 4, 20)
    rng = np.random.default_rng(4)
    v = rng.uniform(0.2, 1.5, size=SHAPE + (uno2d.n_entries(c),))
    # a real operator needs v(k) = v(-k)
    v = 0.5 * (v + v[(-np.arange(SHAPE[0])) % SHAPE[0]][:, (-np.arange(SHAPE[1])) % SHAPE[1]])
    a, b, delta = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    g = uno2d.grad_entries(v, a, b)
    h = 1e-6
    for (k1, k2) in [(1, 2), (3, 0), (0, 3), (4, 3)]:
        conj = ((-k1) % SHAPE[0], (-k2) % SHAPE[1])
        for e in range(uno2d.n_entries(c)):
            vp, vm = v.copy(), v.copy()
            for (x, y) in {(k1, k2), conj}:
                vp[x, y, e] += h
                vm[x, y, e] -= h
            fd = (uno2d.loss_by_definition(uno2d.blocks(vp, c), f, u) -
                  uno2d.loss_by_definition(uno2d.blocks(vm, c), f, u)) / (2 * h)
            an = g[k1, k2, e] + (g[conj][e] if conj != (k1, k2) else 0.0)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k1, k2, e, fd, an)


def test_hessian_c2_matches_differences_of_the_gradient():
    f, u = _data(2, 3, 30)
    a, b, _ = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    rng = np.random.default_rng(5)
    v = rng.normal(size=SHAPE + (3,))
    H = uno2d.hess_entries(a)
    assert np.allclose(H, np.swapaxes(H, -1, -2))
    h = 1e-5
    for e in range(3):
        dv = np.zeros(3)
        dv[e] = h
        fd = (uno2d.grad_entries(v + dv, a, b) - uno2d.grad_entries(v - dv, a, b)) / (2 * h)
        assert np.allclose(fd, H[..., :, e], rtol=1e-9, atol=1e-9)


def test_minimiser_recovers_a_generating_operator():
    """u = P_true f for SPD blocks Q_true: the stationary point of the loss at every mode (the
    3 x 3 system of the printed Hessian and gradient) returns Q_true's entries and zero loss."""
    c, M, Ns = 2, 2, 6
    Q_true = uno2d.modes_Q(_weights(c, M, 7), M, SHAPE, c)
    f = np.stack([random_field((c,) + SHAPE, seed=40 + j) for j in range(Ns)])
    u = np.stack([fem2d.uno_apply(Q_true, fj, SHAPE, (False, False)) for fj in f])
    a, b, delta = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    H = uno2d.hess_entries(a)
    v = np.linalg.solve(H, b[..., None])[..., 0]
    assert np.allclose(v, uno2d.entries(Q_true), rtol=1e-9, atol=1e-9)
    assert abs(uno2d.loss_from_features(v, a, b, delta)) <= 1e-9 * delta


def test_c2_reduces_to_two_c1_problems_without_coupling():
    f, u = _data(2, 4, 50)
    R, U = uno2d.spectra(f), uno2d.spectra(u)
    R[:, 1] = 0.0          # no y data: a2 = a3 = 0 and b2 = b3 = 0 except b3 from R_x U_y
    U[:, 1] = 0.0
    a, b, _ = uno2d.features(R, U)
    a1, b1, _ = uno2d.features(R[:, :1], U[:, :1])
    assert np.allclose(a[..., 0], a1[..., 0]) and np.allclose(b[..., 0], b1[..., 0])
    assert np.allclose(a[..., 1:], 0.0) and np.allclose(b[..., 1:], 0.0)


@pytest.mark.parametrize("c", [1, 2])
def test_extruded_3d_operator_equals_the_2d_operator(c):
    """The 2D cell as the x1-invariant 3D problem on `layers` voxels: the 3D blocks of the
    embedded 2D weights (training.modes2d_blocks3d) applied by the oracle's 3D UNO to an
    extruded field give the 2D operator on every layer, and no extrusion component."""
    from paper_2508_02681_gb300 import training
    M, layers = 2, 4
    w = _weights(c, M, 9)
    Q2 = uno2d.modes_Q(w, M, SHAPE, c)
    v3 = training.modes2d_blocks3d(w, M, SHAPE, layers, c)     # [layers, N1, N2/2+1, C3]
    shape3 = (layers,) + SHAPE
    c3 = 1 if c == 1 else 3
    Q3h = uno.blocks_from_entries(v3, c3)
    assert v3.shape == (layers, SHAPE[0], SHAPE[1] // 2 + 1, 1 if c == 1 else 6)
    assert np.linalg.eigvalsh(Q3h.reshape(-1, c3, c3)).min() > 0
    r2 = random_field((c,) + SHAPE, seed=61)
    r3 = np.zeros((c3,) + shape3)
    comps = [0] if c == 1 else [1, 2]
    for i, ci in enumerate(comps):
        r3[ci] = r2[i][None]
    s3 = uno.uno_apply(Q3h, r3)
    s2 = fem2d.uno_apply(Q2, r2, SHAPE, (False, False))
    for i, ci in enumerate(comps):
        for l in range(layers):
            assert np.allclose(s3[ci, l], s2[i], rtol=0, atol=1e-12 * np.max(np.abs(s2)))
    if c == 2:
        assert np.max(np.abs(s3[0])) <= 1e-12 * np.max(np.abs(s2))
