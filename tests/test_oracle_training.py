"""Pins of the oracle's training loss and gradients (Eq. fnocg-loss, Sec. 5.4)."""
import numpy as np
import pytest

from oracle import dft, training, uno
from synth import random_field


def _data(c, shape, B, seed):
    f = np.stack([random_field((c,) + shape, seed=seed + b) for b in range(B)])
    u = np.stack([random_field((c,) + shape, seed=seed + 100 + b) for b in range(B)])
    return f, u


@pytest.mark.parametrize("c", [1, 3])
def test_loss_spectral_equals_definition(c):
    shape = (4, 3, 6)
    f, u = _data(c, shape, 3, 1)
    rng = np.random.default_rng(2)
    th = rng.standard_normal((4, 3, 4, c * (c + 1) // 2))
    Q = uno.symmetrize_half(uno.psi(th, c), 6)
    R, U = training.spectra(f), training.spectra(u)
    assert training.loss_from_spectra(Q, R, U, shape) == pytest.approx(
        training.loss_by_definition(Q, f, u), rel=1e-12)


def test_c1_closed_form_gradient_matches_fd():
    shape = (4, 4, 6)
    f, u = _data(1, shape, 2, 3)
    rng = np.random.default_rng(4)
    v = np.abs(rng.standard_normal((4, 4, 4))) + 0.1
    v = uno.symmetrize_half(v[..., None, None], 6)[..., 0, 0]
    R, U = training.spectra(f), training.spectra(u)
    g = training.grad_v_c1(v, R, U, shape)
    # independent check: central differences of the loss by definition, perturbing one
    # half-grid entry (and its mirror on the self-conjugate planes)
    for idx in [(1, 2, 1), (0, 1, 0), (2, 3, 3), (3, 0, 2)]:
        eps = 1e-6
        vp, vm = v.copy(), v.copy()
        mirror = ((-idx[0]) % 4, (-idx[1]) % 4, idx[2])
        for vv, s in ((vp, eps), (vm, -eps)):
            vv[idx] += s
            if idx[2] in (0, 3) and mirror != idx:
                vv[mirror] += s
        lp = training.loss_by_definition(vp[..., None, None], f, u)
        lm = training.loss_by_definition(vm[..., None, None], f, u)
        fd = (lp - lm) / (2 * eps)
        an = g[idx] + (g[mirror] if idx[2] in (0, 3) and mirror != idx else 0.0)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_c3_gradient_and_theta_chain_match_fd():
    shape = (3, 2, 4)
    f, u = _data(3, shape, 2, 5)
    rng = np.random.default_rng(6)
    th = rng.standard_normal((3, 2, 3, 6))
    R, U = training.spectra(f), training.spectra(u)
    Q = uno.psi(th, 3)
    ge = training.grad_entries_general(Q, R, U, shape)
    gt = training.grad_theta(th, ge, 3)

    def L(theta):
        return training.loss_from_spectra(uno.psi(theta, 3), R, U, shape)

    for idx in [(0, 1, 1, 0), (2, 0, 2, 4), (1, 1, 1, 5), (0, 0, 1, 2)]:
        eps = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[idx] += eps
        tm[idx] -= eps
        fd = (L(tp) - L(tm)) / (2 * eps)
        assert gt[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("c,shape,M", [(1, (6, 6, 6), 2), (3, (4, 6, 6), 1)])
def test_grad_modes_matches_central_differences(c, shape, M):
    """Bypass-plus-modes weights: the chained gradient against central differences of the loss
    evaluated by definition (real-space application of P)."""
    rng = np.random.default_rng(11)
    w = rng.standard_normal((1 + len(uno.mode_list(M)), uno.n_unique(c))) * 0.4 + 0.7
    B = 2
    f = rng.standard_normal((B, c) + shape)
    u = rng.standard_normal((B, c) + shape)

    def loss(wv):
        return training.loss_by_definition(uno.modes_Q(wv, M, shape, c), f, u)

    Q = uno.modes_Q(w, M, shape, c)
    R, U = training.spectra(f), training.spectra(u)
    g = training.grad_modes(w, M, shape, c, training.grad_entries_general(Q, R, U, shape))
    for (i, m) in [(0, 0), (1, 0), (len(w) - 1, 0), (len(w) // 2, uno.n_unique(c) - 1), (3, c - 1)]:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i, m] += h
        wm[i, m] -= h
        fd = (loss(wp) - loss(wm)) / (2 * h)
        assert g[i, m] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_optimum_modes_c1_is_the_global_minimizer():
    """The bypass-plus-modes optimum from the features: the loss from the features equals the
    loss by definition up to its constant, the gradient vanishes wherever the weight is free,
    and no perturbation lowers the loss."""
    shape = (6, 6, 8)
    M = 1
    rng = np.random.default_rng(12)
    f, u = _data(1, shape, 6, 40)
    f -= f.mean(axis=(2, 3, 4), keepdims=True)  # zero-mean data: the k = 0 features vanish
    R, U = training.spectra(f), training.spectra(u)
    a, b = training.features_c1(R, U, shape)
    w = training.optimum_modes_c1(a, b, M, shape)
    delta = np.mean(np.sum(u ** 2, axis=(1, 2, 3, 4)))
    # features reproduce the loss of Eq. (fnocg-loss)
    lf = training.modes_loss_c1(w, M, shape, a, b) + delta
    ld = training.loss_by_definition(uno.modes_Q(w, M, shape, 1), f, u)
    assert lf == pytest.approx(ld, rel=1e-10)
    # stationary in every weight (a weight at zero sits on the boundary psi = 0 with psi' = 0)
    Q = uno.modes_Q(w, M, shape, 1)
    g = training.grad_modes(w, M, shape, 1, training.grad_entries_general(Q, R, U, shape))
    assert np.max(np.abs(g)) < 1e-7 * max(1.0, float(np.max(np.abs(b))))
    # no perturbation lowers the loss
    l0 = training.modes_loss_c1(w, M, shape, a, b)
    for _ in range(50):
        wp = w + 1e-3 * rng.standard_normal(w.shape)
        assert training.modes_loss_c1(wp, M, shape, a, b) >= l0 - 1e-12 * abs(l0)


@pytest.mark.parametrize("c,shape", [(1, (6, 8, 4)), (3, (4, 6, 6))])
def test_general_features_give_the_loss_and_gradient(c, shape):
    # Sec. 5.4 / App. C: the loss is a quadratic in the block entries whose coefficients are the
    # features; its value equals the loss by definition up to delta = mean ||u||^2, and its
    # gradient equals the pinned per-entry gradient of the definition
    rng = np.random.default_rng(c)
    B = 3
    f = rng.standard_normal((B, c) + shape)
    u = rng.standard_normal((B, c) + shape)
    R, U = training.spectra(f), training.spectra(u)
    a, b = training.features_general(R, U, shape)
    C = 1 if c == 1 else 6
    th = rng.standard_normal(shape[:2] + (shape[2] // 2 + 1, C)) * 0.4
    th[..., 0] += 1.0
    if c == 3:
        th[..., 1] += 1.0
        th[..., 3] += 1.0
    Q = uno.psi(th, c)
    v = uno.entries_from_blocks(Q)
    delta = float(np.sum(u ** 2)) / B
    assert training.loss_from_features(v, a, b) + delta == pytest.approx(training.loss_from_spectra(Q, R, U, shape), rel=1e-12)
    g = training.grad_entries_general(Q, R, U, shape)
    rng2 = np.random.default_rng(5)
    for _ in range(6):
        idx = tuple(rng2.integers(0, s) for s in v.shape)
        hs = 1e-6
        vp, vm = v.copy(), v.copy()
        vp[idx] += hs
        vm[idx] -= hs
        fd = (training.loss_from_features(vp, a, b) - training.loss_from_features(vm, a, b)) / (2 * hs)
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-9)
    if c == 1:
        a1, b1 = training.features_c1(R, U, shape)
        assert np.max(np.abs(a[..., 0] - a1)) < 1e-14 and np.max(np.abs(b[..., 0] - b1)) < 1e-14
