"""Algorithm 4 on the device (unocg_newton_*, k_newton.cu) against its host restatement
(tests/newton_host.py) and the oracle: c = 1 (3D features of Eq. (features-c-1)), c = 2 (2D
features of Eq. (features-c-2)) and c = 3 (App. C) from seeded data; the device weights and loss
history equal the host ones to 1e-10, and for c = 1 the device reaches the oracle's global
optimum of the bypass-plus-modes loss."""
import numpy as np
import pytest

from oracle import training as ot, uno, uno2d
from synth import random_field
from tests import newton_host as nh
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _close(w_dev, h_dev, w_host, h_host):
    assert len(h_dev) == len(h_host), (len(h_dev), len(h_host))
    assert rel(np.asarray(h_dev), np.asarray(h_host)) < 1e-10
    assert rel(w_dev, w_host) < 1e-8


@pytest.mark.parametrize("shape,M,seed", [((8, 8, 8), 2, 0), ((12, 12, 16), 4, 2)])
def test_device_newton_c1_equals_host_and_reaches_the_optimum(shape, M, seed):
    from paper_2508_02681_gb300 import training as tr
    rng = np.random.default_rng(seed)
    f = np.stack([random_field((1,) + shape, seed=100 * seed + b) for b in range(5)])
    f -= f.mean(axis=(2, 3, 4), keepdims=True)
    u = np.stack([random_field((1,) + shape, seed=100 * seed + 50 + b) for b in range(5)])
    a, b = ot.features_c1(ot.spectra(f), ot.spectra(u), shape)
    w_opt = ot.optimum_modes_c1(a, b, M, shape)
    w0 = 0.5 + rng.random(w_opt.shape)
    w, hist = tr.second_order_modes(a, b, M, w0)
    wh, hh = nh.second_order_modes(a, b, M, w0)
    _close(w, hist, wh, hh)
    l_opt = ot.modes_loss_c1(w_opt, M, shape, a, b)
    assert ot.modes_loss_c1(w, M, shape, a, b) == pytest.approx(l_opt, rel=1e-9, abs=1e-12)


def test_device_newton_c3_equals_host_and_recovers_the_operator():
    from paper_2508_02681_gb300 import training as tr
    shape, M, B = (6, 6, 6), 1, 4
    rng = np.random.default_rng(11)
    n_modes = len(uno.mode_list(M))
    ws = rng.standard_normal((1 + n_modes, 6)) * 0.2
    ws[:, [0, 1, 3]] += 1.0
    Qs = uno.modes_Q(ws, M, shape, 3)
    f = np.stack([random_field((3,) + shape, seed=40 + b) for b in range(B)])
    u = np.stack([uno.uno_apply(Qs, f[b]) for b in range(B)])
    a, b = ot.features_general(ot.spectra(f), ot.spectra(u), shape)
    w0 = ws + rng.standard_normal(ws.shape) * 0.05
    w, hist = tr.second_order_modes_c3(a, b, M, w0)
    wh, hh = nh.second_order_modes_c3(a, b, M, w0)
    _close(w, hist, wh, hh)
    assert np.max(np.abs(uno.modes_Q(w, M, shape, 3) - Qs)) < 1e-5 * np.max(np.abs(Qs))


@pytest.mark.parametrize("c", [1, 2])
def test_device_newton_2d_equals_host(c):
    from paper_2508_02681_gb300 import training as tr
    shape, M, Ns = (12, 10), 2, 6
    rng = np.random.default_rng(30 + c)
    f = np.stack([random_field((c,) + shape, seed=60 + j) for j in range(Ns)])
    u = np.stack([random_field((c,) + shape, seed=80 + j) for j in range(Ns)])
    a, b, _ = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    N2 = shape[1]

    def half(x):
        h = x[:, : N2 // 2 + 1].copy()
        h[:, 1: (N2 + 1) // 2] *= 2.0
        return h

    C = uno2d.n_entries(c)
    n = len(uno2d.mode_list(M))
    w0 = np.abs(rng.normal(size=(1 + n, C))) + 0.5
    w, hist = tr.second_order_modes_2d(half(a), half(b), M, w0, c)
    wh, hh = nh.second_order_modes_2d(half(a), half(b), M, w0, c)
    _close(w, hist, wh, hh)
    assert hist[-1] < hist[0]
