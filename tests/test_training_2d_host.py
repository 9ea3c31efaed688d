"""The 2D learned-UNO training restated on the host (tests/newton_host.py, the reference for the
device Newton of the library) against the 2D oracle, without a GPU: Algorithm 4 on the 2D mode
set recovers a generating bypass-plus-modes operator from features that the oracle computes on
the full grid (folded onto the half grid with the multiplicity of the conjugate modes), and its
loss history is the oracle's loss of the iterates."""
import numpy as np
import pytest

from oracle import fem2d, uno2d
from synth import random_field

SHAPE = (12, 10)


def _half(x):
    """Full-grid features [N1, N2, C] -> half grid [N1, N2/2+1, C] with multiplicities."""
    N2 = SHAPE[1]
    h = x[:, : N2 // 2 + 1].copy()
    h[:, 1: (N2 + 1) // 2] *= 2.0
    return h


@pytest.mark.parametrize("c", [1, 2])
def test_newton_2d_recovers_a_generating_operator(c):
    from tests import newton_host as training
    M, Ns = 2, 8
    rng = np.random.default_rng(3 + c)
    C = uno2d.n_entries(c)
    n = len(uno2d.mode_list(M))
    w_true = np.abs(rng.normal(size=(1 + n, C))) * 0.5 + 0.5
    if c == 2:
        w_true[:, 2] = rng.normal(size=1 + n) * 0.3
    # symmetric data on the line k2 = 0: (k1, 0) and (-k1, 0) carry the same weights
    for i, (k1, k2) in enumerate(uno2d.mode_list(M)):
        if k2 == 0 and k1 < 0:
            w_true[1 + i] = w_true[1 + uno2d.mode_list(M).index((-k1, 0))]
    Q = uno2d.modes_Q(w_true, M, SHAPE, c)
    f = np.stack([random_field((c,) + SHAPE, seed=10 + j) for j in range(Ns)])
    u = np.stack([fem2d.uno_apply(Q, fj, SHAPE, (False, False)) for fj in f])
    a, b, delta = uno2d.features(uno2d.spectra(f), uno2d.spectra(u))
    w0 = w_true * (1.0 + 0.2 * rng.normal(size=w_true.shape))
    for i, (k1, k2) in enumerate(uno2d.mode_list(M)):
        if k2 == 0 and k1 < 0:
            w0[1 + i] = w0[1 + uno2d.mode_list(M).index((-k1, 0))]
    w, hist = training.second_order_modes_2d(_half(a), _half(b), M, w0, c)
    # the loss history is the oracle's loss (without delta) of the iterates
    assert abs(hist[0] + delta - uno2d.modes_loss(w0, M, SHAPE, c, a, b, 0.0) - delta) <= 1e-9 * delta
    assert abs(hist[-1] + delta - uno2d.modes_loss(w, M, SHAPE, c, a, b, delta)) <= 1e-9 * delta
    assert hist[-1] + delta <= 1e-12 * delta
    assert np.allclose(uno2d.modes_Q(w, M, SHAPE, c), Q, rtol=0, atol=1e-6 * np.max(np.abs(Q)))
