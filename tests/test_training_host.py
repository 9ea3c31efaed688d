"""Second-order training (Algorithm 4) restated on the host (tests/newton_host.py, the reference
for the device Newton of the library): the Newton-Raphson iteration on the bypass-plus-modes
weights reaches the oracle's global optimum from the features (c = 1) and recovers a generating
operator (c = 3); host parametrization and mode order against the oracle."""
import numpy as np
import pytest

from oracle import training as ot
from paper_2508_02681_gb300 import training as pt
from synth import random_field
from tests import newton_host as nh


@pytest.mark.parametrize("shape,M,seed", [((8, 8, 8), 2, 0), ((6, 10, 8), 1, 1), ((12, 12, 16), 4, 2)])
def test_newton_reaches_the_global_optimum(shape, M, seed):
    rng = np.random.default_rng(seed)
    f = np.stack([random_field((1,) + shape, seed=100 * seed + b) for b in range(5)])
    f -= f.mean(axis=(2, 3, 4), keepdims=True)
    u = np.stack([random_field((1,) + shape, seed=100 * seed + 50 + b) for b in range(5)])
    R, U = ot.spectra(f), ot.spectra(u)
    a, b = ot.features_c1(R, U, shape)
    w_opt = ot.optimum_modes_c1(a, b, M, shape)
    w0 = 0.5 + rng.random(w_opt.shape)
    w, hist = nh.second_order_modes(a, b, M, w0)
    l_opt = ot.modes_loss_c1(w_opt, M, shape, a, b)
    assert ot.modes_loss_c1(w, M, shape, a, b) == pytest.approx(l_opt, rel=1e-9, abs=1e-12)
    assert all(h1 <= h0 + 1e-12 * abs(h0) for h0, h1 in zip(hist, hist[1:]))  # monotone
    assert len(hist) < 60


@pytest.mark.parametrize("c", [1, 3])
def test_host_psi_and_its_inverse(c):
    # the host parametrization agrees with the oracle's psi (Sec. 5.2.2), and psi_inverse
    # recovers weights whose psi is a given SPD block
    from oracle import uno
    rng = np.random.default_rng(c)
    C = c * (c + 1) // 2
    w = rng.standard_normal((7, C))
    assert np.max(np.abs(pt.psi(w, c) - uno.psi(w, c))) < 1e-15
    A = rng.standard_normal((7, c, c))
    Q = A @ np.swapaxes(A, -1, -2) + 0.1 * np.eye(c)
    w2 = pt.psi_inverse(Q)
    assert np.max(np.abs(uno.psi(w2, c) - Q)) < 1e-12 * np.max(np.abs(Q))
    if c == 3:  # the Cholesky factor has a non-negative diagonal (w1, w2, w4)
        assert np.all(w2[:, [0, 1, 3]] > 0)


def test_mode_set_order_matches_oracle():
    from oracle import uno
    for M in (1, 2, 5):
        assert pt.mode_set(M) == [tuple(k) for k in uno.mode_list(M)]


def test_newton_c3_recovers_a_generating_preconditioner():
    """Algorithm 4 for c = 3: data u = P* f from a bypass-plus-modes preconditioner P* (the
    oracle applies it); the loss from the features reaches -delta (zero residual), and the
    expanded Q equals Q* on the half grid."""
    from oracle import training as ot, uno
    shape, M, B = (6, 6, 6), 1, 4
    rng = np.random.default_rng(11)
    n_modes = len(uno.mode_list(M))
    ws = rng.standard_normal((1 + n_modes, 6)) * 0.2
    ws[:, [0, 1, 3]] += 1.0
    Qs = uno.modes_Q(ws, M, shape, 3)
    f = np.stack([random_field((3,) + shape, seed=40 + b) for b in range(B)])
    u = np.stack([uno.uno_apply(Qs, f[b]) for b in range(B)])
    R, U = ot.spectra(f), ot.spectra(u)
    a, b = ot.features_general(R, U, shape)
    delta = float(np.sum(u ** 2)) / B
    w0 = ws + rng.standard_normal(ws.shape) * 0.05
    w, hist = nh.second_order_modes_c3(a, b, M, w0)
    assert all(h1 <= h0 + 1e-12 * abs(h0) for h0, h1 in zip(hist, hist[1:]))
    assert hist[-1] + delta < 1e-9 * delta
    Q = uno.modes_Q(w, M, shape, 3)
    assert np.max(np.abs(Q - Qs)) < 1e-5 * np.max(np.abs(Qs))
    # the features-based loss of the result equals the oracle's loss from features
    v = uno.entries_from_blocks(Q)
    assert ot.loss_from_features(v, a, b) == pytest.approx(hist[-1], rel=1e-8, abs=1e-10 * delta)


def test_autotune_cache_round_trip(tmp_path):
    """The autotune cache stores the measured setting per key and applies it without measuring
    on the next call (host logic; the measurement itself runs on the GPU)."""
    from paper_2508_02681_gb300.solver import _tuning_cache
    path = str(tmp_path / "tune.json")
    applied, measured = [], []

    def measure():
        measured.append(1)
        return [2, 1], np.array([[3.0, np.nan], [2.0, 2.5], [1.0, np.nan]])

    s1, t1 = _tuning_cache(path, "k1", measure, applied.append)
    s2, t2 = _tuning_cache(path, "k1", measure, applied.append)
    s3, _ = _tuning_cache(path, "k2", measure, applied.append)
    assert s1 == s2 == s3 == [2, 1] and t1 is not None and t2 is None
    assert len(measured) == 2 and applied == [[2, 1]] * 3
    import json
    assert set(json.load(open(path))) == {"k1", "k2"}


def test_checkpoint_round_trip(tmp_path):
    """Checkpoint / resume of the training state: weights, Adam moments and metadata."""
    import torch
    th = torch.tensor(np.arange(6.0).reshape(3, 2), dtype=torch.float32, requires_grad=True)
    opt = torch.optim.Adam([th], lr=0.1)
    for _ in range(3):
        opt.zero_grad()
        (th ** 2).sum().backward()
        opt.step()
    path = str(tmp_path / "ck.pt")
    pt.save_checkpoint(path, th, opt, epoch=3, losses=[3.0, 2.0, 1.0])
    th2, state, meta = pt.load_checkpoint(path, device="cpu")
    assert torch.equal(th2.detach(), th.detach()) and th2.requires_grad
    assert meta["epoch"] == 3 and meta["losses"] == [3.0, 2.0, 1.0]
    opt2 = torch.optim.Adam([th2], lr=0.1)
    opt2.load_state_dict(state)
    for o in (opt, opt2):
        o.zero_grad()
    (th ** 2).sum().backward()
    (th2 ** 2).sum().backward()
    opt.step()
    opt2.step()
    assert torch.allclose(th.detach(), th2.detach())
