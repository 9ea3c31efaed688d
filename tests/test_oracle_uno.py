"""Pins of the oracle's transform and UNO preconditioner: DFT identities, A1-A3, Lemma 1,
FANS special cases and Table 3's FANS spectrum."""
import json
import os

import numpy as np
import pytest

from oracle import dft, fem, homogenize as hz, pcg, uno
from synth import random_field, random_phase, rsa_spheres


def test_dft_roundtrip_parseval_delta_and_numpy():
    x = random_field((2, 6, 5, 8), seed=1)
    X = dft.fftn_u(x)
    assert np.max(np.abs(dft.ifftn_u(X).real - x)) < 1e-14
    assert np.sum(np.abs(X) ** 2) == pytest.approx(np.sum(x ** 2), rel=1e-13)
    d = np.zeros((6, 5, 8))
    d[0, 0, 0] = 1.0
    assert np.max(np.abs(dft.fftn_u(d) - 1.0 / np.sqrt(240.0))) < 1e-15
    ref = np.fft.fftn(x, axes=(-3, -2, -1), norm="ortho")
    assert np.max(np.abs(X - ref)) < 1e-13
    Xh = dft.rfftn_u(x)
    assert np.max(np.abs(Xh - np.fft.rfftn(x, axes=(-3, -2, -1), norm="ortho"))) < 1e-13
    assert np.max(np.abs(dft.irfftn_u(Xh, 8) - x)) < 1e-14
    xo = random_field((3, 4, 7), seed=2)  # odd last axis
    assert np.max(np.abs(dft.irfftn_u(dft.rfftn_u(xo), 7) - xo)) < 1e-14


def test_half_multiplicity_counts_full_grid():
    for shape in [(4, 6, 8), (3, 5, 7)]:
        w = dft.half_multiplicity(shape)
        assert w.sum() == np.prod(shape)
        x = random_field(shape, seed=3)
        Xh = dft.rfftn_u(x)
        assert np.sum(w * np.abs(Xh) ** 2) == pytest.approx(np.sum(x ** 2), rel=1e-13)


def test_psi_is_cholesky_like():
    rng = np.random.default_rng(0)
    th = rng.standard_normal((10, 6))
    th[:, :2] = np.abs(th[:, :2]) + 0.1
    th[:, 3] = np.abs(th[:, 3]) + 0.1
    Q = uno.psi(th, 3)
    for i in range(10):
        L = np.linalg.cholesky(Q[i])
        assert L[0, 0] == pytest.approx(th[i, 0]) and L[1, 1] == pytest.approx(th[i, 1])
        assert L[2, 2] == pytest.approx(th[i, 3]) and L[1, 0] == pytest.approx(th[i, 2])
        assert L[2, 1] == pytest.approx(th[i, 4]) and L[2, 0] == pytest.approx(th[i, 5])
    t1 = rng.standard_normal((5, 1))
    assert np.allclose(uno.psi(t1, 1)[:, 0, 0], t1[:, 0] ** 2)
    v = uno.entries_from_blocks(Q)
    # paper layout [[v1, v3, v6], [v3, v2, v5], [v6, v5, v4]]
    assert np.allclose(Q[:, 0, 2], v[:, 5]) and np.allclose(Q[:, 1, 2], v[:, 4])
    assert np.allclose(Q[:, 2, 2], v[:, 3]) and np.allclose(Q[:, 0, 1], v[:, 2])
    assert np.allclose(uno.blocks_from_entries(v, 3), Q)


def _random_Q(shape, c, seed):
    rng = np.random.default_rng(seed)
    C = c * (c + 1) // 2
    th = rng.standard_normal((shape[0], shape[1], shape[2] // 2 + 1, C))
    return uno.symmetrize_half(uno.psi(th, c), shape[2])


@pytest.mark.parametrize("c", [1, 3])
def test_A1_A2_A3(c):
    shape = (4, 6, 8)
    Q = _random_Q(shape, c, 7)
    x = random_field((c,) + shape, seed=8)
    y = random_field((c,) + shape, seed=9)
    Px, Py = uno.uno_apply(Q, x), uno.uno_apply(Q, y)
    assert np.max(np.abs(uno.uno_apply(Q, 2.5 * x + y) - (2.5 * Px + Py))) < 1e-12
    assert np.sum(x * Py) == pytest.approx(np.sum(y * Px), rel=1e-12)
    assert np.sum(x * Px) > 0


@pytest.mark.parametrize("c,shape", [(1, (4, 4, 4)), (3, (3, 2, 4))])
def test_spectrum_lemma(c, shape):
    # eig(P) = union over the full grid of eig(Q(k)) (Lemma 1)
    Q = _random_Q(shape, c, 21)
    n = int(np.prod(shape))
    P = np.zeros((c * n, c * n))
    for j in range(c * n):
        e = np.zeros(c * n)
        e[j] = 1.0
        P[:, j] = uno.uno_apply(Q, e.reshape((c,) + shape)).ravel()
    evP = np.sort(np.linalg.eigvalsh(0.5 * (P + P.T)))
    assert np.max(np.abs(P - P.T)) < 1e-12
    w = dft.half_multiplicity(shape).astype(int)
    evQ = []
    flatQ = Q.reshape(-1, c, c)
    for i, m in enumerate(w.ravel()):
        evQ += list(np.linalg.eigvalsh(flatQ[i])) * m
    assert np.max(np.abs(evP - np.sort(evQ))) < 1e-11


@pytest.mark.parametrize("physics", [1, 3])
def test_fans_exact_on_homogeneous(physics):
    # reference medium = the material itself: P K is the zero-mean projector, so PCG converges
    # in one iteration for any right-hand side in range(K)
    shape = (4, 5, 6)
    props = [2.0] if physics == 1 else [[3.0, 0.25]]
    c = 1 if physics == 1 else 3
    K = fem.assemble_K(np.zeros(shape, np.uint8), props, physics)
    Q = uno.reference_medium_Q(physics, props, shape)
    x = random_field((c,) + shape, seed=4)
    y = uno.uno_apply(Q, fem.to_soa(K @ fem.from_soa(x), c, shape))
    xm = x - x.mean(axis=(1, 2, 3), keepdims=True)
    assert np.max(np.abs(y - xm)) < 1e-12
    f = K @ fem.from_soa(random_field((c,) + shape, seed=5))
    P = hz.preconditioner("uno", K, physics, props, shape, Q)
    _, it, _ = pcg.pcg(lambda v: K @ v, f, P, 1e-10, 50)
    assert it == 1


def test_reference_symbol_even_on_self_conjugate_planes():
    shape = (6, 4, 8)
    Q = uno.reference_medium_Q(3, [[1.0, 0.3], [10.0, 0.2]], shape)
    assert np.max(np.abs(uno.symmetrize_half(Q, 8) - Q)) < 1e-15


def test_fans_spectrum_table3():
    # Two-phase FANS with kappa_ref = arithmetic mean: the nonzero spectrum of P K lies in
    # [kappa_min/kappa_ref, kappa_max/kappa_ref]; both ends are attained when some node has all
    # eight elements in one phase.  Table 3 prints these ends for kappa = (1, 0.2).
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table3_spectra.json")))
    kap = gold["kappa"]
    shape = (6, 6, 6)
    phase = np.zeros(shape, np.uint8)
    phase[:3, :3, :3] = 1
    phase[4, 4, 4] = 1
    K = fem.assemble_K(phase, kap, 1).toarray()
    Q = uno.reference_medium_Q(1, kap, shape)
    n = K.shape[0]
    P = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        P[:, j] = uno.uno_apply(Q, e.reshape((1,) + shape)).ravel()
    ev = np.sort(np.linalg.eigvals(P @ K).real)
    ev = ev[np.abs(ev) > 1e-9]
    assert ev.min() == pytest.approx(gold["FANS"]["lambda_min"], abs=0.5e-4)
    assert ev.max() == pytest.approx(gold["FANS"]["lambda_max"], abs=0.5e-4)
    assert ev.max() / ev.min() == pytest.approx(gold["FANS"]["cond"], abs=0.5e-3)


def test_spd_check():
    shape = (4, 4, 4)
    Q = uno.reference_medium_Q(1, [1.0, 10.0], shape)
    assert uno.spd_check(Q, 1e-12)
    Q2 = Q.copy()
    Q2[1, 2, 1] = -1e-3
    assert not uno.spd_check(Q2, 1e-12)


# ---------------------------------------------------------------- bypass + limited mode set
def _w_modes(M, c, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((1 + len(uno.mode_list(M)), uno.n_unique(c))) * 0.5 + 0.8


def test_mode_list_is_the_periodic_row_of_the_mode_table():
    # (2M+1)^(d-1) (M+1) - 1 modes, k3 >= 0, no k = 0, all distinct
    for M in range(0, 4):
        m = uno.mode_list(M)
        assert len(m) == (2 * M + 1) ** 2 * (M + 1) - 1 == len(set(m))
        assert all(k[2] >= 0 and max(abs(x) for x in k) <= M for k in m) and (0, 0, 0) not in m


@pytest.mark.parametrize("c", [1, 3])
def test_modes_M0_is_the_bypass_alone(c):
    # M = 0: no kernel modes, P r = W r node by node with W = psi(w_0)
    shape = (4, 6, 8)
    w = _w_modes(0, c, 1)
    Q = uno.modes_Q(w, 0, shape, c)
    r = random_field((c,) + shape, seed=2)
    W = uno.psi(w[0], c)
    assert np.max(np.abs(uno.uno_apply(Q, r) - np.einsum("ij,jxyz->ixyz", W, r))) < 1e-13


def test_modes_single_fourier_mode_closed_form():
    # a real Fourier mode cos(2 pi k.x / N) is an eigenfunction: P multiplies it by
    # W + K(k) (k3 > 0), by W + (K(k) + K(-k)) / 2 on the k3 = 0 plane, by W outside K_M
    shape = (8, 8, 8)
    M = 2
    w = _w_modes(M, 1, 3)
    Q = uno.modes_Q(w, M, shape, 1)
    idx = {k: i for i, k in enumerate(uno.mode_list(M))}
    x = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    W = w[0, 0] ** 2
    cases = [((1, -2, 1), W + w[1 + idx[(1, -2, 1)], 0] ** 2),
             ((2, 1, 0), W + 0.5 * (w[1 + idx[(2, 1, 0)], 0] ** 2 + w[1 + idx[(-2, -1, 0)], 0] ** 2)),
             ((3, 0, 1), W), ((0, 0, 3), W)]
    for k, lam in cases:
        ph = 2 * np.pi * sum(k[a] * x[a] / shape[a] for a in range(3))
        r = np.cos(ph)[None]
        assert np.max(np.abs(uno.uno_apply(Q, r) - lam * r)) < 1e-12


@pytest.mark.parametrize("c", [1, 3])
def test_modes_spectrum_bounded_below_by_the_bypass(c):
    shape = (6, 6, 6)
    w = _w_modes(2, c, 4)
    Q = uno.modes_Q(w, 2, shape, c)
    lw = np.linalg.eigvalsh(uno.psi(w[0], c)).min()
    assert uno.min_eigenvalue(Q, skip_zero_mode=False) >= lw - 1e-12
