"""Pins of the 2D oracle (bilinear quadrilaterals, Sec. 4.1 / 6.1 / 6.2 in two dimensions):
Table 3's spectra, homogeneous cells, the energy ordering of the boundary conditions, and the
x3-invariant 3D problem on an extruded grid (the reading the GPU path uses for 2D cells)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, fem2d as f2, mixedbc as mb
from synth import random_phase

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table3_spectra.json")))


def _phase2d(shape, seed, frac=0.35):
    rng = np.random.default_rng(seed)
    # blobs: a smoothed random field thresholded at the given fraction
    x = rng.standard_normal(shape)
    for _ in range(3):
        x = (x + np.roll(x, 1, 0) + np.roll(x, -1, 0) + np.roll(x, 1, 1) + np.roll(x, -1, 1)) / 5.0
    return (x > np.quantile(x, 1 - frac)).astype(np.uint8)


def test_table3_cg_and_jacobi_extremes():
    # homogeneous kappa = 1 on a periodic 2D grid: lambda_max(K) = 4 (Table 3, CG 3.9998 on the
    # two-phase 400^2 sample), lambda_max(D^-1 K) = 4 / (8/3) = 1.5 (Jac-CG 1.5000)
    shape = (8, 8)
    K = f2.assemble_K(np.zeros(shape, np.uint8), [1.0], 1, (False, False)).toarray()
    ev = np.linalg.eigvalsh(K)
    assert ev.max() == pytest.approx(4.0, abs=1e-12)
    assert abs(ev.max() - GOLD["CG"]["lambda_max"]) < 0.5e-3
    evj = np.linalg.eigvals(K / np.diag(K)[:, None]).real
    assert evj.max() == pytest.approx(GOLD["JacCG"]["lambda_max"], abs=0.5e-4)


def test_table3_fans_spectrum_bounds():
    # FANS with the arithmetic-mean reference medium: the spectrum of P K lies in
    # [kappa_min, kappa_max] / kappa_ref = [0.3333, 1.6667], condition number <= 5 (Table 3)
    shape = (16, 16)
    phase = _phase2d(shape, seed=4)
    kap = GOLD["kappa"]
    K = f2.assemble_K(phase, kap, 1, (False, False)).toarray()
    Q = f2.reference_Q(1, kap, shape, (False, False))
    n = K.shape[0]
    P = np.stack([f2.uno_apply(Q, np.eye(n)[i].reshape(1, *shape), shape, (False, False)).ravel() for i in range(n)])
    ev = np.sort(np.linalg.eigvals(P @ K).real)[1:]   # drop the constant null mode
    assert ev.min() >= GOLD["FANS"]["lambda_min"] - 1e-4
    assert ev.max() <= GOLD["FANS"]["lambda_max"] + 1e-4
    assert ev.max() / ev.min() <= GOLD["FANS"]["cond"] + 1e-3


@pytest.mark.parametrize("bc", [(False, False), (True, True), (False, True)])
@pytest.mark.parametrize("physics,props", [(1, [2.5]), (3, [[4.0, 0.3]])])
def test_homogeneous_cell(bc, physics, props):
    shape = (6, 8)
    phase = np.zeros(shape, np.uint8)
    dim = 2 if physics == 1 else 3
    loads = np.eye(dim)
    assert np.max(np.abs(f2.assemble_f(phase, props, physics, bc, loads[0]))) < 1e-14
    out = f2.solve(phase, props, physics, bc, loads, tol=1e-10)
    C = f2.effective_tensor(phase, props, physics, bc, out["u"], loads)
    assert np.max(np.abs(C - f2.material_matrix(physics, props[0]))) < 1e-13


@pytest.mark.parametrize("physics,props,load", [(1, [1.0, 10.0], [0.4, -1.0]),
                                                (3, [[1.0, 0.3], [10.0, 0.2]], [0.2, -0.5, 0.7])])
def test_energy_ordering_and_direct_solve(physics, props, load):
    shape = (10, 12)
    phase = _phase2d(shape, seed=7)
    W = {}
    for name, bc in (("per", (False, False)), ("mix", (False, True)), ("dir", (True, True))):
        out = f2.solve(phase, props, physics, bc, [load], tol=1e-12)
        ud = spla.spsolve(out["K"].tocsc(), f2.assemble_f(phase, props, physics, bc, load))
        if name == "per":
            c = f2.n_comp(physics)
            v = ud.reshape(-1, c)
            ud = (v - v.mean(axis=0)).ravel()
        assert np.max(np.abs(out["u"][0] - ud)) < 1e-9 * np.max(np.abs(ud))
        W[name] = float(f2.effective_tensor(phase, props, physics, bc, out["u"], [load])[:, 0] @ np.asarray(load))
    assert W["per"] < W["mix"] < W["dir"]


@pytest.mark.parametrize("bc2", [(False, False), (False, True), (True, True)])
@pytest.mark.parametrize("physics", [1, 3])
def test_extruded_3d_problem_equals_2d(bc2, physics):
    """A 2D cell extruded along x3 (periodic, any number of layers) has the x3-invariant 3D
    solution: u_3D(x1, x2, x3) = u_2D(x1, x2) (plane strain, u3 = 0 for in-plane loads) and the
    in-plane block of the 3D averages equals the 2D averages."""
    shape2 = (6, 8)
    phase2 = _phase2d(shape2, seed=9)
    props = [1.0, 7.0] if physics == 1 else [[1.0, 0.3], [7.0, 0.2]]
    load2 = np.array([0.3, -1.0]) if physics == 1 else np.array([0.2, -0.4, 0.6])
    load3 = np.array([0.3, -1.0, 0.0]) if physics == 1 else np.array([0.2, -0.4, 0.0, 0.6, 0.0, 0.0])
    r2 = f2.solve(phase2, props, physics, bc2, [load2], tol=1e-12)
    N3 = 2
    phase3 = np.repeat(phase2[:, :, None], N3, axis=2)
    bc3 = (bc2[0], bc2[1], False)
    r3 = mb.solve(phase3, props, 1 if physics == 1 else 3, bc3, [load3], tol=1e-12)
    c3 = 1 if physics == 1 else 3
    Ms = mb.free_shape(phase3.shape, bc3)
    u3 = r3["u"][0].reshape(Ms + (c3,))
    u2 = r2["u"][0].reshape(f2.free_shape(shape2, bc2) + (f2.n_comp(physics),))
    for z in range(N3):
        assert np.max(np.abs(u3[:, :, z, :f2.n_comp(physics)] - u2)) < 1e-9 * np.max(np.abs(u2))
    if physics == 3:
        assert np.max(np.abs(u3[..., 2])) < 1e-12
    C3 = mb.effective_tensor(phase3, props, c3, bc3, r3["u"], [load3])[:, 0]
    C2 = f2.effective_tensor(phase2, props, physics, bc2, r2["u"], [load2])[:, 0]
    sel = [0, 1] if physics == 1 else [0, 1, 3]
    assert np.max(np.abs(C3[sel] - C2)) < 1e-10 * np.max(np.abs(C2))
    assert r3["iters"][0] == r2["iters"][0]
