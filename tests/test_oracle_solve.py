"""Pins of the oracle's PCG and homogenization layer: dense direct solves, exact laminate
results, Voigt/Reuss bounds, symmetry, invariances, the CG error bound and sensitivities."""
import numpy as np
import pytest

from oracle import fem, homogenize as hz, pcg, uno
from synth import laminate, random_phase, rsa_spheres, unit_loads

TH = [1.0, 10.0]
EL = [[1.0, 0.3], [10.0, 0.2]]


@pytest.mark.parametrize("physics,props", [(1, TH), (3, EL)])
def test_pcg_matches_dense_direct(physics, props):
    shape = (4, 4, 4)
    phase = random_phase(shape, 2, seed=31)
    c = 1 if physics == 1 else 3
    loads = unit_loads(physics)[:2]
    for pc in ("none", "jacobi", "uno"):
        res = hz.solve(phase, props, physics, loads, precond=pc, tol=1e-13, max_iter=2000)
        for u, f, it in zip(res["u"], res["f"], res["iters"]):
            ud = hz.direct_solve(res["K"], f, c)
            assert np.max(np.abs(u - ud)) < 1e-10 * max(1.0, np.max(np.abs(ud)))
            assert it <= c * phase.size


def test_flexible_equals_standard_with_fixed_preconditioner():
    phase, _ = rsa_spheres((8, 8, 8), 2.0, 0.3, seed=4)
    a = hz.solve(phase, TH, 1, unit_loads(1)[:1], "uno", tol=1e-12)
    b = hz.solve(phase, TH, 1, unit_loads(1)[:1], "uno", tol=1e-12, flexible=True)
    assert abs(a["iters"][0] - b["iters"][0]) <= 1
    assert np.max(np.abs(a["u"][0] - b["u"][0])) < 1e-10


def test_homogeneous_returns_its_own_tensor():
    shape = (4, 5, 6)
    ph = np.zeros(shape, np.uint8)
    # f is zero up to rounding here, so the relative stopping test cannot fire: cap the loop
    r1 = hz.solve(ph, [2.5], 1, unit_loads(1), "uno", tol=1e-10, max_iter=20)
    C1 = hz.effective_tensor(ph, [2.5], 1, r1["u"], unit_loads(1))
    assert np.max(np.abs(C1 - 2.5 * np.eye(3))) < 1e-14
    r3 = hz.solve(ph, [[3.0, 0.2]], 3, unit_loads(3), "uno", tol=1e-10, max_iter=20)
    C3 = hz.effective_tensor(ph, [[3.0, 0.2]], 3, r3["u"], unit_loads(3))
    assert np.max(np.abs(C3 - fem.material_matrix(3, (3.0, 0.2)))) < 1e-13


def test_thermal_laminate_exact_means():
    shape = (8, 4, 4)
    ph = laminate(shape, axis=0)
    k = np.array([1.0, 10.0])
    res = hz.solve(ph, k, 1, unit_loads(1), "uno", tol=1e-13, max_iter=200)
    C = hz.effective_tensor(ph, k, 1, res["u"], unit_loads(1))
    harm = 1.0 / np.mean(1.0 / k)
    arith = np.mean(k)
    assert C[0, 0] == pytest.approx(harm, rel=1e-11)
    assert C[1, 1] == pytest.approx(arith, rel=1e-12)
    assert C[2, 2] == pytest.approx(arith, rel=1e-12)
    assert np.max(np.abs(C - np.diag(np.diag(C)))) < 1e-12


def test_elastic_laminate_matches_layer_averaging():
    # Layers normal to x1: traction components (11, 12, 13) and in-plane strains (22, 33, 23)
    # are continuous, which gives the exact laminate stiffness by layer averaging.
    shape = (8, 4, 4)
    ph = laminate(shape, axis=0)
    res = hz.solve(ph, EL, 3, unit_loads(3), "uno", tol=1e-13, max_iter=300)
    C = hz.effective_tensor(ph, EL, 3, res["u"], unit_loads(3))
    Nn = [0, 3, 4]
    Tt = [1, 2, 5]
    Ds = [fem.material_matrix(3, p) for p in EL]
    inv_nn = [np.linalg.inv(D[np.ix_(Nn, Nn)]) for D in Ds]
    A = np.mean(inv_nn, axis=0)
    Ai = np.linalg.inv(A)
    Bm = np.mean([inv_nn[i] @ Ds[i][np.ix_(Nn, Tt)] for i in range(2)], axis=0)
    Cm = np.mean([Ds[i][np.ix_(Tt, Nn)] @ inv_nn[i] for i in range(2)], axis=0)
    Tm = np.mean([Ds[i][np.ix_(Tt, Tt)] - Ds[i][np.ix_(Tt, Nn)] @ inv_nn[i] @ Ds[i][np.ix_(Nn, Tt)]
                  for i in range(2)], axis=0)
    Cx = np.zeros((6, 6))
    Cx[np.ix_(Nn, Nn)] = Ai
    Cx[np.ix_(Nn, Tt)] = Ai @ Bm
    Cx[np.ix_(Tt, Nn)] = Cm @ Ai
    Cx[np.ix_(Tt, Tt)] = Tm + Cm @ Ai @ Bm
    # loads whose right-hand side is zero up to rounding leave ~1e-9 noise in their columns
    assert np.max(np.abs(C - Cx)) < 1e-8 * np.max(np.abs(Cx))


@pytest.mark.parametrize("physics,props", [(1, TH), (3, EL)])
def test_effective_tensor_symmetric_and_bounded(physics, props):
    phase, vf = rsa_spheres((8, 8, 8), 2.0, 0.3, seed=12)
    loads = unit_loads(physics)
    res = hz.solve(phase, props, physics, loads, "uno", tol=1e-11)
    C = hz.effective_tensor(phase, props, physics, res["u"], loads)
    W = hz.energy_tensor(phase, props, physics, res["u"], loads)
    assert np.max(np.abs(C - C.T)) < 1e-8 * np.max(np.abs(C))
    assert np.max(np.abs(C - W)) < 1e-8 * np.max(np.abs(C))
    Ds = [fem.material_matrix(physics, p) for p in props]
    frac = np.array([1 - phase.mean(), phase.mean()])
    voigt = frac[0] * Ds[0] + frac[1] * Ds[1]
    reuss = np.linalg.inv(frac[0] * np.linalg.inv(Ds[0]) + frac[1] * np.linalg.inv(Ds[1]))
    Cs = 0.5 * (C + C.T)
    assert np.linalg.eigvalsh(voigt - Cs).min() > -1e-9
    assert np.linalg.eigvalsh(Cs - reuss).min() > -1e-9


def test_shift_and_permutation_invariance():
    phase, _ = rsa_spheres((6, 6, 6), 1.5, 0.3, seed=13)
    L = unit_loads(1)
    C = hz.effective_tensor(phase, TH, 1, hz.solve(phase, TH, 1, L, "uno", 1e-12)["u"], L)
    ps = np.roll(phase, (2, -1, 3), axis=(0, 1, 2))
    Cs = hz.effective_tensor(ps, TH, 1, hz.solve(ps, TH, 1, L, "uno", 1e-12)["u"], L)
    assert np.max(np.abs(C - Cs)) < 1e-9
    pp = np.ascontiguousarray(phase.transpose(2, 0, 1))  # new axes (x3, x1, x2)
    Cp = hz.effective_tensor(pp, TH, 1, hz.solve(pp, TH, 1, L, "uno", 1e-12)["u"], L)
    perm = [2, 0, 1]
    assert np.max(np.abs(Cp - C[np.ix_(perm, perm)])) < 1e-9


def test_cg_energy_error_bound():
    # ||e_m||_A <= 2 C^m ||e_0||_A with C from the condition number of P K (Eq. cg-convergence)
    shape = (5, 5, 5)
    phase = random_phase(shape, 2, seed=14)
    K = fem.assemble_K(phase, TH, 1)
    f = fem.assemble_f(phase, TH, 1, [1.0, 0.0, 0.0])
    ustar = hz.direct_solve(K, f, 1)
    d = K.diagonal()
    Kd = K.toarray()
    ev = np.sort(np.linalg.eigvals(Kd / d[:, None]).real)[1:]
    cond = ev.max() / ev.min()
    C = (np.sqrt(cond) - 1) / (np.sqrt(cond) + 1)
    errs = []

    def A(v):
        return K @ v

    u = np.zeros_like(f)
    r = f.copy()
    dd = np.zeros_like(f)
    g1 = 1.0
    e0 = None
    for m in range(40):
        e = u - ustar
        e = e - e.mean()
        en = np.sqrt(e @ (K @ e))
        if e0 is None:
            e0 = en
        if 2 * C ** m > 1e-7:  # below this the energy norm is at its rounding floor
            errs.append(en <= 2 * C ** m * e0 * (1 + 1e-9))
        s = r / d
        g0, g1 = g1, r @ s
        dd = s + g1 / g0 * dd
        p = A(dd)
        al = g1 / (dd @ p)
        r = r - al * p
        u = u + al * dd
    assert all(errs)


@pytest.mark.parametrize("physics,props", [(1, [1.0, 5.0]), (3, [[1.0, 0.3], [4.0, 0.2]])])
def test_sensitivity_matches_central_fd(physics, props):
    shape = (4, 4, 4)
    phase = random_phase(shape, 2, seed=15)
    loads = unit_loads(physics)[: (3 if physics == 1 else 2)]
    c = 1 if physics == 1 else 3

    def tensor(pr):
        K = fem.assemble_K(phase, pr, physics)
        us = [hz.zero_mean(hz.direct_solve(K, fem.assemble_f(phase, pr, physics, l), c), c)
              for l in loads]
        return us, hz.energy_tensor(phase, pr, physics, us, loads)

    us, _ = tensor(props)
    S = hz.sensitivity(phase, props, physics, us, loads)
    pr = np.array(props, dtype=np.float64)
    flat = pr.reshape(-1)
    for q in range(flat.size):
        hstep = 1e-4 * max(1.0, abs(flat[q]))
        fp, fm = flat.copy(), flat.copy()
        fp[q] += hstep
        fm[q] -= hstep
        Wp = tensor(fp.reshape(pr.shape))[1]
        Wm = tensor(fm.reshape(pr.shape))[1]
        fd = (Wp - Wm) / (2 * hstep)
        # O(h^2) truncation of the central difference dominates for nu near 0.5
        assert np.max(np.abs(S[q] - fd)) < 1e-6 * max(1.0, np.max(np.abs(fd)))
