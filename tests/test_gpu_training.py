"""GPU UNO operator for training (Sec. 5.3, Algorithm 3): FP32 apply s = P_theta r and the
hand-written backward (input gradient P g and weight gradient through psi), against the FP64
oracle and central finite differences of the loss of Eq. (fnocg-loss)."""
import numpy as np
import pytest

from oracle import training, uno
from synth import random_field
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _theta(shape, c, seed):
    rng = np.random.default_rng(seed)
    C = c * (c + 1) // 2
    th = rng.standard_normal((shape[0], shape[1], shape[2] // 2 + 1, C)) * 0.3
    th[..., 0] += 1.0
    if c == 3:
        th[..., 1] += 1.0
        th[..., 3] += 1.0
    return th


@pytest.mark.parametrize("c,shape", [(1, (8, 6, 10)), (3, (6, 8, 8)), (1, (32, 32, 32)), (3, (16, 32, 32)),
                                     (1, (8, 64, 64)), (3, (64, 16, 16)), (1, (4, 128, 128))])
def test_apply_fp32_matches_oracle(c, shape):
    import torch
    from paper_2508_02681_gb300 import api
    th = _theta(shape, c, 1)
    B = 2
    r = np.stack([random_field((c,) + shape, seed=10 + b) for b in range(B)])
    op = api.unocg_uno_create(c, *shape)
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    api.unocg_uno_set_theta_dev(op, tt)
    rr = torch.tensor(r, dtype=torch.float32, device="cuda")
    ss = torch.empty_like(rr)
    api.unocg_uno_apply_dev(op, B, rr, ss)
    torch.cuda.synchronize()
    Q = uno.symmetrize_half(uno.psi(th.astype(np.float32).astype(np.float64), c), shape[2])
    for b in range(B):
        assert rel(ss[b].cpu().numpy().astype(np.float64), uno.uno_apply(Q, r[b])) < 2e-5
    api.unocg_uno_destroy(op)


@pytest.mark.parametrize("c,shape", [(1, (6, 8, 8)), (3, (4, 6, 8))])
def test_backward_matches_oracle_gradient_and_fd(c, shape):
    import torch
    from paper_2508_02681_gb300 import api
    th = _theta(shape, c, 2).astype(np.float32).astype(np.float64)
    B = 3
    f = np.stack([random_field((c,) + shape, seed=20 + b) for b in range(B)])
    u = np.stack([random_field((c,) + shape, seed=40 + b) for b in range(B)])
    N3 = shape[2]

    def loss(theta):
        return training.loss_by_definition(uno.symmetrize_half(uno.psi(theta, c), N3), f, u)

    Q = uno.symmetrize_half(uno.psi(th, c), N3)
    s = np.stack([uno.uno_apply(Q, f[b]) for b in range(B)])
    gs = 2.0 * (s - u) / B  # dL/ds
    op = api.unocg_uno_create(c, *shape)
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    api.unocg_uno_set_theta_dev(op, tt)
    fr = torch.tensor(f, dtype=torch.float32, device="cuda")
    gg = torch.tensor(gs, dtype=torch.float32, device="cuda")
    gr = torch.empty_like(fr)
    gt = torch.empty_like(tt)
    api.unocg_uno_backward_dev(op, B, fr, gg, gr, gt)
    torch.cuda.synchronize()
    # input gradient: P is self-adjoint
    for b in range(B):
        assert rel(gr[b].cpu().numpy().astype(np.float64), uno.uno_apply(Q, gs[b])) < 2e-5
    gt = gt.cpu().numpy().astype(np.float64)
    # weight gradient against central differences of the oracle loss
    rng = np.random.default_rng(7)
    flat = th.reshape(-1)
    for _ in range(6):
        i = int(rng.integers(flat.size))
        eps = 1e-4
        tp, tm = flat.copy(), flat.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (loss(tp.reshape(th.shape)) - loss(tm.reshape(th.shape))) / (2 * eps)
        assert gt.reshape(-1)[i] == pytest.approx(fd, rel=2e-3, abs=2e-4 * max(1.0, np.max(np.abs(gt))))
    api.unocg_uno_destroy(op)


def test_autograd_function_training_decreases_loss():
    """Adam steps of Algorithm 3 (gradients from the hand-written backward through the
    autograd Function) reduce the loss of Eq. (fnocg-loss) toward a known optimum."""
    import torch
    from paper_2508_02681_gb300 import api
    from paper_2508_02681_gb300.solver import uno_function
    shape = (16, 16, 16)
    c = 1
    rng = np.random.default_rng(3)
    th_target = 1.0 + 0.3 * rng.standard_normal((16, 16, 9, 1))
    Qt = uno.symmetrize_half(uno.psi(th_target, 1), 16)
    f = np.stack([random_field((c,) + shape, seed=60 + b) for b in range(4)])
    u = np.stack([uno.uno_apply(Qt, f[b]) for b in range(4)])
    theta = torch.tensor(0.5 * th_target, dtype=torch.float32, device="cuda", requires_grad=True)
    F = torch.tensor(f, dtype=torch.float32, device="cuda")
    U = torch.tensor(u, dtype=torch.float32, device="cuda")
    op = api.unocg_uno_create(c, *shape)
    Fn = uno_function()
    opt = torch.optim.Adam([theta], lr=5e-2)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        s = Fn.apply(F, theta, op)
        L = ((s - U) ** 2).sum() / F.shape[0]
        L.backward()
        opt.step()
        losses.append(float(L.detach()))
    api.unocg_uno_destroy(op)
    assert losses[-1] < 0.05 * losses[0]


def test_config4_training_workload():
    """The 32^3 training workload: 512 seeded thermal microstructures (radius U[2,5], volume
    fraction U[0.1,0.4], contrast log-uniform in [5,100]), targets from this library's solves,
    Adam at batch 64 for 200 epochs on the paper's weight layout.  Checks: the loss decreases;
    the trained weights drive UNO-CG to tolerance on held-out instances; the weight gradient and
    the adjoint d(kappa_eff)/d(kappa_p) match central differences (h = 1e-4) on 4 instances."""
    import torch
    from paper_2508_02681_gb300 import _lib, api, training as tr
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import workload
    import multiprocessing as mp
    import os
    shape = (32, 32, 32)
    # the inputs are drawn on the host cores; spawned workers (this process already uses CUDA)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        ws = pool.starmap(workload, [(4, i) for i in range(512)])
    f, u, iters = tr.generate_data([w["phase"] for w in ws], [w["props"] for w in ws],
                                   np.array([1.0, 0.0, 0.0]), shape)
    assert max(iters) < 5000
    # the paper's layout (inner bypass + modes of K_M, M = 8), started from the reference medium
    # at the geometric-mean contrast; Adam as in Algorithm 3
    M = 8
    w0 = tr.reference_modes(shape, M, 0.5 * (1.0 + np.sqrt(5.0 * 100.0)))
    wt, losses = tr.train(f, u, w0, epochs=200, batch=64, lr=1e-2, modes_M=M)
    # first-order training lowers the loss of Eq. (fnocg-loss) by a few per cent and settles
    assert losses[-1] < 0.97 * losses[0]
    assert losses[-1] <= 1.02 * min(losses)
    # trained weights in solves of held-out instances: SPD through the bypass, to tolerance in
    # FP64 and mixed precision, in about as many iterations as the starting weights
    wtr = wt.cpu().numpy().astype(np.float64)
    its_start, its_trained = 0, 0
    for i in range(512, 516):
        w = workload(4, i)
        for weights, prec in ((w0, _lib.FP64), (wtr, _lib.FP64), (wtr, _lib.MIXED)):
            h = Homogenization(_lib.THERMAL, shape)
            h.set_microstructure(w["phase"], 2)
            h.set_phase_properties(w["props"])
            h.set_macro_load(np.eye(3)[:1])
            h.set_uno_modes(M, np.asarray(weights, dtype=np.float64))
            info = h.solve(tol=1e-6, max_iter=3000, precond=_lib.PRECOND_UNO, precision=prec)
            assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
            if prec == _lib.FP64:
                if weights is w0:
                    its_start += int(info.iters[0])
                else:
                    its_trained += int(info.iters[0])
            h.close()
    assert its_trained <= 1.1 * its_start + 2
    # second-order training (Algorithm 4) from the features of the same data reaches the
    # global optimum of the loss: at or below what Adam reached
    a_f, b_f = tr.features(f, u)
    w2, hist = tr.second_order_modes(a_f, b_f, M, w0)
    delta = float((u.double() ** 2).sum()) / u.shape[0]
    assert hist[-1] + delta <= losses[-1] * (1 + 1e-3)
    assert all(h1 <= h0 + 1e-9 * abs(h0) for h0, h1 in zip(hist, hist[1:]))
    # weight gradient on 4 instances against central differences of the FP64 oracle loss
    f4 = f[:4].cpu().numpy().astype(np.float64)
    u4 = u[:4].cpu().numpy().astype(np.float64)
    Q = uno.modes_Q(wtr, M, shape, 1)
    s = np.stack([uno.uno_apply(Q, f4[b]) for b in range(4)])
    gs = 2.0 * (s - u4) / 4
    op = api.unocg_uno_create(1, *shape)
    tt = torch.tensor(wtr, dtype=torch.float32, device="cuda")
    api.unocg_uno_set_modes_dev(op, M, tt)
    gt = torch.empty_like(tt)
    api.unocg_uno_backward_dev(op, 4, torch.tensor(f4, dtype=torch.float32, device="cuda"),
                               torch.tensor(gs, dtype=torch.float32, device="cuda"), None, gt)
    torch.cuda.synchronize()
    gt = gt.cpu().numpy().reshape(-1).astype(np.float64)
    api.unocg_uno_destroy(op)

    def loss(wv):
        return training.loss_by_definition(uno.modes_Q(wv, M, shape, 1), f4, u4)

    rng = np.random.default_rng(9)
    flat = wtr.reshape(-1)
    big = np.argsort(-np.abs(gt))[:64]
    for i in [0] + list(rng.choice(big, 4, replace=False)):
        hstep = 1e-4 * max(1.0, abs(flat[i]))
        tp, tm = flat.copy(), flat.copy()
        tp[i] += hstep
        tm[i] -= hstep
        fd = (loss(tp.reshape(wtr.shape)) - loss(tm.reshape(wtr.shape))) / (2 * hstep)
        assert gt[i] == pytest.approx(fd, rel=5e-3)
    # adjoint sensitivities on 4 instances against central differences of the solver
    for i in range(4):
        w = ws[i]

        def keff(props):
            hh = Homogenization(_lib.THERMAL, shape)
            hh.set_microstructure(w["phase"], 2)
            hh.set_phase_properties(props)
            hh.set_macro_load(np.eye(3))
            hh.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
            hh.solve(tol=1e-12, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
            C = hh.effective_tensor()[0]
            S = hh.sensitivity()[0]
            hh.close()
            return C, S

        C0, S0 = keff(w["props"])
        for p in range(2):
            hstep = 1e-4 * w["props"][p]
            pp, pm = w["props"].copy(), w["props"].copy()
            pp[p] += hstep
            pm[p] -= hstep
            fd = (keff(pp)[0] - keff(pm)[0]) / (2 * hstep)
            assert rel(S0[p], fd) < 1e-6


@pytest.mark.parametrize("c,shape,M", [(1, (8, 10, 12), 2), (3, (6, 8, 8), 1), (1, (32, 32, 32), 8),
                                       (3, (16, 16, 16), 3)])
def test_modes_operator_matches_oracle(c, shape, M):
    """The paper's weight layout (inner bypass + modes of K_M) in the training operator: apply,
    input gradient and weight gradient against the FP64 oracle."""
    import torch
    from paper_2508_02681_gb300 import api
    rng = np.random.default_rng(5)
    w = (rng.standard_normal((1 + len(uno.mode_list(M)), uno.n_unique(c))) * 0.4 + 0.7)
    w = w.astype(np.float32).astype(np.float64)
    B = 2
    f = np.stack([random_field((c,) + shape, seed=70 + b) for b in range(B)])
    u = np.stack([random_field((c,) + shape, seed=80 + b) for b in range(B)])
    Q = uno.modes_Q(w, M, shape, c)
    s_ref = np.stack([uno.uno_apply(Q, f[b]) for b in range(B)])
    gs = 2.0 * (s_ref - u) / B
    op = api.unocg_uno_create(c, *shape)
    wt = torch.tensor(w, dtype=torch.float32, device="cuda")
    api.unocg_uno_set_modes_dev(op, M, wt)
    fr = torch.tensor(f, dtype=torch.float32, device="cuda")
    ss = torch.empty_like(fr)
    api.unocg_uno_apply_dev(op, B, fr, ss)
    gr = torch.empty_like(fr)
    gw = torch.empty_like(wt)
    api.unocg_uno_backward_dev(op, B, fr, torch.tensor(gs, dtype=torch.float32, device="cuda"), gr, gw)
    torch.cuda.synchronize()
    for b in range(B):
        assert rel(ss[b].cpu().numpy().astype(np.float64), s_ref[b]) < 2e-5
        assert rel(gr[b].cpu().numpy().astype(np.float64), uno.uno_apply(Q, gs[b])) < 2e-5
    R, U = training.spectra(f), training.spectra(u)
    g_ref = training.grad_modes(w, M, shape, c, training.grad_entries_general(Q, R, U, shape))
    assert rel(gw.cpu().numpy().astype(np.float64), g_ref) < 1e-4
    api.unocg_uno_destroy(op)


@pytest.mark.parametrize("physics", [1, 3])
def test_solver_modes_weights_match_oracle_and_converge(physics):
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    shape = (16, 16, 16)
    c = 1 if physics == 1 else 3
    M = 3
    rng = np.random.default_rng(6)
    w = rng.standard_normal((1 + len(uno.mode_list(M)), uno.n_unique(c))) * 0.3 + 0.9
    from synth import rsa_spheres, unit_loads
    phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=8)
    props = np.array([1.0, 10.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])
    h = Homogenization(physics, shape)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(unit_loads(physics)[:2])
    h.set_uno_modes(M, w)
    nh = shape[0] * shape[1] * (shape[2] // 2 + 1)
    got = api.unocg_get_uno_weights(h.ctx, 0, nh, uno.n_unique(c)).reshape(shape[0], shape[1], -1, uno.n_unique(c))
    ref = uno.entries_from_blocks(uno.modes_Q(w, M, shape, c))
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    for prec in (_lib.FP64, _lib.MIXED):
        info = h.solve(tol=1e-6, max_iter=5000, precond=_lib.PRECOND_UNO, precision=prec)
        assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
    h.close()


@pytest.mark.parametrize("shape", [(8, 6, 10), (16, 32, 32), (32, 32, 32)])
def test_features_match_oracle(shape):
    """Features of Eq. (features-c-1) from the GPU transform passes against the oracle."""
    import torch
    from paper_2508_02681_gb300 import training as tr
    B = 5
    f = np.stack([random_field((1,) + shape, seed=300 + b) for b in range(B)])
    u = np.stack([random_field((1,) + shape, seed=400 + b) for b in range(B)])
    a, b = tr.features(torch.tensor(f, dtype=torch.float32, device="cuda"),
                       torch.tensor(u, dtype=torch.float32, device="cuda"), chunk=2)
    fr = f.astype(np.float32).astype(np.float64)
    ur = u.astype(np.float32).astype(np.float64)
    a_ref, b_ref = training.features_c1(training.spectra(fr), training.spectra(ur), shape)
    assert rel(a, a_ref) < 1e-5
    assert rel(b, b_ref) < 1e-5


@pytest.mark.parametrize("physics,M,shape", [(1, 3, (12, 10, 12)), (3, 2, (8, 10, 6))])
def test_reference_modes_blocks_match_oracle(physics, M, shape):
    """Bypass-plus-modes weights built from the reference medium (c = 1 and c = 3): Q equals the
    oracle's FANS weights S_ref(k)^{-1} on the modes of K_M and lambda_min I elsewhere."""
    from paper_2508_02681_gb300 import _lib, training as tr
    c = 1 if physics == 1 else 3
    ref = 2.0 if physics == 1 else (5.0, 0.25)
    w = tr.reference_modes_blocks(physics, shape, M, ref)
    Qref = uno.reference_medium_Q(physics, [ref] if physics == 1 else [list(ref)], shape)
    lam = uno.min_eigenvalue(Qref)
    Qm = uno.modes_Q(w, M, shape, c)
    in_set = np.zeros(Qm.shape[:3], bool)
    for k1, k2, k3 in uno.mode_list(M):
        in_set[k1 % shape[0], k2 % shape[1], k3] = True
    scale = np.max(np.abs(Qref))
    assert np.max(np.abs(Qm[in_set] - Qref[in_set])) < 1e-12 * scale
    assert np.max(np.abs(Qm[~in_set] - lam * np.eye(c))) < 1e-12 * scale
    if physics == 1:
        assert np.max(np.abs(w - tr.reference_modes(shape, M, ref))) < 1e-12 * np.max(np.abs(w))


def _band_limited(c, n, M, seed):
    """Samples on an n^3 grid of a real zero-mean field whose Fourier modes lie in [-M, M]^3."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    X = np.meshgrid(x, x, x, indexing="ij")
    out = np.zeros((c, n, n, n))
    for comp in range(c):
        for _ in range(12):
            k = rng.integers(-M, M + 1, 3)
            if not k.any():
                continue
            a, b = rng.standard_normal(2)
            ph = 2 * np.pi * (k[0] * X[0] + k[1] * X[1] + k[2] * X[2])
            out[comp] += a * np.cos(ph) + b * np.sin(ph)
    return out


@pytest.mark.parametrize("physics,M", [(1, 4), (3, 3)])
def test_modes_weights_resolution_invariant_on_band_limited_fields(physics, M):
    """Sec. 5.2.2: the learned modes act on the continuous operator, so one set of weights
    preconditions every resolution.  For a field band-limited to [-M, M]^3 the unitary
    transform carries its Fourier coefficients scaled by sqrt(n), Q(k) multiplies them and the
    inverse transform undoes the scale: s = P r samples the same continuous field on a 16^3 and
    a 32^3 grid."""
    import torch
    from paper_2508_02681_gb300 import _lib, api
    from paper_2508_02681_gb300.solver import Homogenization
    c = 1 if physics == 1 else 3
    rng = np.random.default_rng(11)
    w = rng.standard_normal((1 + len(uno.mode_list(M)), uno.n_unique(c))) * 0.3 + 0.9
    out = {}
    for n in (16, 32):
        shape = (n, n, n)
        h = Homogenization(physics, shape)
        h.set_microstructure(np.zeros(shape, np.uint8), 1)
        h.set_phase_properties(np.array([1.0]) if c == 1 else np.array([[1.0, 0.3]]))
        h.set_macro_load(np.eye(3 if c == 1 else 6)[:1])
        h.set_uno_modes(M, w)
        r = torch.tensor(_band_limited(c, n, M, seed=5), dtype=torch.float64, device="cuda")
        s = torch.empty_like(r)
        api.unocg_apply_uno_dev(h.ctx, 0, r, s)
        torch.cuda.synchronize()
        out[n] = s.cpu().numpy()
        h.close()
    fine = out[32][:, ::2, ::2, ::2]
    assert np.max(np.abs(fine - out[16])) < 1e-12 * np.max(np.abs(out[16]))
    assert np.max(np.abs(out[16])) > 1.0


@pytest.mark.parametrize("physics,M", [(1, 8), (3, 4)])
def test_weights_from_32_solve_at_64(physics, M):
    """Resolution transfer (Sec. 5.2.2): bypass-plus-modes weights built at 32^3 precondition the
    same cell at 64^3 (spheres of radius 6 voxels, volume fraction 0.3) to the true residual
    1e-6 in FP64 and mixed precision, in at most 10 % more iterations than the weights built at
    64^3."""
    from paper_2508_02681_gb300 import _lib, training as tr
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import rsa_spheres, unit_loads
    c = 1 if physics == 1 else 3
    ref = 5.5 if physics == 1 else (5.5, 0.25)
    props = np.array([1.0, 100.0]) if physics == 1 else np.array([[1.0, 0.3], [10.0, 0.2]])
    shape = (64, 64, 64)
    phase, _ = rsa_spheres(shape, 6.0, 0.3, seed=77)
    w32 = tr.reference_modes_blocks(physics, (32, 32, 32), M, ref)
    w64 = tr.reference_modes_blocks(physics, shape, M, ref)
    its = {}
    for name, w in (("from32", w32), ("native", w64)):
        for prec in ((_lib.FP64, _lib.MIXED) if name == "from32" else (_lib.FP64,)):
            h = Homogenization(physics, shape)
            h.set_microstructure(phase, 2)
            h.set_phase_properties(props)
            h.set_macro_load(unit_loads(physics)[:1])
            h.set_uno_modes(M, w)
            info = h.solve(tol=1e-6, max_iter=3000, precond=_lib.PRECOND_UNO, precision=prec)
            assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
            its[name, prec] = int(info.iters[0])
            h.close()
    assert its["from32", _lib.FP64] <= 1.1 * its["native", _lib.FP64] + 2


@pytest.mark.parametrize("shape", [(8, 6, 10), (16, 32, 32)])
def test_features_c3_match_oracle(shape):
    """Features of App. C (c = 3, six a and six b per mode) from the GPU transform passes."""
    import torch
    from paper_2508_02681_gb300 import training as tr
    B = 4
    f = np.stack([random_field((3,) + shape, seed=500 + b) for b in range(B)])
    u = np.stack([random_field((3,) + shape, seed=600 + b) for b in range(B)])
    a, b = tr.features(torch.tensor(f, dtype=torch.float32, device="cuda"),
                       torch.tensor(u, dtype=torch.float32, device="cuda"), chunk=3)
    fr = f.astype(np.float32).astype(np.float64)
    ur = u.astype(np.float32).astype(np.float64)
    a_ref, b_ref = training.features_general(training.spectra(fr), training.spectra(ur), shape)
    assert a.shape == a_ref.shape == shape[:2] + (shape[2] // 2 + 1, 6)
    assert rel(a, a_ref) < 1e-5
    assert rel(b, b_ref) < 1e-5


def test_second_order_training_elastic():
    """Algorithm 4 for c = 3 on solver-generated elastic data (16^3, 16 microstructures with the
    six unit strains each, as the paper's elastic training sets; spheres of radius 3, fraction
    0.25, stiffness contrast log-uniform in [5, 50]): features from the GPU passes, Newton-Raphson
    on the bypass-plus-modes weights from the reference-medium start.  The loss falls
    monotonically, the loss from the GPU features matches the oracle's loss of the trained
    weights on the same data, and the trained preconditioner drives held-out FP64 and mixed
    solves to tolerance."""
    import torch
    from paper_2508_02681_gb300 import _lib, api, training as tr
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import rsa_spheres, unit_loads
    shape, n_ms, M = (16, 16, 16), 16, 2
    rng = np.random.default_rng(21)
    contrast = np.exp(rng.uniform(np.log(5.0), np.log(50.0), n_ms + 2))
    n = 6 * n_ms
    f = torch.empty((n, 3) + shape, dtype=torch.float32, device="cuda")
    u = torch.empty_like(f)
    tmp = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")

    def setup(i):
        phase, _ = rsa_spheres(shape, 3.0, 0.25, seed=700 + i)
        props = np.array([[1.0, 0.3], [contrast[i], 0.2]])
        h = Homogenization(_lib.ELASTIC, shape)
        h.set_microstructure(phase, 2)
        h.set_phase_properties(props)
        h.set_macro_load(unit_loads(3))
        return h

    for i in range(n_ms):
        h = setup(i)
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        info = h.solve(tol=1e-8, max_iter=3000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
        assert info.status == _lib.OK
        for l in range(6):
            api.unocg_rhs_dev(h.ctx, 0, l, tmp)
            f[6 * i + l].copy_(tmp)
            api.unocg_get_fluctuation_dev(h.ctx, 0, l, tmp)
            u[6 * i + l].copy_(tmp)
        torch.cuda.synchronize()
        h.close()
    a, b = tr.features(f, u, chunk=32)
    kref = (float(np.sqrt(contrast.mean())), 0.25)
    w0 = tr.reference_modes_blocks(_lib.ELASTIC, shape, M, kref)
    w, hist = tr.second_order_modes_c3(a, b, M, w0)
    assert hist[-1] < hist[0]
    assert all(h1 <= h0 + 1e-9 * abs(h0) for h0, h1 in zip(hist, hist[1:]))
    fr = f.cpu().numpy().astype(np.float64)
    ur = u.cpu().numpy().astype(np.float64)
    delta = float(np.sum(ur ** 2)) / n
    ref = training.loss_from_spectra(uno.modes_Q(w, M, shape, 3), training.spectra(fr), training.spectra(ur), shape)
    assert abs(hist[-1] + delta - ref) <= 1e-4 * delta, (hist[-1], delta, ref)
    # the reference-medium start already fits the data fairly well (loss + delta 46 at 16^3);
    # Newton-Raphson lowers it about five-fold
    assert hist[-1] + delta < 0.5 * (hist[0] + delta)
    # The trained weights are a fixed outcome of the seeded data: the bypass block stays inside
    # the image of psi with eigenvalues near those of the start (0.69-0.71 against 0.70), the
    # safety check of the Remark after Algorithm 2 accepts them, and they drive held-out FP64
    # and mixed solves to tolerance in about as many iterations as the start weights.
    ev0 = np.linalg.eigvalsh(tr.psi(w[0], 3))
    ev_start = np.linalg.eigvalsh(tr.psi(w0[0], 3))
    assert ev0.min() > 0.5 * ev_start.min(), (ev0, ev_start)
    its = {}
    for i in (n_ms, n_ms + 1):
        h = setup(i)
        for used, wt in (("trained", w), ("start", w0)):
            h.set_uno_modes(M, wt)
            for prec in (_lib.FP64, _lib.MIXED):
                info = h.solve(tol=1e-6, max_iter=5000, precond=_lib.PRECOND_UNO, precision=prec)
                assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
                its[i, prec, used] = int(info.c.max_iters)
        h.close()
        for prec in (_lib.FP64, _lib.MIXED):
            assert its[i, prec, "trained"] <= 1.2 * its[i, prec, "start"] + 2, its
    print("loss + delta", hist[0] + delta, "->", hist[-1] + delta, "in", len(hist) - 1, "steps; trained bypass "
          "eigenvalues", ev0, "(start", ev_start, "); held-out iterations", its)


def test_training_checkpoint_resume(tmp_path):
    """Adam training resumed from the checkpoint of epoch 2 continues as the uninterrupted run."""
    import torch
    from paper_2508_02681_gb300 import training as tr
    shape = (8, 8, 8)
    f = torch.tensor(np.stack([random_field((1,) + shape, seed=800 + b) for b in range(16)]), dtype=torch.float32,
                     device="cuda")
    u = torch.tensor(np.stack([random_field((1,) + shape, seed=900 + b) for b in range(16)]), dtype=torch.float32,
                     device="cuda")
    th0 = _theta(shape, 1, 3)
    full, lf = tr.train(f, u, th0, epochs=4, batch=8, lr=1e-2)
    path = str(tmp_path / "ck.pt")
    tr.train(f, u, th0, epochs=2, batch=8, lr=1e-2, checkpoint=path)
    res, lr_ = tr.train(f, u, None, epochs=4, batch=8, lr=1e-2, resume=path)
    assert len(lr_) == 4
    assert np.allclose(lr_, lf, rtol=1e-5)
    assert torch.allclose(res, full, rtol=1e-5, atol=1e-7)
