"""Learned UNO for 2D problems (c = 1 thermal, c = 2 plane strain with the parametrization of
Eq. (local-param-2)), trained by Algorithm 4 on solver-generated data and applied in solves,
against the 2D oracle (oracle/uno2d.py, oracle/fem2d.py).

The library solves a 2D cell as the x1-invariant 3D problem on an extruded grid; the features
of Eq. (features-c-1) / Eq. (features-c-2) come from the GPU transform passes of the extruded
fields (k1 = 0, in-plane entries), the Newton-Raphson steps run on the 2D mode set, and the
trained weights are embedded into the extruded 3D operator.  Checks: the loss falls, the
trained loss equals the oracle's loss of Eq. (fnocg-loss) evaluated in real space on the same
data, and held-out solves with the trained UNO agree with the oracle's 2D PCG with the same
blocks (iterations within 2 % at the 1e-6 tolerance; fields and effective tensor at the FP64 bars
once both are converged to 1e-10)."""
import numpy as np
import pytest

from oracle import fem2d, uno2d
from synth import rsa_disks
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _props(physics, contrast):
    return np.array([1.0, contrast]) if physics == 1 else np.array([[1.0, 0.3], [contrast, 0.2]])


def _solver(physics, phase, props, loads, layers):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization2D
    h = Homogenization2D(physics, phase.shape, layers=layers)
    h.set_microstructure(phase, 2)
    h.set_phase_properties(props)
    h.set_macro_load(loads)
    return h


@pytest.mark.parametrize("physics", [1, 3])
def test_2d_learned_uno_trains_and_solves_like_the_oracle(physics):
    import torch
    from paper_2508_02681_gb300 import _lib, api, training
    shape2, layers, M, n_ms = (32, 32), 4, 4, 16
    c = 1 if physics == 1 else 2
    c3 = 1 if physics == 1 else 3
    dim = 2 if physics == 1 else 3
    loads = np.eye(dim)
    comps = [0] if c == 1 else [1, 2]
    rng = np.random.default_rng(77)
    contrast = np.exp(rng.uniform(np.log(5.0), np.log(50.0), n_ms + 1))
    n = n_ms * dim
    f3 = torch.empty((n, c3, layers) + shape2, dtype=torch.float32, device="cuda")
    u3 = torch.empty_like(f3)
    tmp = torch.empty((c3, layers) + shape2, dtype=torch.float64, device="cuda")
    for i in range(n_ms):
        phase, _ = rsa_disks(shape2, 4.0, 0.3, seed=900 + i)
        h = _solver(physics, phase, _props(physics, contrast[i]), loads, layers)
        h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
        info = h.solve(tol=1e-8, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
        assert info.status == _lib.OK
        for l in range(dim):
            api.unocg_rhs_dev(h.h.ctx, 0, l, tmp)
            f3[dim * i + l].copy_(tmp)
            api.unocg_get_fluctuation_dev(h.h.ctx, 0, l, tmp)
            u3[dim * i + l].copy_(tmp)
        torch.cuda.synchronize()
        h.close()
    a, b = training.features_2d(f3, u3, layers, c)
    w0 = training.reference_modes_2d(physics, _props(physics, float(np.mean(contrast))), shape2, M, layers)
    w, hist = training.second_order_modes_2d(a, b, M, w0, c)
    assert len(hist) > 1 and hist[-1] < hist[0]
    assert all(h1 <= h0 + 1e-9 * abs(h0) for h0, h1 in zip(hist, hist[1:]))
    # the oracle's loss by definition on the same data (one layer of the x1-invariant fields)
    f2 = f3.cpu().numpy().astype(np.float64)[:, comps, 0]
    u2 = u3.cpu().numpy().astype(np.float64)[:, comps, 0]
    delta = float(np.sum(u2 ** 2)) / n
    for ww, hh in ((w0, hist[0]), (w, hist[-1])):
        L_or = uno2d.loss_by_definition(uno2d.modes_Q(ww, M, shape2, c), f2, u2)
        assert abs(hh + delta - L_or) <= 2e-4 * L_or, (hh + delta, L_or)
    # held-out problem: the trained UNO in the extruded GPU solve and in the oracle's 2D PCG
    phase, _ = rsa_disks(shape2, 4.0, 0.3, seed=999)
    props = _props(physics, float(contrast[-1]))
    Q2 = uno2d.modes_Q(w, M, shape2, c)
    blocks3 = training.modes2d_blocks3d(w, M, shape2, layers, c)
    bcb = (False, False)
    for tol in (1e-6, 1e-10):
        ref = fem2d.solve(phase, props, physics, bcb, loads, precond="uno", tol=tol, Q=Q2)
        Cref = fem2d.effective_tensor(phase, props, physics, bcb, ref["u"], loads)
        h = _solver(physics, phase, props, loads, layers)
        h.set_uno_weights(_lib.W_BLOCKS, blocks3.ravel())
        info = h.solve(tol=tol, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.FP64)
        assert info.status == _lib.OK
        for l in range(dim):
            if tol > 1e-8:
                # CG's sensitivity to rounding grows with the iteration count: within 2 %
                it, it_ref = int(info.iters[l]), ref["iters"][l]
                assert abs(it - it_ref) <= max(1, 0.02 * it_ref), (l, it, it_ref)
            else:
                assert rel(h.fluctuation(0, l), ref["u"][l]) < 1e-9
        assert rel(h.effective_tensor()[0], Cref) < (1e-10 if tol < 1e-8 else 1e-7)
        if tol == 1e-6:
            info = h.solve(tol=tol, max_iter=5000, precond=_lib.PRECOND_UNO, precision=_lib.MIXED)
            assert info.status == _lib.OK and np.all(info.true_rel_res <= 1e-6)
            assert rel(h.effective_tensor()[0], Cref) < 1e-6
        h.close()
    print("2D c =", c, "loss + delta", hist[0] + delta, "->", hist[-1] + delta, "in", len(hist) - 1,
          "Newton steps; held-out oracle iterations with the trained UNO", ref["iters"])
