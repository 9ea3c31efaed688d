"""The serving-style uneven batch: 256 thermal instances with grid sizes drawn from 32^3..128^3,
contrast log-uniform in [5, 1000], three load cases each; the instances of one size share a
batched context and all sizes are solved together (mixed precision, tolerance 1e-6)."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import homogenize as hz
from synth import unit_loads, workload
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu


def _inputs(n):
    # drawn on the host cores by spawned workers (this process already uses CUDA)
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        return pool.starmap(workload, [(5, i) for i in range(n)])


def test_uneven_batch_256_instances():
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import UnevenBatch
    ws = _inputs(256)
    loads = unit_loads(1)
    ub = UnevenBatch(_lib.THERMAL, [w["phase"] for w in ws], [w["props"] for w in ws], loads)
    assert sorted(set(w["phase"].shape[0] for w in ws)) == [32, 48, 64, 96, 128]
    res = ub.solve(tol=1e-6, max_iter=3000, precision=_lib.MIXED)
    C = ub.effective_tensors()
    for i, (iters, tres, status) in enumerate(res):
        assert np.all(status == _lib.OK) and np.all(tres <= 1e-6) and np.all(iters > 0), i
        # symmetric and between the Reuss and Voigt bounds of the two phases
        k0, k1 = ws[i]["props"]
        vf = ws[i]["vf"]
        Ci = C[i]
        assert np.max(np.abs(Ci - Ci.T)) < 1e-5 * np.max(np.abs(Ci)), i
        ev = np.linalg.eigvalsh(0.5 * (Ci + Ci.T))
        assert ev.min() > 1.0 / ((1 - vf) / k0 + vf / k1) * (1 - 1e-6), i
        assert ev.max() < ((1 - vf) * k0 + vf * k1) * (1 + 1e-6), i
    # the oracle on the first two 32^3 instances
    small = [i for i, w in enumerate(ws) if w["phase"].shape[0] == 32][:2]
    for i in small:
        w = ws[i]
        ref = hz.solve(w["phase"], w["props"], 1, loads, "uno", tol=1e-10)
        Cref = hz.effective_tensor(w["phase"], w["props"], 1, ref["u"], loads)
        assert rel(C[i], Cref) < 1e-6
    ub.close()


def _ctx(shape, seed, contrast, batch=1):
    from paper_2508_02681_gb300 import _lib
    from paper_2508_02681_gb300.solver import Homogenization
    from synth import rsa_spheres
    h = Homogenization(_lib.THERMAL, shape, batch=batch)
    ph = np.stack([rsa_spheres(shape, 2.0, 0.3, seed=seed + b)[0] for b in range(batch)])
    h.set_microstructure(ph, 2)
    h.set_phase_properties(np.stack([np.array([1.0, contrast * (b + 1)]) for b in range(batch)]))
    h.set_macro_load(unit_loads(1))
    h.set_uno_weights(_lib.W_REFERENCE_MEDIUM)
    return h


@pytest.mark.parametrize("precision", [0, 1])
def test_one_graph_batch_equals_separate_solves(precision):
    """The batch graph (all contexts as branches of one graph launch) gives the separate solves'
    results: bit for bit in FP64 (same kernels, same launch shapes, deterministic reductions),
    to the mixed-precision tolerance in mixed precision; it is reused on the next call, rebuilt
    when a context's set-up changes its graph, and dropped with a destroyed context."""
    from paper_2508_02681_gb300 import _lib, api
    shapes = [(16, 16, 16), (24, 24, 24), (32, 16, 32)]
    opts = dict(tol=1e-8 if precision == 0 else 1e-6, max_iter=3000, precision=precision)

    def separate():
        hs = [_ctx(s, 10 * i, 10.0 + i, batch=2) for i, s in enumerate(shapes)]
        out = []
        for h in hs:
            info = h.solve(**opts)
            out.append((info.iters.copy(), h.effective_tensor(), h.fluctuation(1, 2)))
            h.close()
        return out

    ref = separate()
    hs = [_ctx(s, 10 * i, 10.0 + i, batch=2) for i, s in enumerate(shapes)]
    for call in range(2):  # built, then reused
        infos = api.unocg_batch_solve([h.ctx for h in hs], api.make_opts(**opts), [2 * 3] * len(hs))
        for h, info, (it, C, u) in zip(hs, infos, ref):
            assert info.status == _lib.OK
            assert np.array_equal(info.iters, it)
            if precision == 0:
                assert np.array_equal(h.effective_tensor(), C)
                assert np.array_equal(h.fluctuation(1, 2), u)
            else:
                assert rel(h.effective_tensor(), C) < 1e-6
    # a change of tile shape invalidates the second context's captured launches
    api.unocg_set_ku_tile(hs[1].ctx, 0)
    infos = api.unocg_batch_solve([h.ctx for h in hs], api.make_opts(**opts), [2 * 3] * len(hs))
    assert all(i.status == _lib.OK for i in infos)
    assert rel(hs[1].effective_tensor(), ref[1][1]) < (1e-12 if precision == 0 else 1e-6)
    # a destroyed context leaves the batch; a new one at possibly the same address joins
    hs[2].close()
    hs[2] = _ctx(shapes[2], 20, 12.0, batch=2)
    infos = api.unocg_batch_solve([h.ctx for h in hs], api.make_opts(**opts), [2 * 3] * len(hs))
    assert all(i.status == _lib.OK for i in infos)
    assert rel(hs[2].effective_tensor(), ref[2][1]) < (1e-12 if precision == 0 else 1e-6)
    for h in hs:
        h.close()
