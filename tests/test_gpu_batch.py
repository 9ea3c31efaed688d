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
