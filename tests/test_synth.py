"""The seeded input generators: the blocked RSA sampler against a one-candidate-at-a-time
statement of the same procedure, jam handling, and the workload recipes' ranges."""
import numpy as np
import pytest

from synth import rsa_spheres, workload


def _rsa_one_at_a_time(shape, radius, vf, seed, max_rejections, overlap_on_jam=True):
    n = np.asarray(shape, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    phase = np.zeros(shape, dtype=np.uint8)
    centres = []
    rejections, jammed = 0, False
    grid = np.stack(np.meshgrid(*[np.arange(s) + 0.5 for s in shape], indexing="ij"), axis=-1)
    while True:
        c = rng.uniform(0.0, 1.0, size=3) * n
        if centres and not jammed:
            dmin = min(float(np.sum((q - c - n * np.round((q - c) / n)) ** 2)) for q in centres)
            if dmin < (2.0 * radius) ** 2:
                rejections += 1
                if rejections >= max_rejections:
                    if not overlap_on_jam:
                        raise RuntimeError("jammed")
                    jammed = True
                continue
        rejections = 0
        centres.append(c)
        d = grid - c
        d -= n * np.round(d / n)
        phase[np.sum(d * d, axis=-1) <= radius * radius] = 1
        if phase.mean() >= vf:
            return phase, float(phase.mean())


@pytest.mark.parametrize("shape,radius,vf,seed,maxrej", [((16, 16, 16), 3.0, 0.25, 5, 10_000),
                                                          ((12, 10, 14), 2.0, 0.3, 7, 10_000),
                                                          ((10, 10, 10), 2.0, 0.45, 3, 300)])
def test_rsa_matches_one_candidate_at_a_time(shape, radius, vf, seed, maxrej):
    got, f = rsa_spheres(shape, radius, vf, seed, max_rejections=maxrej)
    ref, fr = _rsa_one_at_a_time(shape, radius, vf, seed, maxrej)
    assert np.array_equal(got, ref) and f == fr and f >= vf


def test_rsa_jam_raises_without_overlap():
    with pytest.raises(RuntimeError):
        rsa_spheres((10, 10, 10), 2.0, 0.6, 3, max_rejections=300, overlap_on_jam=False)


def test_training_workload_ranges():
    for i in range(8):
        w = workload(4, i)
        assert w["phase"].shape == (32, 32, 32)
        assert 0.1 <= w["vf"] <= 0.45
        assert 5.0 <= w["props"][1] <= 100.0


def test_rsa_disks_seeded_non_overlapping_and_periodic():
    from synth import rsa_disks
    p1, f1 = rsa_disks((40, 50), 3.0, 0.3, seed=4)
    p2, f2 = rsa_disks((40, 50), 3.0, 0.3, seed=4)
    assert np.array_equal(p1, p2) and f1 == f2
    assert 0.3 <= f1 < 0.36 and p1.dtype == np.uint8
    # a disk near the edge wraps: the inclusion set is invariant under no shift but touches edges
    p3, _ = rsa_disks((16, 16), 2.5, 0.5, seed=9)
    assert p3[0].any() or p3[:, 0].any()
