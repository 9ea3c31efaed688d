"""Seeded periodic microstructure generators.

The paper's experiments use image datasets of two-phase microstructures (2D 400^2 images and
3D 192^3 voxel images, Sec. 6 "Problem formulations").  Those datasets are not available, so
synthetic two-phase voxel images stand in for them: spherical inclusions placed by periodic
random sequential addition (RSA) inside a matrix phase.

Conventions
-----------
* A microstructure is a ``uint8`` array ``phase[i1, i2, i3]`` of shape ``(N1, N2, N3)``; one
  entry per voxel (= per trilinear hexahedral element), ``0`` = matrix, ``1`` = inclusion.
  ``i3`` is the fastest (C-order) axis.
* Voxel ``(i1, i2, i3)`` has its centre at ``(i + 1/2)`` in voxel units.
* All draws use ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["rsa_spheres", "random_phase", "laminate", "random_field", "unit_loads",
           "config_seed", "workload"]

SEED_BASE = 2508002681


def config_seed(config: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of workload ``config`` (1-based workload numbers)."""
    return SEED_BASE + 1000 * config + instance


def _min_image(delta: np.ndarray, n: np.ndarray) -> np.ndarray:
    return delta - n * np.round(delta / n)


def rsa_spheres(shape, radius: float, volume_fraction: float, seed: int,
                max_rejections: int = 10_000, overlap_on_jam: bool = True):
    """Periodic RSA of non-overlapping spheres until the voxel fraction reaches a target.

    Centres are drawn uniformly in ``[0, N1) x [0, N2) x [0, N3)``.  A candidate is accepted
    when its minimum-image distance to every accepted centre is at least ``2 * radius``.  A voxel
    belongs to the inclusion phase when its centre lies within ``radius`` (minimum image) of an
    accepted centre.  Placement stops at the first accepted sphere that brings the inclusion
    voxel fraction to ``volume_fraction`` or above.

    Non-overlapping RSA jams near a sphere fraction of 0.38, below the top of some requested
    ranges (0.4).  After ``max_rejections`` consecutive rejected candidates the packing counts as
    jammed: with ``overlap_on_jam`` the remaining spheres are placed without the distance test
    (penetrable spheres, the same random stream), else ``RuntimeError`` is raised.

    Returns ``(phase, achieved_fraction)``.
    """
    shape = tuple(int(s) for s in shape)
    n = np.asarray(shape, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    phase = np.zeros(shape, dtype=np.uint8)
    if volume_fraction <= 0.0:
        return phase, 0.0
    centres = np.zeros((0, 3))
    total = float(np.prod(shape))
    rejections = 0
    jammed = False
    r = float(radius)
    reach = int(np.ceil(r)) + 1
    # candidates are drawn in blocks (the same stream as one draw of three per candidate) and
    # tested against the accepted centres all at once, in drawing order
    block = np.zeros((0, 3))
    pos = 0
    while True:
        if pos == block.shape[0]:
            block = rng.uniform(0.0, 1.0, size=(1024, 3)) * n
            pos = 0
        if centres.shape[0] and not jammed:
            # window grows with the run of rejections (few candidates while most are accepted)
            cand = block[pos:pos + max(16, rejections)]
            d = _min_image(centres[None, :, :] - cand[:, None, :], n)
            ok = np.min(np.einsum("mij,mij->mi", d, d), axis=1) >= (2.0 * r) ** 2
            first = int(np.argmax(ok)) if ok.any() else cand.shape[0]
            if rejections + first >= max_rejections:
                # the candidate that completes max_rejections consecutive rejections
                if not overlap_on_jam:
                    raise RuntimeError("RSA: too many consecutive rejections")
                jammed = True
                pos += max_rejections - rejections
                continue
            if first == cand.shape[0]:
                rejections += first
                pos += first
                continue
            pos += first
        c = block[pos]
        pos += 1
        rejections = 0
        centres = np.vstack([centres, c])
        # mark voxels of this sphere (periodic bounding box)
        idx = []
        for a in range(3):
            lo = int(np.floor(c[a] - r)) - 1
            rng_a = np.arange(lo, lo + 2 * reach + 2)
            idx.append(rng_a)
        g1, g2, g3 = np.meshgrid(*idx, indexing="ij")
        dx = (g1 + 0.5) - c[0]
        dy = (g2 + 0.5) - c[1]
        dz = (g3 + 0.5) - c[2]
        inside = dx * dx + dy * dy + dz * dz <= r * r
        phase[g1[inside] % shape[0], g2[inside] % shape[1], g3[inside] % shape[2]] = 1
        frac = float(phase.sum()) / total
        if frac >= volume_fraction:
            return phase, frac


def rsa_disks(shape, radius: float, area_fraction: float, seed: int, max_rejections: int = 10_000):
    """2D periodic RSA of non-overlapping disks (the 2D counterpart of ``rsa_spheres``): centres
    uniform in [0, N1) x [0, N2), accepted at a minimum-image distance of at least 2 radius from
    every accepted centre, pixels whose centre lies within the radius belong to the inclusion
    phase; stops at the first disk that reaches the area fraction, or after ``max_rejections``
    consecutive rejections (jammed).  Returns ``(phase uint8 [N1, N2], achieved_fraction)``."""
    shape = tuple(int(s) for s in shape)
    n = np.asarray(shape, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    phase = np.zeros(shape, dtype=np.uint8)
    if area_fraction <= 0.0:
        return phase, 0.0
    centres = np.zeros((0, 2))
    total = float(np.prod(shape))
    r = float(radius)
    reach = int(np.ceil(r)) + 1
    rejections = 0
    while rejections < max_rejections:
        c = rng.uniform(0.0, 1.0, size=2) * n
        if centres.shape[0]:
            d = _min_image(centres - c[None, :], n)
            if np.min(np.einsum("ij,ij->i", d, d)) < (2.0 * r) ** 2:
                rejections += 1
                continue
        rejections = 0
        centres = np.vstack([centres, c])
        g1, g2 = np.meshgrid(*[np.arange(int(np.floor(c[a] - r)) - 1, int(np.floor(c[a] - r)) + 2 * reach + 1)
                               for a in range(2)], indexing="ij")
        inside = ((g1 + 0.5) - c[0]) ** 2 + ((g2 + 0.5) - c[1]) ** 2 <= r * r
        phase[g1[inside] % shape[0], g2[inside] % shape[1]] = 1
        frac = float(phase.sum()) / total
        if frac >= area_fraction:
            return phase, frac
    return phase, float(phase.sum()) / total


def random_phase(shape, n_phases: int, seed: int) -> np.ndarray:
    """Voxel-wise independent uniform phase labels in ``[0, n_phases)`` (a rough test image)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, n_phases, size=tuple(shape), dtype=np.uint8)


def laminate(shape, axis: int = 0, period: int | None = None) -> np.ndarray:
    """Two-phase laminate whose phase depends on one coordinate only (half-and-half layers)."""
    shape = tuple(int(s) for s in shape)
    n = shape[axis]
    period = n if period is None else period
    lay = ((np.arange(n) % period) >= period // 2).astype(np.uint8)
    view = [1, 1, 1]
    view[axis] = n
    return np.broadcast_to(lay.reshape(view), shape).copy()


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal field of the given shape (test inputs for operators)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=tuple(shape)).astype(dtype)


def unit_loads(physics: int) -> np.ndarray:
    """The unit macroscopic load cases: 3 gradients (thermal) or 6 Mandel strains (elastic)."""
    dim = 3 if physics == 1 else 6
    return np.eye(dim)


def workload(config: int, instance: int = 0):
    """Inputs of the five benchmark workloads, drawn with their documented recipes.

    Returns a dict with ``phase`` (uint8 image), ``physics`` (1 thermal / 3 elastic),
    ``props`` (per-phase conductivity, or per-phase (E, nu)), ``loads`` and ``tol``.
    """
    seed = config_seed(config, instance)
    if config == 1:
        phase, vf = rsa_spheres((16, 16, 16), 3.0, 0.25, seed)
        return dict(phase=phase, vf=vf, physics=1, props=np.array([1.0, 10.0]),
                    loads=unit_loads(1), tol=1e-8)
    if config == 2:
        phase, vf = rsa_spheres((64, 64, 64), 6.0, 0.3, seed)
        return dict(phase=phase, vf=vf, physics=1, props=np.array([1.0, 100.0]),
                    loads=unit_loads(1), tol=1e-6)
    if config == 3:
        phase, vf = rsa_spheres((64, 64, 64), 6.0, 0.3, seed)
        return dict(phase=phase, vf=vf, physics=3,
                    props=np.array([[1.0, 0.3], [10.0, 0.2]]),
                    loads=unit_loads(3), tol=1e-6)
    if config == 4:
        rng = np.random.Generator(np.random.PCG64(seed))
        r = rng.uniform(2.0, 5.0)
        vf_t = rng.uniform(0.1, 0.4)
        contrast = float(np.exp(rng.uniform(np.log(5.0), np.log(100.0))))
        phase, vf = rsa_spheres((32, 32, 32), r, vf_t, seed + 500_000)
        return dict(phase=phase, vf=vf, physics=1, props=np.array([1.0, contrast]),
                    loads=unit_loads(1)[:1], tol=1e-6)
    if config == 5:
        rng = np.random.Generator(np.random.PCG64(seed))
        n = int(rng.choice([32, 48, 64, 96, 128]))
        contrast = float(np.exp(rng.uniform(np.log(5.0), np.log(1000.0))))
        # radius 6 voxels and fraction 0.3, as in the 64^3 thermal workload
        phase, vf = rsa_spheres((n, n, n), 6.0, 0.3, seed + 500_000)
        return dict(phase=phase, vf=vf, physics=1, props=np.array([1.0, contrast]),
                    loads=unit_loads(1), tol=1e-6)
    raise ValueError(f"unknown workload {config}")
