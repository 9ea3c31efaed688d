"""Host checks of the element-by-element K d scheme (Sec. 4.1) before it reaches the GPU.

1. The element force in the Walsh basis of the trilinear brick (corner sums with signs
   prod_{k in M} (2 a_k - 1), G linear in them, inverse Walsh sum) equals the oracle's element
   stiffness from 2x2x2 Gauss quadrature, for elasticity and conduction.
2. A host restatement of the kernels' tiling (32 x 8 node tiles, 33 x 9 element columns with the
   lower halo, KE_CZ node planes per block marched along axis 1, double-buffered corner sums):
   every load stays in bounds, every node is written exactly once, and the result equals the
   oracle's assembled K on ragged and wrapped grids."""
import numpy as np
import pytest

from oracle import fem
from synth import random_field, random_phase

T3, T2, CZ = 32, 8, 8          # the kernels' node tile and planes per block
S3, S2 = T3 + 1, T2 + 1
SLOTS = S3 * S2


def walsh2(u00, u01, u10, u11):
    """(sum, sum s3 u, sum s2 u, sum s2 s3 u) of one node plane's corners"""
    s0, d0, s1, d1 = u00 + u01, u01 - u00, u10 + u11, u11 - u10
    return np.array([s0 + s1, d0 + d1, s1 - s0, d1 - d0])


def element_forces(L, H, physics, lam_or_kappa, mu, h):
    """Corner forces (a1 = 0, a1 = 1) x [a2 * 2 + a3] x component from the plane Walsh sums
    L, H (component x 4) of the lower and upper node planes."""
    e, k3, k2, k23 = 0, 1, 2, 3
    c1, c2, c3 = H[:, e] - L[:, e], L[:, k2] + H[:, k2], L[:, k3] + H[:, k3]
    c12, c13, c23, c123 = H[:, k2] - L[:, k2], H[:, k3] - L[:, k3], L[:, k23] + H[:, k23], H[:, k23] - L[:, k23]
    if physics == 1:
        k = h * lam_or_kappa
        G1, G2, G3 = k / 16 * c1, k / 16 * c2, k / 16 * c3
        G12, G13, G23, G123 = k / 24 * c12, k / 24 * c13, k / 24 * c23, k / 48 * c123
    else:
        lam = lam_or_kappa
        A1, b1, a2, b2 = h * mu / 8, h * lam / 16, h * mu / 48, h * lam / 48
        A2, g3 = h * (3 * mu + lam) / 48, h * (4 * mu + lam) / 144
        G1, G2, G3, G12, G13, G23 = (np.zeros(3) for _ in range(6))
        t0 = b1 * (c1[0] + c2[1] + c3[2])
        G1[0], G2[1], G3[2] = A1 * c1[0] + t0, A1 * c2[1] + t0, A1 * c3[2] + t0
        s01, s02, s12 = A1 / 2 * (c2[0] + c1[1]), A1 / 2 * (c3[0] + c1[2]), A1 / 2 * (c3[1] + c2[2])
        G2[0] = G1[1] = s01
        G3[0] = G1[2] = s02
        G3[1] = G2[2] = s12
        G12[0], G12[1], G12[2] = A2 * c12[0] + b2 * c23[2], A2 * c12[1] + b2 * c13[2], a2 * (2 * c12[2] + c23[0] + c13[1])
        G13[0], G13[2], G13[1] = A2 * c13[0] + b2 * c23[1], A2 * c13[2] + b2 * c12[1], a2 * (2 * c13[1] + c23[0] + c12[2])
        G23[1], G23[2], G23[0] = A2 * c23[1] + b2 * c13[0], A2 * c23[2] + b2 * c12[0], a2 * (2 * c23[0] + c13[1] + c12[2])
        G123 = g3 * c123
    E = [-G2 - (G3 - G23), -G2 + (G3 - G23), G2 - (G3 + G23), G2 + (G3 + G23)]
    F = [(G1 - G12) - (G13 - G123), (G1 - G12) + (G13 - G123), (G1 + G12) - (G13 + G123), (G1 + G12) + (G13 + G123)]
    return np.array([E[c] - F[c] for c in range(4)]), np.array([E[c] + F[c] for c in range(4)])


@pytest.mark.parametrize("physics,prop", [(3, (1.0, 0.3)), (3, (10.0, 0.2)), (3, (3.0, -0.5)), (1, 2.5)])
def test_walsh_element_force_equals_gauss_element_matrix(physics, prop):
    h = 0.37
    c = 1 if physics == 1 else 3
    Ke = fem.element_stiffness(physics, fem.material_matrix(physics, prop), h)
    lam, mu = (prop, 0.0) if physics == 1 else fem.lame(*prop)
    rng = np.random.default_rng(7)
    for _ in range(5):
        u = rng.standard_normal((2, 2, 2, c))            # [a1][a2][a3][component]
        ref = (Ke @ u.reshape(-1)).reshape(2, 2, 2, c)
        L = np.stack([walsh2(u[0, 0, 0, i], u[0, 0, 1, i], u[0, 1, 0, i], u[0, 1, 1, i]) for i in range(c)])
        H = np.stack([walsh2(u[1, 0, 0, i], u[1, 0, 1, i], u[1, 1, 0, i], u[1, 1, 1, i]) for i in range(c)])
        flo, fhi = element_forces(L, H, physics, lam, mu, h)
        f = np.stack([flo.reshape(2, 2, c), fhi.reshape(2, 2, c)])
        assert np.max(np.abs(f - ref)) <= 1e-14 * np.max(np.abs(ref))


def _tiled_Kd(shape, phase, lamu, d, physics, h):
    """The kernels' tiling restated on the host; returns p and the per-node write counts."""
    c = 1 if physics == 1 else 3
    n1, n2, n3 = shape
    n, S = n1 * n2 * n3, n2 * n3
    p = np.full((c, n), np.nan)
    writes = np.zeros(n, int)
    nt3, nt2, nt1 = -(-n3 // T3), -(-n2 // T2), -(-n1 // CZ)
    for tile in range(nt3 * nt2 * nt1):
        b3, rest = tile % nt3, tile // nt3
        b2, b1 = rest % nt2, rest // nt2
        t3, t2, z0 = b3 * T3, b2 * T2, b1 * CZ
        zend = min(z0 + CZ, n1)
        offs = []
        for tid in range(SLOTS):
            s2, s3 = divmod(tid, S3)
            e2, e3 = (t2 - 1 + s2) % n2, (t3 - 1 + s3) % n3
            e2p, e3p = (e2 + 1) % n2, (e3 + 1) % n3
            offs.append((e2 * n3 + e3, e2 * n3 + e3p, e2p * n3 + e3, e2p * n3 + e3p))

        def plane(z, o):
            idx = [z * S + x for x in o]
            assert all(0 <= q < n for q in idx)
            return np.stack([walsh2(*[d[i, q] for q in idx]) for i in range(c)])

        def forces(z, tid, L, H):
            lam, mu = lamu[phase[z * S + offs[tid][0]]]
            return element_forces(L, H, physics, lam, mu, h)

        zm = z0 - 1 if z0 else n1 - 1
        Hs, carry = [], []
        for tid in range(SLOTS):
            L, H = plane(zm, offs[tid]), plane(z0, offs[tid])
            Hs.append(H)
            carry.append(forces(zm, tid, L, H)[1])
        for z in range(z0, zend):
            buf = np.zeros((c, 4, SLOTS))
            for tid in range(SLOTS):
                L, H = Hs[tid], plane((z + 1) % n1, offs[tid])
                Hs[tid] = H
                flo, fhi = forces(z, tid, L, H)
                buf[:, :, tid] = (flo + carry[tid]).T
                carry[tid] = fhi
            for tid in range(T3 * T2):
                r2, r3 = tid >> 5, tid & 31
                if not (t2 + r2 < n2 and t3 + r3 < n3):
                    continue
                sA, sB = (r2 + 1) * S3 + r3 + 1, r2 * S3 + r3
                q = z * S + (t2 + r2) * n3 + t3 + r3
                flat = buf.reshape(c, -1)
                p[:, q] = flat[:, sA] + flat[:, SLOTS + sA - 1] + flat[:, 2 * SLOTS + sB + 1] + flat[:, 3 * SLOTS + sB]
                writes[q] += 1
    return p, writes


@pytest.mark.parametrize("physics,shape", [(3, (3, 4, 5)), (3, (2, 9, 34)), (1, (10, 10, 33)), (1, (1, 3, 2))])
def test_tiled_element_scheme_equals_assembled_K(physics, shape):
    c = 1 if physics == 1 else 3
    props = [(1.0, 0.3), (10.0, 0.2)] if physics == 3 else [1.0, 7.0]
    phase = random_phase(shape, 2, seed=3).reshape(-1)
    lamu = [fem.lame(*pr) for pr in props] if physics == 3 else [(k, 0.0) for k in props]
    d = random_field((c,) + shape, seed=4).reshape(c, -1)
    h = 1.0 / shape[0]
    p, writes = _tiled_Kd(shape, phase, lamu, d, physics, h)
    assert np.all(writes == 1)
    K = fem.assemble_K(phase.reshape(shape), np.array(props, dtype=float), physics)
    ref = fem.to_soa(K @ fem.from_soa(d.reshape((c,) + shape)), c, shape).reshape(c, -1)
    assert np.max(np.abs(p - ref)) <= 1e-13 * np.max(np.abs(ref))
