"""The tiling of the TMA-staged thermal K d (k_ku_tma.cu) restated on the host, before any GPU
run: block -> (load, row tile, plane chunk), the node-plane and phase-plane rings with their
wrapped halo rows, the thread -> (row, 4 columns) map with the axis-3 neighbours taken from the
neighbouring thread of the row (periodic within a warp segment, from shared memory at the warp
edges of rows wider than a warp), the register window along i1 and the stencil with the pair
sums of the kernel.  Checks: every node written exactly once, every buffer index in range, the
TMA destinations 128-byte aligned, and the result equal to the assembled K of the oracle."""
import numpy as np
import pytest

from oracle import fem
from synth import random_field, random_phase

# the kernel's constants: nodes per thread along i3, node-plane and phase-plane ring depths
NV, DS, PS = 4, 4, 3


def supported(shape, rows):
    """Rows of the tile if the kernel takes this (grid, rows), else None (ku_tma_supported)."""
    n1, n2, n3 = shape
    if n3 % 32 or n3 > 256:
        return None
    threads = rows * (n3 // NV)
    if threads % 32 or not 64 <= threads <= 512:
        return None
    if n2 % rows or (rows * n3) % 128:
        return None
    return rows


def smem_layout(ty, n3):
    dslot = (ty + 2) * n3 * 4
    kslot = (ty + 1) * n3 * 4
    pslot = ((ty + 1) * n3 + 127) // 128 * 128
    return dslot, kslot, pslot


def emulate(shape, rows, planes, d, phase, kappa):
    """p = K d as the kernel computes it (FP64 here; h = 1 / N1, scaled conductivities h/12 k)."""
    n1, n2, n3 = shape
    ty_rows = supported(shape, rows)
    tpr = n3 // NV
    threads = ty_rows * tpr
    h12 = (1.0 / n1) / 12.0
    mt = kappa * h12
    dslot, kslot, pslot = smem_layout(ty_rows, n3)
    # TMA destinations (byte offsets from the 128-aligned base) must be 128-byte aligned
    for s in range(DS):
        for row in (0, ty_rows, ty_rows + 1):
            assert (s * dslot + row * n3 * 4) % 128 == 0
    kbase = DS * dslot
    pbase = kbase + 2 * kslot
    assert kbase % 128 == 0 and pbase % 128 == 0
    for s in range(PS):
        for row in (0, ty_rows):
            assert (pbase + s * pslot + row * n3) % 128 == 0
    p = np.full(d.shape, np.nan)
    writes = np.zeros(d.shape, dtype=np.int64)
    ntile2 = n2 // ty_rows
    nz = (n1 + planes - 1) // planes
    tid = np.arange(threads)
    t_row = tid // tpr
    x0 = (tid % tpr) * NV
    xr_ = tid % tpr
    # the neighbouring threads of the row (periodic); the shuffle reads that lane of the own
    # warp, the kernel replaces it by a shared-memory read where the neighbour is in another warp
    tl = np.where(xr_ == 0, tid + tpr - 1, tid - 1)
    tr = np.where(xr_ == tpr - 1, tid - tpr + 1, tid + 1)
    src_l = (tid & ~31) | (tl & 31)
    src_r = (tid & ~31) | (tr & 31)
    fix_l = (tl >> 5) != (tid >> 5)
    fix_r = (tr >> 5) != (tid >> 5)
    xl = np.where(x0 == 0, n3, x0) - 1
    xr = np.where(x0 + NV == n3, 0, x0 + NV)
    rm = np.where(t_row == 0, ty_rows, t_row - 1)
    rc = t_row
    rp = np.where(t_row + 1 == ty_rows, ty_rows + 1, t_row + 1)
    assert np.all(src_l < threads) and np.all(src_r < threads)

    def node_plane(q, i2_0):
        # the ring buffer of node plane q: rows 0..TY-1 tile, TY = i2_0 - 1, TY + 1 = i2_0 + TY
        rows = list(range(i2_0, i2_0 + ty_rows)) + [(i2_0 - 1) % n2, (i2_0 + ty_rows) % n2]
        return d[q % n1][rows]

    def phase_plane(e, i2_0):
        rows = list(range(i2_0, i2_0 + ty_rows)) + [(i2_0 - 1) % n2]
        return mt[phase[e % n1][rows]]

    def row_vals(buf, r):
        # v[0] = x0 - 1, v[1..4] = x0..x0+3, v[5] = x0 + 4, gathered as the kernel does
        q = np.stack([buf[r, x0 + k] for k in range(NV)], axis=1)     # [threads, 4]
        left = q[src_l, NV - 1]
        right = q[src_r, 0]
        left = np.where(fix_l, buf[r, xl], left)
        right = np.where(fix_r, buf[r, xr], right)
        return np.concatenate([left[:, None], q, right[:, None]], axis=1)

    for blk in range(1 * ntile2 * nz):
        tile2, zc = blk % ntile2, blk // ntile2
        i2_0 = tile2 * ty_rows
        z0 = zc * planes
        nsteps = min(planes, n1 - z0)
        bufs = [node_plane(z0 - 1, i2_0), node_plane(z0, i2_0)]
        assert bufs[0].shape == (ty_rows + 2, n3)
        D_m = [row_vals(bufs[0], r) for r in (rm, rc, rp)]
        D_c = [row_vals(bufs[1], r) for r in (rm, rc, rp)]
        kb = phase_plane(z0 - 1, i2_0)
        K_m = [row_vals(kb, rc)[:, :NV + 1], row_vals(kb, rm)[:, :NV + 1]]
        for j in range(nsteps):
            z = z0 + j
            bn = node_plane(z + 1, i2_0)
            D_n = [row_vals(bn, r) for r in (rm, rc, rp)]
            kc = phase_plane(z, i2_0)
            K_c = [row_vals(kc, rc)[:, :NV + 1], row_vals(kc, rm)[:, :NV + 1]]
            Q0 = K_c[0] + K_c[1]
            Q1 = K_m[0] + K_m[1]
            E0 = K_c[0] + K_m[0]
            E1 = K_c[1] + K_m[1]
            out = np.zeros((threads, NV))
            for i in range(NV):
                sk = (Q0[:, i] + Q0[:, i + 1]) + (Q1[:, i] + Q1[:, i + 1])
                acc = 4 * sk * D_c[1][:, i + 1]
                acc -= E1[:, i] * D_c[0][:, i] + E1[:, i + 1] * D_c[0][:, i + 2]
                acc -= E0[:, i] * D_c[2][:, i] + E0[:, i + 1] * D_c[2][:, i + 2]
                acc -= Q0[:, i] * D_n[1][:, i] + Q0[:, i + 1] * D_n[1][:, i + 2]
                acc -= Q1[:, i] * D_m[1][:, i] + Q1[:, i + 1] * D_m[1][:, i + 2]
                acc -= (K_c[1][:, i] + K_c[1][:, i + 1]) * D_n[0][:, i + 1]
                acc -= (K_c[0][:, i] + K_c[0][:, i + 1]) * D_n[2][:, i + 1]
                acc -= (K_m[1][:, i] + K_m[1][:, i + 1]) * D_m[0][:, i + 1]
                acc -= (K_m[0][:, i] + K_m[0][:, i + 1]) * D_m[2][:, i + 1]
                acc -= K_c[1][:, i] * D_n[0][:, i] + K_c[1][:, i + 1] * D_n[0][:, i + 2]
                acc -= K_c[0][:, i] * D_n[2][:, i] + K_c[0][:, i + 1] * D_n[2][:, i + 2]
                acc -= K_m[1][:, i] * D_m[0][:, i] + K_m[1][:, i + 1] * D_m[0][:, i + 2]
                acc -= K_m[0][:, i] * D_m[2][:, i] + K_m[0][:, i + 1] * D_m[2][:, i + 2]
                out[:, i] = acc
            i2 = i2_0 + t_row
            assert np.all(i2 < n2) and z < n1
            for i in range(NV):
                p[z, i2, x0 + i] = out[:, i]
                np.add.at(writes, (np.full(threads, z), i2, x0 + i), 1)
            D_m, D_c = D_c, D_n
            K_m = K_c
    return p, writes


# (grid, rows TY, planes per block): one and several row tiles, ragged plane chunks, two-node
# axes, rows in one warp (N3 <= 128), across warps (N3 = 160, 192, 256)
CASES = [((2, 16, 32), 16, 6), ((5, 16, 64), 16, 6), ((13, 16, 64), 8, 6), ((7, 8, 256), 4, 12),
         ((9, 8, 256), 8, 12), ((6, 32, 128), 8, 24), ((3, 4, 256), 2, 6), ((5, 8, 192), 4, 12),
         ((4, 12, 96), 4, 6), ((3, 8, 160), 4, 6)]


@pytest.mark.parametrize("shape,rows,planes", CASES)
def test_tma_tiling_writes_each_node_once_and_equals_assembled_K(shape, rows, planes):
    assert supported(shape, rows) is not None
    phase = random_phase(shape, 3, seed=sum(shape))
    kappa = np.array([1.0, 6.0, 0.4])
    d = random_field(shape, seed=3)
    p, writes = emulate(shape, rows, planes, d, phase, kappa)
    assert np.all(writes == 1)
    K = fem.assemble_K(phase, kappa, 1)
    p_ref = (K @ d.ravel()).reshape(shape)
    assert np.max(np.abs(p - p_ref)) <= 1e-13 * np.max(np.abs(p_ref))
