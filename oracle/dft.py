"""Unitary discrete Fourier transform written out by its definition (oracle; tests only).

The UNO preconditioner uses a unitary transform T with T^{-1} = T^H (Sec. 5.2.1).  For the
Fourier transform on an ``N1 x N2 x N3`` grid with ``n = N1 N2 N3`` nodes:

    X(k) = n^{-1/2} sum_x x(x) exp(-2 pi i sum_a k_a x_a / N_a)

computed axis by axis (the multi-dimensional DFT is separable), each axis by a dense matrix
product with ``W[k, j] = exp(-2 pi i ((j k) mod N) / N)`` whose angle is reduced exactly in
integers.  Real fields are stored on the half grid ``k3 = 0 .. N3//2`` (the conjugate modes
of the last axis are implied, Sec. 3.2.2).
"""
from __future__ import annotations

import numpy as np


def dft_matrix(N: int, inverse: bool = False) -> np.ndarray:
    j = np.arange(N)
    m = np.outer(j, j) % N
    sign = 1.0 if inverse else -1.0
    return np.exp(sign * 2j * np.pi * m / N)


def _along(x: np.ndarray, W: np.ndarray, axis: int) -> np.ndarray:
    x = np.moveaxis(x, axis, -1)
    y = x @ W.T
    return np.moveaxis(y, -1, axis)


def fftn_u(x: np.ndarray) -> np.ndarray:
    """Unitary forward DFT over the last three axes."""
    y = np.asarray(x, dtype=np.complex128)
    n = 1
    for ax in (-3, -2, -1):
        N = y.shape[ax]
        y = _along(y, dft_matrix(N), ax)
        n *= N
    return y / np.sqrt(n)


def ifftn_u(X: np.ndarray) -> np.ndarray:
    """Unitary inverse DFT over the last three axes (the adjoint of ``fftn_u``)."""
    y = np.asarray(X, dtype=np.complex128)
    n = 1
    for ax in (-3, -2, -1):
        N = y.shape[ax]
        y = _along(y, dft_matrix(N, inverse=True), ax)
        n *= N
    return y / np.sqrt(n)


def rfftn_u(x: np.ndarray) -> np.ndarray:
    """Unitary DFT of a real field restricted to the half grid ``k3 <= N3//2``."""
    N3 = x.shape[-1]
    return fftn_u(x)[..., : N3 // 2 + 1]


def hermitian_extend(Xh: np.ndarray, N3: int) -> np.ndarray:
    """Full spectrum from the half grid using ``X(-k) = conj(X(k))``."""
    N1, N2 = Xh.shape[-3], Xh.shape[-2]
    full = np.zeros(Xh.shape[:-1] + (N3,), dtype=np.complex128)
    full[..., : N3 // 2 + 1] = Xh
    k1 = (-np.arange(N1)) % N1
    k2 = (-np.arange(N2)) % N2
    for k3 in range(N3 // 2 + 1, N3):
        src = Xh[..., :, :, N3 - k3]
        full[..., k3] = np.conj(src[..., k1, :][..., :, k2])
    return full


def irfftn_u(Xh: np.ndarray, N3: int, imag_tol: float = 1e-12) -> np.ndarray:
    """Inverse of ``rfftn_u``: Hermitian extension, inverse DFT, real part.

    Asserts that the imaginary part of the result is negligible (relative ``imag_tol``), i.e.
    that the half-grid data were consistent with a real field.
    """
    y = ifftn_u(hermitian_extend(Xh, N3))
    scale = max(1.0, float(np.max(np.abs(y.real))) if y.size else 1.0)
    if y.size and float(np.max(np.abs(y.imag))) > imag_tol * scale:
        raise AssertionError("inverse transform is not real: non-Hermitian half-grid data")
    return y.real.copy()


def half_multiplicity(shape) -> np.ndarray:
    """Number of full-grid modes each half-grid mode stands for: 1 on the self-conjugate planes
    ``k3 = 0`` and ``k3 = N3/2`` (N3 even), else 2.  Shape ``(N1, N2, N3//2+1)``."""
    N1, N2, N3 = shape
    w = np.full((N1, N2, N3 // 2 + 1), 2.0)
    w[:, :, 0] = 1.0
    if N3 % 2 == 0:
        w[:, :, N3 // 2] = 1.0
    return w
