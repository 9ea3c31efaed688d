"""Helpers of the GPU tests: host <-> device layouts and oracle fixtures."""
import numpy as np


def soa_from_interleaved(u, c, shape):
    return u.reshape(tuple(shape) + (c,)).transpose(3, 0, 1, 2).copy()


def interleaved_from_soa(a):
    return np.ascontiguousarray(np.moveaxis(a, 0, -1)).ravel()


def rel(a, b):
    den = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / den)
