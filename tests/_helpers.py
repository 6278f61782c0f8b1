"""Shared helpers for the tests (not part of the product or the oracle)."""
import functools

import numpy as np

from oracle import tensor as T, demag as D


def padded_length(n):
    """The padded FFT length rule of the GPU plan, restated independently:
    1 for n = 1, 2n for a power of two, else the smallest 2^a 3^b 5^c >= 2n-1.
    Any L >= 2n-1 gives the same exact convolution."""
    if n == 1:
        return 1
    if n & (n - 1) == 0:
        return 2 * n

    def smooth(m):
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        return m == 1
    L = 2 * n - 1
    while not smooth(L):
        L += 1
    return L


@functools.lru_cache(maxsize=16)
def oracle_octant(grid, cell):
    return T.tensor_octant(grid, cell)


@functools.lru_cache(maxsize=16)
def oracle_spectrum(grid, cell, L=None):
    L = L or D.default_lengths(grid)
    return D.kernel_spectrum(oracle_octant(grid, cell), L), L


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
