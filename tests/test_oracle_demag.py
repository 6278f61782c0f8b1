"""Pins of the FP64 demag convolution (oracle/demag.py): the FFT method of
Sec. 2 (Eqs. (8)-(10), (13)) must reproduce the plain double sum of
Eq. (11)/(12) exactly (up to rounding) for any padded length L >= 2n - 1,
and a uniformly magnetised prism must feel Aharoni's mean field."""
import numpy as np
import pytest

from oracle import tensor as T
from oracle import demag as D
from paper_1406_7459_gb300 import inputs

GRIDS = [(1, 1, 1), (2, 3, 1), (5, 3, 2), (8, 8, 4), (7, 5, 3), (1, 6, 1)]
CELL = (5e-9, 4e-9, 3e-9)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("grid", GRIDS)
def test_fft_convolution_equals_brute_force(grid):
    M = inputs.random_unit_m(grid, 8.6e5, seed=7).astype(np.float64)
    octant = T.tensor_octant(grid, CELL)
    Hb = D.demag_brute(M, octant)
    for L in (D.default_lengths(grid),                       # paper: 2n
              tuple(max(2 * n - 1, 1) for n in grid),        # minimum
              tuple(2 * n + 3 for n in grid)):               # any larger
        Kt = D.kernel_spectrum(octant, L)
        Hf = D.demag_fft(M, Kt, L)
        assert _rel(Hf, Hb) < 1e-12, L


@pytest.mark.parametrize("grid", [(5, 3, 2), (8, 8, 4), (7, 5, 3)])
def test_threaded_fft_convolution_equals_brute_force(grid):
    """The multi-threaded demag (scipy transforms, tensor product on a
    thread pool), used to time the oracle on all host cores, is the same
    convolution: it must also equal the plain double sum."""
    M = inputs.random_unit_m(grid, 8.6e5, seed=8).astype(np.float64)
    octant = T.tensor_octant(grid, CELL)
    Hb = D.demag_brute(M, octant)
    L = D.default_lengths(grid)
    Kt = D.kernel_spectrum(octant, L)
    D.set_workers(3)
    try:
        Hf = D.demag_fft(M, Kt, L)
    finally:
        D.set_workers(1)
    assert D.get_workers() == 1
    assert _rel(Hf, Hb) < 1e-12


def test_too_short_padding_is_rejected():
    octant = T.tensor_octant((4, 4, 1), CELL)
    with pytest.raises(ValueError):
        D.wrap_pad_kernel(octant, (6, 8, 1))


def test_kernel_spectrum_is_real_and_symmetric():
    # parity of each component makes every K~ real (imag part ~ rounding)
    grid = (6, 5, 3)
    octant = T.tensor_octant(grid, CELL)
    Kt = D.kernel_spectrum(octant, D.default_lengths(grid))
    assert np.max(np.abs(Kt.imag)) < 1e-12 * np.max(np.abs(Kt.real))


def test_direct_sampling_matches_brute_force():
    grid = (6, 4, 3)
    M = inputs.random_unit_m(grid, 8.6e5, seed=3).astype(np.float64)
    Hb = D.demag_brute(M, T.tensor_octant(grid, CELL))
    cells = [(0, 0, 0), (5, 3, 2), (2, 1, 1), (4, 0, 2)]
    Hs = D.demag_at_cells(M, CELL, cells)
    for s, (i, j, k) in enumerate(cells):
        assert np.allclose(Hs[s], Hb[:, k, j, i], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("direction", [(1, 0, 0), (0, 1, 0), (0, 0, 1)])
def test_uniform_prism_mean_field_is_aharoni(direction):
    grid, cell = (12, 6, 3), (5e-9, 5e-9, 3e-9)
    Ms = 8.6e5
    M = inputs.uniform_m(grid, Ms, direction).astype(np.float64)
    L = D.default_lengths(grid)
    H = D.demag_fft(M, D.kernel_spectrum(T.tensor_octant(grid, cell), L), L)
    a, b, c = grid[0] * cell[0] / 2, grid[1] * cell[1] / 2, grid[2] * cell[2] / 2
    Dfac = {0: T.aharoni_factor(b, c, a), 1: T.aharoni_factor(c, a, b),
            2: T.aharoni_factor(a, b, c)}[int(np.argmax(direction))]
    axis = int(np.argmax(direction))
    assert abs(np.mean(H[axis]) / Ms + Dfac) < 1e-9
    # transverse components average to zero by symmetry
    for o in range(3):
        if o != axis:
            assert abs(np.mean(H[o])) < 1e-9 * Ms
