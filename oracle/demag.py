"""Demagnetising field, FP64 (test infrastructure only).

Two independent evaluations of Eq. (11)/(12):

* ``demag_brute``  -- the plain O(N^2) double sum over source and observation
  cells, Eq. (12) for each component (H_a = sum_b K_ab * M_b).
* ``demag_fft``    -- the paper's method: zero-pad M to L_a >= 2 n_a - 1 per
  axis (Sec. 2 steps (1)-(2): the paper takes L_a = 2 n_a), place K in
  cyclic ("wrap") order with zeros in the unused slots, forward FFT of M and
  K (Eq. (8)/(14)), member-wise 3x3 product (Eq. (9)/(13)/(15)), inverse FFT
  (Eq. (10)/(16)) and keep the first n_a outputs on each axis ("discard the
  latter half", Sec. 2 step (5)).

Readings: forward transform unnormalised, inverse divided by Lx*Ly*Lz
(numpy's convention); K = -N with N from ``oracle.tensor``.

``set_workers(n)`` lets ``demag_fft`` use n host threads (for timing the
oracle on all cores): the transforms then come from ``scipy.fft`` (the same
pocketfft algorithm numpy uses) with ``workers=n`` and the member-wise
product runs on n threads over slabs of the padded z axis.  The default is
one thread and numpy's FFT.
"""
import concurrent.futures

import numpy as np

from .tensor import COMPONENTS, demag_tensor, tensor_full_offsets

_PAIR = {("x", "x"): 0, ("x", "y"): 1, ("x", "z"): 2, ("y", "y"): 3,
         ("y", "z"): 4, ("z", "z"): 5}


def _comp(a, b):
    """Index into the 6-component order of the symmetric pair (a, b)."""
    axes = "xyz"
    a, b = sorted((axes[a], axes[b]))
    return _PAIR[(a, b)]


_WORKERS = 1
_POOL = None


def set_workers(n):
    """Host threads for demag_fft (1 = numpy's single-threaded FFT)."""
    global _WORKERS, _POOL
    n = max(1, int(n))
    if n != _WORKERS and _POOL is not None:
        _POOL.shutdown()
        _POOL = None
    _WORKERS = n
    if n > 1:
        _POOL = concurrent.futures.ThreadPoolExecutor(max_workers=n)


def get_workers():
    return _WORKERS


def default_lengths(grid):
    """Paper's padded lengths: 2 n_a per axis (Sec. 2, step (1))."""
    return tuple(2 * n for n in grid)


def wrap_pad_kernel(octant, L):
    """K = -N in cyclic layout on an Lz x Ly x Lx box (Sec. 2 step (2)):
    slot p holds offset p for p < n, offset p - L for p > L - n, and 0
    otherwise.  Returns (6, Lz, Ly, Lx)."""
    _, nz, ny, nx = octant.shape
    Lx, Ly, Lz = L
    if Lx < 2 * nx - 1 or Ly < 2 * ny - 1 or Lz < 2 * nz - 1:
        raise ValueError("padded length must be >= 2n-1 on every axis")
    full = tensor_full_offsets(octant)      # offsets -(n-1)..(n-1)
    out = np.zeros((6, Lz, Ly, Lx))

    def slots(n, Lp):
        off = np.arange(-(n - 1), n)
        return np.mod(off, Lp)
    sz, sy, sx = slots(nz, Lz), slots(ny, Ly), slots(nx, Lx)
    out[:, sz[:, None, None], sy[None, :, None], sx[None, None, :]] = -full
    return out


def kernel_spectrum(octant, L):
    """Half-spectrum of the wrap-padded K (Eq. (8) for K; done once,
    Sec. 3): complex (6, Lz, Ly, Lx//2 + 1)."""
    Kp = wrap_pad_kernel(octant, L)
    return np.fft.rfftn(Kp, axes=(1, 2, 3))


def demag_fft(M, Kt, L):
    """H_demag of M (3, nz, ny, nx) from the precomputed half-spectrum Kt."""
    _, nz, ny, nx = M.shape
    Lx, Ly, Lz = L
    Mp = np.zeros((3, Lz, Ly, Lx))
    Mp[:, :nz, :ny, :nx] = M                                  # step (1)
    if _WORKERS == 1:
        Mt = np.fft.rfftn(Mp, axes=(1, 2, 3))                  # Eq. (14)
    else:
        import scipy.fft
        Mt = scipy.fft.rfftn(Mp, axes=(1, 2, 3), workers=_WORKERS)
    Ht = np.empty_like(Mt)

    def product(z0, z1):                                       # Eq. (15)
        for a in range(3):
            Ht[a, z0:z1] = sum(Kt[_comp(a, b), z0:z1] * Mt[b, z0:z1] for b in range(3))
    if _WORKERS == 1 or Lz < 2:
        product(0, Lz)
    else:
        cuts = np.linspace(0, Lz, min(_WORKERS, Lz) + 1).astype(int)
        list(_POOL.map(lambda i: product(cuts[i], cuts[i + 1]), range(len(cuts) - 1)))
    if _WORKERS == 1:
        H = np.fft.irfftn(Ht, s=(Lz, Ly, Lx), axes=(1, 2, 3))  # Eq. (16)
    else:
        H = scipy.fft.irfftn(Ht, s=(Lz, Ly, Lx), axes=(1, 2, 3), workers=_WORKERS)
    return H[:, :nz, :ny, :nx]                                 # discard


def demag_brute(M, octant):
    """Eq. (12) summed directly: H_a(i) = sum_l sum_b K_ab(i - l) M_b(l),
    K = -N, over every pair of cells.  O(N^2); tiny grids only."""
    _, nz, ny, nx = M.shape
    K = -tensor_full_offsets(octant)
    H = np.zeros_like(M, dtype=np.float64)
    for oz in range(-(nz - 1), nz):
        for oy in range(-(ny - 1), ny):
            for ox in range(-(nx - 1), nx):
                # observation cells i with source l = i - o inside the grid
                iz = slice(max(oz, 0), nz + min(oz, 0))
                iy = slice(max(oy, 0), ny + min(oy, 0))
                ix = slice(max(ox, 0), nx + min(ox, 0))
                lz = slice(max(-oz, 0), nz + min(-oz, 0))
                ly = slice(max(-oy, 0), ny + min(-oy, 0))
                lx = slice(max(-ox, 0), nx + min(-ox, 0))
                kk = K[:, oz + nz - 1, oy + ny - 1, ox + nx - 1]
                for a in range(3):
                    for b in range(3):
                        H[a, iz, iy, ix] += kk[_comp(a, b)] * M[b, lz, ly, lx]
    return H


def demag_at_cells(M, cell, cells):
    """H_demag at selected observation cells [(i, j, k), ...] by the direct
    sum of Eq. (12), with the tensor evaluated afresh at every offset (no FFT,
    no octant table).  Returns (len(cells), 3)."""
    _, nz, ny, nx = M.shape
    dx, dy, dz = cell
    lk, lj, li = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    out = np.zeros((len(cells), 3))
    for s, (i, j, k) in enumerate(cells):
        N = demag_tensor((i - li) * dx, (j - lj) * dy, (k - lk) * dz, cell)
        for a in range(3):
            for b in range(3):
                name = COMPONENTS[_comp(a, b)]
                out[s, a] -= np.sum(N[name] * M[b])
    return out
