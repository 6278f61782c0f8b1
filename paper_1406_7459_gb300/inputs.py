"""Seeded synthetic inputs shared by the GPU path's tests/bench and the oracle.

This module holds only input generation (random numbers and workload
constants); none of the solver's arithmetic.  Every generator returns float32
arrays of shape (3, nz, ny, nx) -- three SoA planes, x fastest -- so that the
GPU path and the FP64 oracle receive the same bytes (the oracle widens them).

The paper's own workload, muMAG standard problem 3 (Sec. 4), is not
reproduced; these synthetic states stand in for it.
"""
import numpy as np

GAMMA0 = 2.211e5      # m/(A s), gyromagnetic ratio times mu0


def random_unit_m(grid, Ms, seed):
    """Gaussian triples from PCG64(seed), normalised, scaled by Ms."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((3, nz, ny, nx))
    v /= np.sqrt(np.sum(v * v, axis=0, keepdims=True))
    return (Ms * v).astype(np.float32)


def uniform_m(grid, Ms, direction=(1.0, 0.0, 0.0)):
    nx, ny, nz = grid
    d = np.asarray(direction, np.float64)
    d = d / np.sqrt(np.sum(d * d))
    out = np.empty((3, nz, ny, nx), np.float32)
    for a in range(3):
        out[a] = Ms * d[a]
    return out


def perturbed_m(grid, Ms, seed, amplitude=0.1, direction=(1.0, 0.0, 0.0)):
    """Uniform direction plus a seeded Gaussian perturbation, renormalised."""
    nx, ny, nz = grid
    rng = np.random.default_rng(seed)
    d = np.asarray(direction, np.float64).reshape(3, 1, 1, 1)
    v = d + amplitude * rng.standard_normal((3, nz, ny, nx))
    v /= np.sqrt(np.sum(v * v, axis=0, keepdims=True))
    return (Ms * v).astype(np.float32)


def field_at_angle(magnitude, degrees):
    t = np.deg2rad(degrees)
    return (magnitude * np.cos(t), magnitude * np.sin(t), 0.0)


# Workload recipes (material in SI units).  "thin_film_32" is the small
# random-start case; "film_sweep" is the size sweep whose 256x256x4 member is
# the benchmark workload; "precision" is the long-run precision study.
THIN_FILM_32 = dict(grid=(32, 32, 1), cell=(5e-9, 5e-9, 3e-9), Ms=8.6e5,
                    A=1.3e-11, Ku=0.0, alpha=0.5, gamma=GAMMA0,
                    H_ext=(0.0, 0.0, 0.0), dt=1e-13, steps=1000, seed=1)

FILM_SWEEP_GRIDS = ((64, 64, 4), (128, 128, 4), (256, 256, 4), (512, 512, 8),
                    (200, 60, 3))
FILM_SWEEP = dict(cell=(4e-9, 4e-9, 4e-9), Ms=8.6e5, A=1.3e-11, Ku=5e2,
                  alpha=0.02, gamma=GAMMA0, H_ext=field_at_angle(2.5e4, 170.0),
                  dt=5e-14, start=(1.0, 0.0, 0.0))

PRECISION_GRIDS = ((1024, 1024, 1), (256, 256, 64))
PRECISION = dict(cell=(2.5e-9, 2.5e-9, 2.5e-9), Ms=8.6e5, A=1.3e-11, Ku=0.0,
                 alpha=0.5, gamma=GAMMA0, H_ext=(0.0, 0.0, 0.0), dt=5e-14,
                 steps=10000, seed=2, amplitude=0.1)

# N x N x N cube relaxation, a synthetic stand-in for the paper's Table 1
# workload (muMAG standard problem 3 is not reproduced): 4 nm cubic cells,
# the size-sweep material, strong damping, seeded random start, no field.
CUBE_SIZES = (8, 16, 32, 64, 128)
CUBE = dict(cell=(4e-9, 4e-9, 4e-9), Ms=8.6e5, A=1.3e-11, Ku=5e2, alpha=0.5, gamma=GAMMA0,
            H_ext=(0.0, 0.0, 0.0), dt=5e-14, seed=5)


def batch_samples(n, seed=3, nx=(16, 256), ny=(16, 64), nz=(1, 2)):
    """Independent samples of uneven size: nx ~ U{16..256}, ny ~ U{16..64},
    nz ~ U{1, 2}, Ku ~ U[0, 1e4] J/m^3, |H_ext| ~ U[0, 5e4] A/m in a
    direction uniform on the sphere, alpha ~ U[0.01, 0.5]; the thin-film
    cell and material otherwise.  Returns a list of dicts with a seeded
    random start M (float32, (3, nz, ny, nx))."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        g = (int(rng.integers(nx[0], nx[1] + 1)), int(rng.integers(ny[0], ny[1] + 1)),
             int(rng.integers(nz[0], nz[1] + 1)))
        d = rng.standard_normal(3)
        d /= np.sqrt(np.sum(d * d))
        h = rng.uniform(0.0, 5e4) * d
        out.append(dict(grid=g, cell=(5e-9, 5e-9, 3e-9), Ms=8.6e5, A=1.3e-11,
                        Ku=float(rng.uniform(0.0, 1e4)), alpha=float(rng.uniform(0.01, 0.5)),
                        gamma=GAMMA0, H_ext=tuple(float(v) for v in h),
                        M=random_unit_m(g, 8.6e5, seed * 100003 + s)))
    return out
