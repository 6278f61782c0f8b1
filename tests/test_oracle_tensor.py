"""Pins of the FP64 demag tensor (oracle/tensor.py) against facts that do
not come from the oracle itself: Aharoni's closed-form prism factor, the
trace identities, the point-dipole limit, and a 50-digit evaluation."""
import numpy as np
import pytest

from oracle import tensor as T

CELLS = [(1.0, 1.0, 1.0), (5e-9, 5e-9, 3e-9), (1.0, 2.0, 3.0),
         (4e-9, 4e-9, 4e-9), (2.0, 0.3, 7.0)]


@pytest.mark.parametrize("cell", CELLS)
def test_self_term_equals_aharoni_prism_factor(cell):
    dx, dy, dz = cell
    N = T.newell_tensor(0.0, 0.0, 0.0, cell)
    a, b, c = dx / 2, dy / 2, dz / 2
    Dx = T.aharoni_factor(b, c, a)
    Dy = T.aharoni_factor(c, a, b)
    Dz = T.aharoni_factor(a, b, c)
    assert abs(N["xx"] - Dx) < 1e-12
    assert abs(N["yy"] - Dy) < 1e-12
    assert abs(N["zz"] - Dz) < 1e-12
    assert abs(N["xx"] + N["yy"] + N["zz"] - 1.0) < 1e-12
    for off in ("xy", "xz", "yz"):
        assert abs(N[off]) < 1e-14


def test_cube_self_factor_is_one_third():
    N = T.demag_tensor(0.0, 0.0, 0.0, (3e-9, 3e-9, 3e-9))
    for d in ("xx", "yy", "zz"):
        assert abs(N[d] - 1.0 / 3.0) < 1e-14


def test_aharoni_independent_limits():
    # thin plate -> D_z -> 1; long square needle along z -> D_z ~ 1/aspect
    # and D_x = D_y -> 1/2
    assert T.aharoni_factor(1e4, 1e4, 1.0) > 0.999
    for aspect in (10.0, 100.0, 1000.0):
        dz = T.aharoni_factor(1.0, 1.0, aspect)
        assert 0.3 / aspect < dz < 0.6 / aspect
        assert abs(T.aharoni_factor(1.0, aspect, 1.0) - 0.5) < 0.6 / aspect


@pytest.mark.parametrize("cell", CELLS[:3])
def test_offsite_trace_vanishes(cell):
    rng = np.random.default_rng(0)
    d = np.array(cell)
    offs = rng.integers(-7, 8, size=(200, 3))
    offs = offs[np.any(offs != 0, axis=1)]
    X, Y, Z = (offs * d).T
    N = T.demag_tensor(X, Y, Z, cell)
    scale = max(np.max(np.abs(N[c])) for c in T.COMPONENTS)
    tr = N["xx"] + N["yy"] + N["zz"]
    assert np.max(np.abs(tr)) < 1e-9 * scale


def test_parity_of_every_component():
    cell = (5e-9, 4e-9, 3e-9)
    grid = (5, 4, 3)
    octant = T.tensor_octant(grid, cell)
    full = T.tensor_full_offsets(octant)
    nx, ny, nz = grid
    for ox in range(-(nx - 1), nx):
        for oy in range(-(ny - 1), ny):
            for oz in range(-(nz - 1), nz):
                direct = T.demag_tensor(ox * cell[0], oy * cell[1],
                                        oz * cell[2], cell)
                for c, name in enumerate(T.COMPONENTS):
                    got = full[c, oz + nz - 1, oy + ny - 1, ox + nx - 1]
                    assert abs(got - direct[name]) <= 1e-12   # max |N| ~ 0.45


@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (5.0, 5.0, 3.0)])
def test_newell_and_quadrature_agree_at_near_boundary(cell):
    rng = np.random.default_rng(1)
    dmax = max(cell)
    dirs = rng.standard_normal((40, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    X, Y, Z = (dirs * T.NEAR_CELLS * dmax).T
    ex = T.newell_tensor(X, Y, Z, cell)
    q = T.quadrature_tensor(X, Y, Z, cell, T.QUAD_TIERS[0][1])
    scale = np.max(np.abs(ex["xx"]))
    for c in T.COMPONENTS:
        assert np.max(np.abs(q[c] - ex[c])) < 1e-9 * scale, c


@pytest.mark.parametrize("cell", [(1.0, 1.0, 1.0), (5.0, 5.0, 3.0)])
def test_quadrature_tiers_converged_at_their_lower_radius(cell):
    """Each tier's node count, at the smallest radius it serves, matches a
    12-node rule to 1e-10 relative (beyond 16 cells the closed form itself
    loses digits to cancellation, so the reference is a finer rule)."""
    rng = np.random.default_rng(2)
    dmax = max(cell)
    lower = T.NEAR_CELLS
    for upper, nq in T.QUAD_TIERS:
        dirs = rng.standard_normal((30, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        X, Y, Z = (dirs * lower * dmax).T
        ref = T.quadrature_tensor(X, Y, Z, cell, 12)
        q = T.quadrature_tensor(X, Y, Z, cell, nq)
        scale = np.max(np.abs(ref["xx"]))
        for c in T.COMPONENTS:
            assert np.max(np.abs(q[c] - ref[c])) < 1e-10 * scale, (lower, c)
        lower = upper


def test_far_field_tends_to_point_dipole_second_order():
    cell = (5e-9, 5e-9, 3e-9)
    V = np.prod(cell)
    u = np.array([0.6, -0.48, 0.64])
    errs = []
    for r in (40e-9, 80e-9, 160e-9, 320e-9):
        X, Y, Z = u * r
        N = T.demag_tensor(X, Y, Z, cell)
        rh = u / np.linalg.norm(u)
        D = V / (4 * np.pi * r ** 3) * (np.eye(3) - 3 * np.outer(rh, rh))
        got = np.array([[N["xx"], N["xy"], N["xz"]], [N["xy"], N["yy"], N["yz"]],
                        [N["xz"], N["yz"], N["zz"]]]).reshape(3, 3)
        errs.append(np.max(np.abs(got - D)) / np.max(np.abs(D)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert errs[-1] < 1e-3
    assert np.all(ratios > 3.5) and np.all(ratios < 4.5), (errs, ratios)


def test_tiered_tensor_matches_50_digit_newell():
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50

    def f(x, y, z):
        x2, y2, z2 = x * x, y * y, z * z
        R = mp.sqrt(x2 + y2 + z2)
        s = (2 * x2 - y2 - z2) * R / 6
        if x2 + z2 > 0:
            s += y * (z2 - x2) / 2 * mp.asinh(y / mp.sqrt(x2 + z2))
        if x2 + y2 > 0:
            s += z * (y2 - x2) / 2 * mp.asinh(z / mp.sqrt(x2 + y2))
        if x * R != 0:
            s -= x * y * z * mp.atan(y * z / (x * R))
        return s

    def g(x, y, z):
        x2, y2, z2 = x * x, y * y, z * z
        R = mp.sqrt(x2 + y2 + z2)
        s = -x * y * R / 3
        if x2 + y2 > 0:
            s += x * y * z * mp.asinh(z / mp.sqrt(x2 + y2))
        if y2 + z2 > 0:
            s += y / 6 * (3 * z2 - y2) * mp.asinh(x / mp.sqrt(y2 + z2))
        if x2 + z2 > 0:
            s += x / 6 * (3 * z2 - x2) * mp.asinh(y / mp.sqrt(x2 + z2))
        if z * R != 0:
            s -= z * z2 / 6 * mp.atan(x * y / (z * R))
        if y * R != 0:
            s -= z * y2 / 2 * mp.atan(x * z / (y * R))
        if x * R != 0:
            s -= z * x2 / 2 * mp.atan(y * z / (x * R))
        return s

    def stencil(fun, X, Y, Z, d):
        acc = mp.mpf(0)
        for ex in (-1, 0, 1):
            for ey in (-1, 0, 1):
                for ez in (-1, 0, 1):
                    w = ((2 if ex == 0 else -1) * (2 if ey == 0 else -1)
                         * (2 if ez == 0 else -1))
                    acc += w * fun(X + ex * d[0], Y + ey * d[1], Z + ez * d[2])
        return acc / (4 * mp.pi * d[0] * d[1] * d[2])

    cell = (5, 5, 3)          # integers: exact in both precisions
    d = [mp.mpf(c) for c in cell]
    for off in [(1, 0, 0), (3, 2, 1), (7, 3, 2), (9, 1, 0), (14, 5, 3),
                (40, 17, 3), (120, 33, 1)]:
        X, Y, Z = (mp.mpf(o * c) for o, c in zip(off, cell))
        ref = {"xx": stencil(f, X, Y, Z, d),
               "xy": stencil(g, X, Y, Z, d),
               "zz": stencil(lambda a, b, c: f(c, b, a), X, Y, Z, d)}
        got = T.demag_tensor(off[0] * 5.0, off[1] * 5.0, off[2] * 3.0,
                             (5.0, 5.0, 3.0))
        scale = max(abs(float(ref["xx"])), abs(float(ref["zz"])))
        for c in ref:
            assert abs(float(ref[c]) - float(got[c])) < 1e-9 * scale, (off, c)


@pytest.mark.parametrize("grid,cell", [((16, 8, 2), (5e-9, 5e-9, 3e-9)),
                                       ((24, 3, 5), (1.0, 2.0, 0.5))])
def test_whole_body_sum_equals_prism_factor(grid, cell):
    """(1/Ncells) sum_i sum_j N(r_i - r_j) is the demagnetising factor of the
    whole prism (uniform magnetisation), given in closed form by Aharoni."""
    nx, ny, nz = grid
    full = T.tensor_full_offsets(T.tensor_octant(grid, cell))
    cz = nz - np.abs(np.arange(-(nz - 1), nz))
    cy = ny - np.abs(np.arange(-(ny - 1), ny))
    cx = nx - np.abs(np.arange(-(nx - 1), nx))
    w = cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
    ncell = nx * ny * nz
    s = {name: np.sum(full[c] * w) / ncell for c, name in enumerate(T.COMPONENTS)}
    a, b, c = nx * cell[0] / 2, ny * cell[1] / 2, nz * cell[2] / 2
    assert abs(s["xx"] - T.aharoni_factor(b, c, a)) < 1e-9
    assert abs(s["yy"] - T.aharoni_factor(c, a, b)) < 1e-9
    assert abs(s["zz"] - T.aharoni_factor(a, b, c)) < 1e-9
    for off in ("xy", "xz", "yz"):
        assert abs(s[off]) < 1e-12
