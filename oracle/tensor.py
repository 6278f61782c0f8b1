"""Cell-averaged demagnetising tensor, FP64 (test infrastructure only).

The paper writes the demag field as the discrete convolution of M with a
tensor K that depends only on the offset between source and observation cell
(Sec. 2, Eq. (7) and Eqs. (11)-(12)) and defers the tensor's formula to its
ref. [11].  Reading used here: K = -N, where N is the cell-to-cell averaged
demagnetising tensor of two identical rectangular cells (Newell, Williams &
Dunlop 1993), so that H_demag(i) = sum_l K(l - i) M(l) = -sum_l N(i - l) M(l).
N is even under full inversion of the offset, so K(l - i) = K(i - l) and the
paper's form of Eq. (7) and the convolution form coincide.

Evaluation (a numerical reading, identical on the oracle and GPU sides):

* |R| <  8 d_max : Newell's closed form, the 27-point second difference of
                   the functions f and g (below).  FP64 cancellation grows
                   like (R/d)^6; at 8 cells it is ~1e-10 relative.
* |R| >= 8 d_max : the same average written as an integral,
                   N(R) = V * int T(R + u) prod_a tri_a(u_a) d^3u,
                   T(s) = (I - 3 s s^T/|s|^2) / (4 pi |s|^3),
                   tri_a(u) = (d_a - |u|)/d_a^2 on |u| <= d_a (the
                   autocorrelation of two cells), by Gauss-Legendre
                   quadrature on each half-axis: 5 nodes per half-axis for
                   8 <= |R|/d_max < 16, 4 nodes for 16..32, 3 beyond 32.
                   Quadrature error there is < 1e-10 relative.

d_max = max(dx, dy, dz).  Component order everywhere: xx, xy, xz, yy, yz, zz.
Parity: xx, yy, zz are even in every axis; xy is odd in x and y; xz in x and
z; yz in y and z.
"""
import numpy as np

MU0 = 4e-7 * np.pi          # vacuum permeability, exact SI value (reading)
COMPONENTS = ("xx", "xy", "xz", "yy", "yz", "zz")
# sign of each component under reflection of (x, y, z)
PARITY = {"xx": (1, 1, 1), "xy": (-1, -1, 1), "xz": (-1, 1, -1),
          "yy": (1, 1, 1), "yz": (1, -1, -1), "zz": (1, 1, 1)}
NEAR_CELLS = 8.0            # Newell closed form below this many d_max
# quadrature tiers: (upper radius in d_max, Gauss-Legendre nodes per half-axis)
QUAD_TIERS = ((16.0, 5), (32.0, 4), (np.inf, 3))


def _safe_div(num, den):
    den_ok = den != 0
    return np.where(den_ok, num / np.where(den_ok, den, 1.0), 0.0), den_ok


def newell_f(x, y, z):
    """Newell's f(x, y, z), whose 27-point second difference gives N_xx."""
    x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0
    q, ok = _safe_div(y, np.sqrt(x2 + z2))
    out = out + np.where(ok, 0.5 * y * (z2 - x2) * np.arcsinh(q), 0.0)
    q, ok = _safe_div(z, np.sqrt(x2 + y2))
    out = out + np.where(ok, 0.5 * z * (y2 - x2) * np.arcsinh(q), 0.0)
    q, ok = _safe_div(y * z, x * R)
    out = out + np.where(ok, -x * y * z * np.arctan(q), 0.0)
    return out


def newell_g(x, y, z):
    """Newell's g(x, y, z), whose 27-point second difference gives N_xy."""
    x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3.0
    q, ok = _safe_div(z, np.sqrt(x2 + y2))
    out = out + np.where(ok, x * y * z * np.arcsinh(q), 0.0)
    q, ok = _safe_div(x, np.sqrt(y2 + z2))
    out = out + np.where(ok, y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(q), 0.0)
    q, ok = _safe_div(y, np.sqrt(x2 + z2))
    out = out + np.where(ok, x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(q), 0.0)
    q, ok = _safe_div(x * y, z * R)
    out = out + np.where(ok, -z * z2 / 6.0 * np.arctan(q), 0.0)
    q, ok = _safe_div(x * z, y * R)
    out = out + np.where(ok, -z * y2 / 2.0 * np.arctan(q), 0.0)
    q, ok = _safe_div(y * z, x * R)
    out = out + np.where(ok, -z * x2 / 2.0 * np.arctan(q), 0.0)
    return out


def _second_difference(fun, X, Y, Z, dx, dy, dz):
    """(1/(4 pi V)) sum_e w(e) fun(X + ex dx, Y + ey dy, Z + ez dz), with
    w(e) = prod_axis (2 if e_axis == 0 else -1): Newell's combination."""
    acc = np.zeros(np.broadcast(X, Y, Z).shape)
    for ex in (-1, 0, 1):
        for ey in (-1, 0, 1):
            for ez in (-1, 0, 1):
                w = ((2 if ex == 0 else -1) * (2 if ey == 0 else -1)
                     * (2 if ez == 0 else -1))
                acc = acc + w * fun(X + ex * dx, Y + ey * dy, Z + ez * dz)
    return acc / (4.0 * np.pi * dx * dy * dz)


def newell_tensor(X, Y, Z, cell):
    """Closed-form N at offsets (X, Y, Z) in metres -> dict of 6 arrays.

    The diagonal terms permute f's arguments so that its first argument is
    the diagonal axis; the off-diagonal terms put the two mixed axes first
    in g."""
    dx, dy, dz = cell
    X = np.asarray(X, np.float64); Y = np.asarray(Y, np.float64)
    Z = np.asarray(Z, np.float64)
    sd = _second_difference
    return {
        "xx": sd(lambda a, b, c: newell_f(a, b, c), X, Y, Z, dx, dy, dz),
        "yy": sd(lambda a, b, c: newell_f(b, a, c), X, Y, Z, dx, dy, dz),
        "zz": sd(lambda a, b, c: newell_f(c, b, a), X, Y, Z, dx, dy, dz),
        "xy": sd(lambda a, b, c: newell_g(a, b, c), X, Y, Z, dx, dy, dz),
        "xz": sd(lambda a, b, c: newell_g(a, c, b), X, Y, Z, dx, dy, dz),
        "yz": sd(lambda a, b, c: newell_g(b, c, a), X, Y, Z, dx, dy, dz),
    }


def _half_axis_rule(nq, d):
    """Nodes and weights for int_{-d}^{d} phi(u) tri(u) du: Gauss-Legendre
    with nq nodes on each half [0, d] and [-d, 0], weight (1 - s)."""
    t, w = np.polynomial.legendre.leggauss(nq)
    s = 0.5 * (t + 1.0)
    w = 0.5 * w * (1.0 - s)
    return np.concatenate([d * s, -d * s]), np.concatenate([w, w])


def quadrature_tensor(X, Y, Z, cell, nq):
    """N at offsets (X, Y, Z) as the quadrature of the cell-cell average of
    the point-dipole tensor (valid only well away from the source cell)."""
    dx, dy, dz = cell
    V = dx * dy * dz
    X = np.asarray(X, np.float64).ravel(); Y = np.asarray(Y, np.float64).ravel()
    Z = np.asarray(Z, np.float64).ravel()
    px, wx = _half_axis_rule(nq, dx)
    py, wy = _half_axis_rule(nq, dy)
    pz, wz = _half_axis_rule(nq, dz)
    out = {c: np.zeros(X.shape) for c in COMPONENTS}
    for a in range(px.size):
        for b in range(py.size):
            for c in range(pz.size):
                w = wx[a] * wy[b] * wz[c]
                sx = X + px[a]; sy = Y + py[b]; sz = Z + pz[c]
                r2 = sx * sx + sy * sy + sz * sz
                inv5 = w / (r2 * r2 * np.sqrt(r2))
                out["xx"] += (r2 - 3.0 * sx * sx) * inv5
                out["yy"] += (r2 - 3.0 * sy * sy) * inv5
                out["zz"] += (r2 - 3.0 * sz * sz) * inv5
                out["xy"] += -3.0 * sx * sy * inv5
                out["xz"] += -3.0 * sx * sz * inv5
                out["yz"] += -3.0 * sy * sz * inv5
    for k in out:
        out[k] *= V / (4.0 * np.pi)
    return out


def demag_tensor(X, Y, Z, cell):
    """N at arbitrary offsets with the three-tier rule of the module doc."""
    X = np.asarray(X, np.float64); Y = np.asarray(Y, np.float64)
    Z = np.asarray(Z, np.float64)
    shape = np.broadcast(X, Y, Z).shape
    X, Y, Z = (np.broadcast_to(a, shape).ravel() for a in (X, Y, Z))
    dmax = max(cell)
    r2 = X * X + Y * Y + Z * Z
    tiers = [(r2 < (NEAR_CELLS * dmax) ** 2,
              lambda a, b, c: newell_tensor(a, b, c, cell))]
    lower = NEAR_CELLS
    for upper, nq in QUAD_TIERS:
        mask = (r2 >= (lower * dmax) ** 2) & (r2 < (upper * dmax) ** 2)
        tiers.append((mask, lambda a, b, c, nq=nq:
                      quadrature_tensor(a, b, c, cell, nq)))
        lower = upper
    out = {c: np.zeros(X.shape) for c in COMPONENTS}
    for mask, fn in tiers:
        if not mask.any():
            continue
        idx = np.nonzero(mask)[0]
        for lo in range(0, idx.size, 1 << 16):       # bounded memory
            sel = idx[lo:lo + (1 << 16)]
            part = fn(X[sel], Y[sel], Z[sel])
            for c in COMPONENTS:
                out[c][sel] = part[c]
    return {c: out[c].reshape(shape) for c in COMPONENTS}


def tensor_octant(grid, cell):
    """N on the non-negative offset octant: array (6, nz, ny, nx), entry
    [c, k, j, i] = N_c at offset (i dx, j dy, k dz), i < nx, j < ny, k < nz."""
    nx, ny, nz = grid
    dx, dy, dz = cell
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    t = demag_tensor(i * dx, j * dy, k * dz, cell)
    return np.stack([t[c] for c in COMPONENTS])


def tensor_full_offsets(octant):
    """Expand an octant (6, nz, ny, nx) to every offset -(n-1)..(n-1) on each
    axis using the parity of each component: array (6, 2nz-1, 2ny-1, 2nx-1)
    whose index (k + nz - 1, j + ny - 1, i + nx - 1) holds offset (i, j, k)."""
    _, nz, ny, nx = octant.shape
    out = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    oz = np.arange(-(nz - 1), nz); oy = np.arange(-(ny - 1), ny)
    ox = np.arange(-(nx - 1), nx)
    for c, name in enumerate(COMPONENTS):
        px, py, pz = PARITY[name]
        sz = np.where(oz < 0, pz, 1)[:, None, None]
        sy = np.where(oy < 0, py, 1)[None, :, None]
        sx = np.where(ox < 0, px, 1)[None, None, :]
        out[c] = (octant[c][np.abs(oz)][:, np.abs(oy)][:, :, np.abs(ox)]
                  * sx * sy * sz)
    return out


def aharoni_factor(a, b, c):
    """Magnetometric demagnetising factor D_z of a prism with edges
    2a x 2b x 2c along x, y, z (Aharoni, J. Appl. Phys. 83, 3432 (1998)).
    Independent of Newell's functions; used only to pin them."""
    r = np.sqrt(a * a + b * b + c * c)
    ab = np.sqrt(a * a + b * b); bc = np.sqrt(b * b + c * c)
    ac = np.sqrt(a * a + c * c)
    s = ((b * b - c * c) / (2 * b * c) * np.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * np.log((r - b) / (r + b))
         + b / (2 * c) * np.log((ab + a) / (ab - a))
         + a / (2 * c) * np.log((ab + b) / (ab - b))
         + c / (2 * a) * np.log((bc - b) / (bc + b))
         + c / (2 * b) * np.log((ac - a) / (ac + a))
         + 2 * np.arctan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / np.pi
