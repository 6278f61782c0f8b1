"""FP64 Fourier neural operator (FNO) for the demag-field surrogate, with a
hand-derived backward pass (test infrastructure only).

Not in the paper: the surrogate maps a magnetisation increment to its demag
field, H_demag(dM)/Ms from dM/Ms on an H x W film (nz = 1), so that between
exact FFT refreshes H_demag(M) = H_demag(M_ref) + FNO(M - M_ref) (H_demag is
linear in M).  Architecture (Li et al., Fourier neural operator):

  v0 = P [x; y/H; x/W] + p                       lift, 3 + 2 coordinate
                                                 channels -> C channels
  for l < L:  u = W_l v + b_l + S_l(v);  v = gelu(u) (identity for l = L-1)
  y  = Q v + q                                   projection, C -> 3

  S(v)[o] = (1/(HW)) Re sum_{ky in K} sum_{kx < m} a_kx * w[o](ky, kx)
                                   * exp(+2 pi i (ky y / H + kx x / W))
  w[o](ky, kx) = sum_c R[c, o](ky, kx) * v^[c](ky, kx)
  v^[c](ky, kx) = sum_{y, x} v[c](y, x) exp(-2 pi i (ky y / H + kx x / W))

with the retained modes K = {0..m-1} U {H-m..H-1} (2m rows) and kx < m
(a_0 = 1, a_kx = 2 otherwise: the real output keeps each kx > 0 and its
conjugate).  gelu(u) = u (1 + erf(u / sqrt 2)) / 2.  Loss: mean of (y - t)^2.

The two coordinate channels (row index / H, column index / W) let the
operator see the film's edges (the spectral part alone is periodic).
Parameters are a dict of float64 arrays: P (C,5), p (C), R_re / R_im
(L, C, C, 2m, m), W (L, C, C) [out, in], b (L, C), Q (3, C), q (3).
"""
import numpy as np
from scipy.special import erf

SQRT2 = np.sqrt(2.0)


def init_params(C, m, L, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    s = scale
    return {
        "P": rng.standard_normal((C, 5)) * s / np.sqrt(5.0),
        "p": np.zeros(C),
        "R_re": rng.standard_normal((L, C, C, 2 * m, m)) * s / C,
        "R_im": rng.standard_normal((L, C, C, 2 * m, m)) * s / C,
        "W": rng.standard_normal((L, C, C)) * s / np.sqrt(C),
        "b": np.zeros((L, C)),
        "Q": rng.standard_normal((3, C)) * s / np.sqrt(C),
        "q": np.zeros(3),
    }


def _ky(H, m):
    return np.concatenate([np.arange(m), np.arange(H - m, H)])


def forward_modes(v, m):
    """v^ on the retained modes: (C, 2m, m) complex."""
    H = v.shape[-2]
    return np.fft.fft2(v)[:, _ky(H, m), :m]


def inverse_modes(w, H, W):
    """(1/(HW)) Re sum a_kx w e^{+i...}: numpy's irfft2 of the zero-filled
    half spectrum is exactly this sum (it adds each kx > 0 term's conjugate
    and keeps the real part of the kx = 0 column); requires m < W/2."""
    m = w.shape[-1]
    full = np.zeros((w.shape[0], H, W // 2 + 1), complex)
    full[:, _ky(H, m), :m] = w
    return np.fft.irfft2(full, s=(H, W))


def retained_mask(H, W, m):
    """(H, W) boolean mask of the full 2-D spectrum that the spectral path
    can carry: (ky, kx) with ky in K and kx < m, and their conjugate partners
    (-ky, -kx), which the real output keeps with them."""
    mask = np.zeros((H, W), bool)
    ky, kx = _ky(H, m), np.arange(m)
    mask[np.ix_(ky, kx)] = True
    mask[np.ix_((-ky) % H, (-kx) % W)] = True
    return mask


def truncation_floor(h, m):
    """Relative L2 norm of the part of the fields h (..., H, W) outside the
    retained modes: sqrt(sum over dropped k of |h^(k)|^2 / sum over all k),
    by Parseval the error left by the best field the spectral path alone
    could output (its output lies in the retained modes)."""
    H, W = h.shape[-2:]
    hf = np.fft.fft2(h)
    keep = retained_mask(H, W, m)
    out = np.sum(np.abs(hf[..., ~keep]) ** 2)
    return float(np.sqrt(out / np.sum(np.abs(hf) ** 2)))


def spectral(v, Rl, m):
    vh = forward_modes(v, m)
    w = np.einsum("coyx,cyx->oyx", Rl, vh)
    return inverse_modes(w, v.shape[-2], v.shape[-1]), vh


def gelu(u):
    return 0.5 * u * (1.0 + erf(u / SQRT2))


def gelu_grad(u):
    return 0.5 * (1.0 + erf(u / SQRT2)) + u * np.exp(-0.5 * u * u) / np.sqrt(2.0 * np.pi)


def with_coords(xb):
    """(3, H, W) -> (5, H, W): the input plus row / H and column / W."""
    _, H, W = xb.shape
    yy, xx = np.meshgrid(np.arange(H) / H, np.arange(W) / W, indexing="ij")
    return np.concatenate([xb, yy[None], xx[None]])


def forward(params, x, m, keep=False):
    """x: (B, 3, H, W) -> y (B, 3, H, W); with keep, the intermediates."""
    L = params["W"].shape[0]
    R = params["R_re"] + 1j * params["R_im"]
    ys, caches = [], []
    for xb in x:
        v = np.einsum("oc,chw->ohw", params["P"], with_coords(xb)) + params["p"][:, None, None]
        cache = {"v": [v], "u": [], "vh": []}
        for l in range(L):
            s, vh = spectral(v, R[l], m)
            u = np.einsum("oc,chw->ohw", params["W"][l], v) + params["b"][l][:, None, None] + s
            v = gelu(u) if l < L - 1 else u
            cache["u"].append(u)
            cache["vh"].append(vh)
            cache["v"].append(v)
        ys.append(np.einsum("oc,chw->ohw", params["Q"], v) + params["q"][:, None, None])
        caches.append(cache)
    y = np.stack(ys)
    return (y, caches) if keep else y


def loss(params, x, t, m):
    y = forward(params, x, m)
    return float(np.mean((y - t) ** 2))


def gradients(params, x, t, m):
    """(loss, dict of gradients) by the chain rule written out layer by
    layer (adjoint of each linear map; see the module doc)."""
    L = params["W"].shape[0]
    R = params["R_re"] + 1j * params["R_im"]
    y, caches = forward(params, x, m, keep=True)
    B, _, H, W = x.shape
    count = y.size
    g = {k: np.zeros_like(v) for k, v in params.items()}
    dR = np.zeros_like(R)
    kys = _ky(H, m)
    a = np.where(np.arange(m) == 0, 1.0, 2.0)
    for bi in range(B):
        c = caches[bi]
        dy = 2.0 * (y[bi] - t[bi]) / count
        g["Q"] += np.einsum("ohw,chw->oc", dy, c["v"][L])
        g["q"] += dy.sum(axis=(1, 2))
        dv = np.einsum("oc,ohw->chw", params["Q"], dy)
        for l in reversed(range(L)):
            du = dv * gelu_grad(c["u"][l]) if l < L - 1 else dv
            vin = c["v"][l]
            g["b"][l] += du.sum(axis=(1, 2))
            g["W"][l] += np.einsum("ohw,chw->oc", du, vin)
            dv = np.einsum("oc,ohw->chw", params["W"][l], du)
            # spectral path: s = A(w), w = R v^, v^ = F(v)
            dw = (a / (H * W)) * np.fft.fft2(du)[:, kys, :m]
            dR[l] += np.einsum("oyx,cyx->coyx", dw, np.conj(c["vh"][l]))
            dvh = np.einsum("coyx,oyx->cyx", np.conj(R[l]), dw)
            full = np.zeros((dvh.shape[0], H, W), complex)
            full[:, kys, :m] = dvh
            dv = dv + (H * W) * np.real(np.fft.ifft2(full))
        g["P"] += np.einsum("ohw,chw->oc", dv, with_coords(x[bi]))
        g["p"] += dv.sum(axis=(1, 2))
    g["R_re"] = dR.real
    g["R_im"] = dR.imag
    return float(np.mean((y - t) ** 2)), g
