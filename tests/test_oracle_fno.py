"""Pins of the FP64 FNO oracle (oracle/fno.py): its spectral convolution
against the explicit double sum of its definition, the identity special
case, and its hand-written gradients against central differences."""
import numpy as np
import pytest

from oracle import fno as F


def test_spectral_conv_matches_explicit_double_sum():
    rng = np.random.default_rng(0)
    C, H, W, m = 3, 8, 10, 3
    v = rng.standard_normal((C, H, W))
    R = rng.standard_normal((C, C, 2 * m, m)) + 1j * rng.standard_normal((C, C, 2 * m, m))
    s, _ = F.spectral(v, R, m)
    ky = np.concatenate([np.arange(m), np.arange(H - m, H)])
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ref = np.zeros((C, H, W))
    for o in range(C):
        for iy, k in enumerate(ky):
            for kx in range(m):
                vh = np.array([np.sum(v[c] * np.exp(-2j * np.pi * (k * yy / H + kx * xx / W))) for c in range(C)])
                w = np.sum(R[:, o, iy, kx] * vh)
                a = 1.0 if kx == 0 else 2.0
                ref[o] += a * np.real(w * np.exp(2j * np.pi * (k * yy / H + kx * xx / W))) / (H * W)
    assert np.max(np.abs(s - ref)) < 1e-12


def test_identity_weights_reproduce_band_limited_input():
    rng = np.random.default_rng(1)
    C, H, W, m = 2, 8, 12, 4
    full = np.zeros((C, H, W // 2 + 1), complex)
    full[:, :, :m] = rng.standard_normal((C, H, m)) + 1j * rng.standard_normal((C, H, m))
    v = np.fft.irfft2(full, s=(H, W))            # only kx < m, every ky (2m = H)
    R = np.zeros((C, C, 2 * m, m), complex)
    for c in range(C):
        R[c, c] = 1.0
    s, _ = F.spectral(v, R, m)
    assert np.max(np.abs(s - v)) < 1e-12


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    C, m, L, H, W, B = 4, 2, 2, 8, 8, 2
    p = F.init_params(C, m, L, seed=3, scale=1.5)
    for k in ("p", "b", "q"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((B, 3, H, W))
    t = rng.standard_normal((B, 3, H, W))
    _, g = F.gradients(p, x, t, m)
    for name in p:
        d = rng.standard_normal(p[name].shape)
        eps = 1e-6
        pp = {k: v.copy() for k, v in p.items()}
        pm = {k: v.copy() for k, v in p.items()}
        pp[name] = p[name] + eps * d
        pm[name] = p[name] - eps * d
        fd = (F.loss(pp, x, t, m) - F.loss(pm, x, t, m)) / (2 * eps)
        an = float(np.sum(g[name] * d))
        assert abs(fd - an) <= 1e-6 * max(1e-8, abs(an)) + 1e-12, (name, fd, an)


def test_truncation_floor_pins():
    """The floor of the FNO's retained modes: zero for a field that lies in
    them, one for a field wholly outside, the exact orthogonal split for a
    mixture, and the same projection as the spectral path with identity
    weights (an independent route through irfft2)."""
    rng = np.random.default_rng(3)
    C, H, W, m = 3, 16, 20, 4
    full = np.zeros((C, H, W // 2 + 1), complex)
    ky = np.concatenate([np.arange(m), np.arange(H - m, H)])
    full[:, ky, :m] = rng.standard_normal((C, 2 * m, m)) + 1j * rng.standard_normal((C, 2 * m, m))
    inside = np.fft.irfft2(full, s=(H, W))
    assert F.truncation_floor(inside, m) < 1e-12
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    outside = np.cos(2 * np.pi * (m * yy / H + (m + 1) * xx / W))[None] * np.ones((C, 1, 1))
    assert abs(F.truncation_floor(outside, m) - 1.0) < 1e-12
    a, b = 0.6, 0.8
    u = inside / np.linalg.norm(inside)
    v = outside / np.linalg.norm(outside)
    assert abs(F.truncation_floor(a * u + b * v, m) - b / np.hypot(a, b)) < 1e-12
    # brute force: least-squares fit of a random field by every real field
    # the spectral path can output (cos and sin of each retained (ky, kx))
    h = rng.standard_normal((C, H, W))
    basis = []
    for k in ky:
        for kx in range(m):
            ph = 2 * np.pi * (k * yy / H + kx * xx / W)
            basis += [np.cos(ph).ravel(), np.sin(ph).ravel()]
    Bm = np.array(basis).T
    res = 0.0
    for c in range(C):
        coef = np.linalg.lstsq(Bm, h[c].ravel(), rcond=None)[0]
        res += np.sum((h[c].ravel() - Bm @ coef) ** 2)
    assert abs(F.truncation_floor(h, m) - np.sqrt(res) / np.linalg.norm(h)) < 1e-12
