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
