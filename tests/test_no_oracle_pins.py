"""Pins of the neural-operator oracle (oracle/no_oracle.py) against brute force and calculus (CPU).

The spectral convolution written with torch.fft must equal its definition as explicit DFT sums;
with identity mode matrices it must pass in-band Fourier modes unchanged and remove the others;
autograd gradients must match central finite differences.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import no_oracle as no  # noqa: E402


def _brute_spectral(h, Wm, D, m):
    """Definition by explicit sums: X(k) = sum_x h(x) e^{-2 pi i k.x/D} on the kept modes,
    Y = W X, s(x) = (1/D^3) Re sum_k c_kx Y(k) e^{+2 pi i k.x/D}, c_0 = 1, c_kx>0 = 2."""
    B, C = h.shape[:2]
    kept = no.kept(D, m)
    ax = np.arange(D)
    out = np.zeros_like(h)
    for b in range(B):
        for kxi in range(m):
            for kyi, ky in enumerate(kept):
                for kzi, kz in enumerate(kept):
                    kx = kxi
                    ph = np.exp(-2j * math.pi * (kz * ax[:, None, None] + ky * ax[None, :, None] + kx * ax[None, None, :]) / D)
                    X = np.array([(h[b, c] * ph).sum() for c in range(C)])
                    Wc = Wm[kxi, kyi, kzi, :, :, 0] + 1j * Wm[kxi, kyi, kzi, :, :, 1]
                    Y = Wc @ X
                    cf = 1.0 if kx == 0 else 2.0
                    out[b] += cf * np.real(Y[:, None, None, None] * np.conj(ph)[None]) / D ** 3
    return out


def test_spectral_conv_equals_dft_definition():
    D, m, C = 6, 2, 3
    rng = np.random.default_rng(0)
    h = rng.normal(size=(2, C, D, D, D))
    Wm = rng.normal(size=(m, 2 * m, 2 * m, C, C, 2))
    got = no.spectral_conv(torch.tensor(h), torch.tensor(Wm), D, m).numpy()
    assert np.allclose(got, _brute_spectral(h, Wm, D, m), atol=1e-12)


def test_identity_modes_keep_band_and_drop_rest():
    D, m, C = 8, 2, 2
    Wm = np.zeros((m, 2 * m, 2 * m, C, C, 2))
    for c in range(C):
        Wm[:, :, :, c, c, 0] = 1.0
    ax = np.arange(D)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    inband = np.cos(2 * math.pi * (1 * x + 7 * y + 1 * z) / D)     # kx = 1, ky = -1, kz = 1
    outband = np.cos(2 * math.pi * (3 * x) / D)                    # kx = 3 >= m
    h = np.stack([inband, outband])[None]
    got = no.spectral_conv(torch.tensor(h), torch.tensor(Wm), D, m).numpy()
    assert np.allclose(got[0, 0], inband, atol=1e-12)
    assert np.allclose(got[0, 1], 0.0, atol=1e-12)


def test_autograd_matches_finite_differences():
    D, W, m, L, Ci, Co = 6, 3, 2, 2, 2, 2
    _, n = no.layout(D, W, m, L, Ci, Co)
    rng = np.random.default_rng(1)
    theta = rng.normal(scale=0.3, size=n)
    a = rng.normal(size=(2, Ci, D, D, D))
    dout = rng.normal(size=(2, Co, D, D, D))
    _, g = no.forward_and_grad(theta, a, dout, D, W, m, L, Ci, Co)

    def f(t):
        return float((no.forward(torch.tensor(t), torch.tensor(a), D, W, m, L, Ci, Co).numpy() * dout).sum())
    for i in rng.choice(n, 12, replace=False):
        e = np.zeros(n)
        e[i] = 1e-6
        fd = (f(theta + e) - f(theta - e)) / 2e-6
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-8), i
