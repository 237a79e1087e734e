"""Pins of the FP64 FNO oracle (the warm-start network) against what its
definition fixes: brute-force DFT sums, a band-limited identity, translation
equivariance on the torus, the GELU identities, and a closed-form gradient."""

import math

import numpy as np
import pytest

from oracle import fno_oracle as F
from paper_1704_00865_gb300 import synth


def _rand_params(rng, width, mx, my, layers, scale=0.3):
    p = F.template(width, mx, my, layers)
    theta = rng.normal(0.0, scale, F.flatten(p).size)
    return F.unflatten(theta, p)


def test_spectral_conv_matches_brute_force_sums():
    rng = np.random.default_rng(0)
    N, Ci, Co, mx, my = 8, 2, 3, 2, 2
    h = rng.standard_normal((1, Ci, N, N))
    R = rng.standard_normal((Ci, Co, 2 * my, mx)) + 1j * rng.standard_normal((Ci, Co, 2 * my, mx))
    kys = list(range(my)) + list(range(N - my, N))
    y = np.arange(N)[:, None]
    x = np.arange(N)[None, :]
    H = np.zeros((Ci, 2 * my, mx), complex)
    for i in range(Ci):
        for j, ky in enumerate(kys):
            for kx in range(mx):
                H[i, j, kx] = (h[0, i] * np.exp(-2j * np.pi * (ky * y + kx * x) / N)).sum()
    out = np.zeros((Co, N, N))
    for o in range(Co):
        Y = sum(R[i, o] * H[i] for i in range(Ci))
        for j, ky in enumerate(kys):
            for kx in range(mx):
                w = 1.0 if kx == 0 else 2.0
                out[o] += w * np.real(Y[j, kx] * np.exp(2j * np.pi * (ky * y + kx * x) / N))
    out /= N * N
    assert np.allclose(F.spectral_conv(h, R, mx, my)[0], out, atol=1e-12)


def _eye(C, mx, my):
    R = np.zeros((C, C, 2 * my, mx), complex)
    for i in range(C):
        R[i, i] = 1.0
    return R


def test_spectral_conv_is_the_identity_on_band_limited_maps():
    rng = np.random.default_rng(1)
    N, C, mx, my = 16, 3, 4, 3
    # a map band limited to |k_y| < my - 1, k_x < mx - 1: both members of every
    # Hermitian pair are retained, so the identity mixing reproduces it
    h = F.spectral_conv(rng.standard_normal((2, C, N, N)), _eye(C, mx - 1, my - 1), mx - 1, my - 1)
    assert np.allclose(F.spectral_conv(h, _eye(C, mx, my), mx, my), h, atol=1e-12)
    # the retained set [0, my) U [N - my, N) holds k_y = -my without +my: on
    # k_x = 0 the real part halves that mode, so K is not a projection there
    g = rng.standard_normal((1, 1, N, N))
    k1 = F.spectral_conv(g, _eye(1, mx, my), mx, my)
    k2 = F.spectral_conv(k1, _eye(1, mx, my), mx, my)
    d = np.fft.rfft2(k1 - k2)[0, 0]
    assert abs(d[N - my, 0]) > 1e-6 and np.allclose(np.delete(d[:, 0], [my, N - my]), 0, atol=1e-10)


def test_network_is_translation_equivariant():
    rng = np.random.default_rng(2)
    p = _rand_params(rng, width=4, mx=3, my=3, layers=2)
    x = rng.standard_normal((1, 2, 16, 16))
    y = F.forward(p, x)
    ys = F.forward(p, np.roll(x, (3, -5), axis=(2, 3)))
    assert np.allclose(ys, np.roll(y, (3, -5), axis=(1, 2)), atol=1e-10)


def test_gelu_identities():
    z = np.linspace(-6, 6, 101)
    # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z)) = z
    assert np.allclose(F.gelu(z) - F.gelu(-z), z, atol=1e-14)
    assert F.gelu(0.0) == 0.0
    assert F.gelu(1.0) == pytest.approx(0.5 * (1 + math.erf(1 / math.sqrt(2))), rel=1e-15)


def test_last_bias_gradient_has_its_closed_form():
    # dL/dq = mean_b sum_p 2 (y_b - t_b) / ||t_b||^2: pins loss() and fd_gradient()
    rng = np.random.default_rng(3)
    p = _rand_params(rng, width=4, mx=2, my=2, layers=2)
    x = rng.standard_normal((2, 2, 8, 8))
    t = rng.standard_normal((2, 8, 8))
    y = F.forward(p, x)
    g_exact = np.mean([2.0 * (y[b] - t[b]).sum() / (t[b] ** 2).sum() for b in range(2)])
    k = F.flatten(p).size - 1
    g_fd = F.fd_gradient(p, x, t, [k])[0]
    assert g_fd == pytest.approx(g_exact, rel=1e-6)


def test_flatten_round_trip_and_initialiser_layout():
    width, mx, my, layers = 6, 3, 2, 3
    theta = synth.fno_init(7, width, mx, my, layers).astype(np.float64)
    p = F.unflatten(theta, F.template(width, mx, my, layers))
    assert np.array_equal(F.flatten(p), theta)
    assert theta.size == width * 2 + width + layers * (width * width + width + width * width * 2 * my * mx * 2) \
        + width + 1


def test_features_definition():
    prob = synth.make_problem(32, 32, 5, mask_frac=0.1)
    x, sigma = F.features(prob.d, prob.pixel_var, prob.mask)
    m = prob.mask.astype(bool)
    assert sigma == pytest.approx(math.sqrt(prob.pixel_var[~m].astype(np.float64).mean()))
    assert np.all(x[0][m] == 0.0) and np.allclose(x[1][m], math.log(1e-6))
    assert np.allclose(x[1][~m], np.log(sigma ** 2 / prob.pixel_var[~m]))
