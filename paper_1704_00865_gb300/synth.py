"""Seeded synthetic inputs for the multi-messenger Wiener filter.

This module makes problem instances only: a Gaussian signal map, the three
noise covariances and one noise realisation drawn from them, and a disc mask.
It contains none of the Wiener-filter arithmetic, so both the FP64 CPU oracle
and the CUDA path can take their inputs from here without sharing any of the
method.

The workloads are flat-sky, periodic N_y x N_x maps standing in for the
paper's HEALPix maps (Sec. 3): an isotropic red signal spectrum, spatially
varying white noise with a mask (Sec. 3.2, Sec. 3.3), isotropic 1/f noise
that is diagonal in 2D Fourier space, and horizontal stripes that are
diagonal in the row-wise 1D Fourier basis (the dense-noise example of
Sec. 3.3, whose harmonic noise puts power into m = 0 to make stripes).

Spectral arrays use the half-spectrum layout [ny][nx/2+1] of a real 2D DFT
(row index ky in FFT order, column index kx = 0..nx/2).  Every spectral value
is an eigenvalue of the covariance matrix; those eigenvalues do not depend on
how the DFT is normalised.

Recipe (seed -> arrays), all with numpy's PCG64 ``default_rng(seed)``:

* k = |(kx, ky)| in integer cycles per map; C(k) = (k + 2)^-2.5.
* rms_s^2 = mean of C over all ny*nx modes (the signal pixel variance).
* signal: s = irfft2(sqrt(C) * rfft2(w)), w ~ N(0, 1) per pixel.
* white: sigma_p = 0.3 rms_s exp(0.5 z_p), z ~ N(0, 1); pixel_var = sigma_p^2.
* 1/f: P1f(k) = sigma_f^2 (1 + (k_knee / max(k, 1))^2), k_knee = 20,
  sigma_f = 0.3 rms_s.
* stripes: Pst(kx) = sigma_s^2 (k_knee_x / max(|kx|, 1))^2.5, k_knee_x = 20,
  sigma_s = 0.3 rms_s; rows are independent; optional per-row amplitude
  a(y) = exp(0.5 z_y) scales row y by a(y) (covariance a(y)^2 Pst).
* mask: discs with centres uniform on the torus and radii uniform in
  [8, 32] * N/1024 pixels are added until at least the requested fraction of
  pixels is masked; d is set to 0 there.
"""

from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

K_KNEE = 20.0
K_KNEE_X = 20.0
NOISE_RMS_FRAC = 0.3


@dataclasses.dataclass
class Problem:
    """One synthetic problem instance (float32 arrays, as both sides see them)."""

    d: np.ndarray                 # [ny][nx] data map
    pixel_var: np.ndarray         # [ny][nx] white-noise variance per pixel
    mask: Optional[np.ndarray]    # [ny][nx] uint8, 1 = masked, or None
    C: np.ndarray                 # [ny][nx/2+1] signal eigenvalues
    P1f: Optional[np.ndarray]     # [ny][nx/2+1] 1/f eigenvalues, or None
    Pst: Optional[np.ndarray]     # [nx/2+1] stripe eigenvalues per kx, or None
    stripe_amp2: Optional[np.ndarray]  # [ny] a(y)^2 per row, or None (== 1)
    s_true: np.ndarray            # [ny][nx] the signal realisation
    meta: dict

    @property
    def shape(self):
        return self.d.shape


def kgrid(ny: int, nx: int) -> np.ndarray:
    """|k| on the half-spectrum grid [ny][nx/2+1], in cycles per map."""
    ky = np.fft.fftfreq(ny, d=1.0 / ny)
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    return np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)


def half_mode_weights(ny: int, nx: int) -> np.ndarray:
    """How many full-grid modes each half-spectrum entry stands for (1 or 2)."""
    w = np.full((ny, nx // 2 + 1), 2.0)
    w[:, 0] = 1.0
    if nx % 2 == 0:
        w[:, nx // 2] = 1.0
    return w


def signal_spectrum(ny: int, nx: int) -> np.ndarray:
    k = kgrid(ny, nx)
    return (k + 2.0) ** -2.5


def _grf(rng, spec_half: np.ndarray, ny: int, nx: int) -> np.ndarray:
    w = rng.standard_normal((ny, nx))
    return np.fft.irfft2(np.sqrt(spec_half) * np.fft.rfft2(w), s=(ny, nx))


def disc_mask(rng, ny: int, nx: int, frac: float) -> np.ndarray:
    """Random discs on the torus until at least ``frac`` of the pixels are masked."""
    m = np.zeros((ny, nx), dtype=bool)
    if frac <= 0:
        return m.astype(np.uint8)
    scale = max(ny, nx) / 1024.0
    yy = np.arange(ny)[:, None]
    xx = np.arange(nx)[None, :]
    while m.mean() < frac:
        cy = rng.uniform(0, ny)
        cx = rng.uniform(0, nx)
        r = rng.uniform(8.0, 32.0) * scale
        r = max(r, 0.75)
        dy = np.abs(yy - cy)
        dy = np.minimum(dy, ny - dy)
        dx = np.abs(xx - cx)
        dx = np.minimum(dx, nx - dx)
        m |= (dy ** 2 + dx ** 2) <= r * r
    return m.astype(np.uint8)


def make_problem(ny: int, nx: int, seed: int, *, white: bool = True,
                 one_over_f: bool = True, stripes: bool = True,
                 mask_frac: float = 0.05, stripe_rows_vary: bool = False,
                 homogeneous: bool = False, noise_scale: float = 1.0,
                 amp_jitter: float = 0.0, k_knee: float = K_KNEE,
                 k_knee_x: float = K_KNEE_X) -> Problem:
    """Draw one problem.

    ``homogeneous=True`` makes every pixel variance equal (the median level),
    which together with ``mask_frac=0`` and ``stripe_rows_vary=False`` gives
    a problem whose noise is diagonal in 2D Fourier space.
    ``amp_jitter`` scales sigma_f and sigma_s by exp(U[-amp_jitter, amp_jitter]).
    ``k_knee`` / ``k_knee_x`` set the knees of the 1/f and stripe spectra
    (20 cycles per map by default; small values give the quickly converging
    tiny problems that unit tests use).
    """
    assert ny >= 2 and nx >= 2 and nx % 2 == 0
    rng = np.random.default_rng(seed)
    C = signal_spectrum(ny, nx)
    rms_s2 = float((C * half_mode_weights(ny, nx)).sum() / (ny * nx))
    sig = NOISE_RMS_FRAC * np.sqrt(rms_s2) * noise_scale

    s_true = _grf(rng, C, ny, nx)
    d = s_true.copy()

    z = rng.standard_normal((ny, nx))
    if homogeneous:
        z[:] = 0.0
    pixel_var = (sig * np.exp(0.5 * z)) ** 2
    n_white = np.sqrt(pixel_var) * rng.standard_normal((ny, nx))
    if white:
        d += n_white

    jf = np.exp(rng.uniform(-amp_jitter, amp_jitter)) if amp_jitter else 1.0
    js = np.exp(rng.uniform(-amp_jitter, amp_jitter)) if amp_jitter else 1.0

    P1f = None
    if one_over_f:
        k = np.maximum(kgrid(ny, nx), 1.0)
        P1f = (sig * jf) ** 2 * (1.0 + (k_knee / k) ** 2)
        d += _grf(rng, P1f, ny, nx)

    Pst = None
    amp2 = None
    if stripes:
        kx = np.maximum(np.arange(nx // 2 + 1, dtype=np.float64), 1.0)
        Pst = (sig * js) ** 2 * (k_knee_x / kx) ** 2.5
        w = rng.standard_normal((ny, nx))
        n_st = np.fft.irfft(np.sqrt(Pst)[None, :] * np.fft.rfft(w, axis=1), n=nx, axis=1)
        if stripe_rows_vary:
            amp2 = np.exp(0.5 * rng.standard_normal(ny)) ** 2
            n_st = n_st * np.sqrt(amp2)[:, None]
        d += n_st

    mask = None
    if mask_frac > 0:
        mask = disc_mask(rng, ny, nx, mask_frac)
        d[mask.astype(bool)] = 0.0

    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    return Problem(
        d=f32(d), pixel_var=f32(pixel_var), mask=mask, C=f32(C), P1f=f32(P1f),
        Pst=f32(Pst), stripe_amp2=f32(amp2), s_true=f32(s_true),
        meta=dict(ny=ny, nx=nx, seed=seed, rms_s2=rms_s2, sigma=sig,
                  mask_frac=float(mask.mean()) if mask is not None else 0.0),
    )


def cfg0_problem(seed: int = 0) -> Problem:
    """64x64, white noise only (log-normal per-pixel std), no mask."""
    return make_problem(64, 64, seed, one_over_f=False, stripes=False, mask_frac=0.0)


def cfg1_problem(seed: int = 1000, n: int = 1024, **kw) -> Problem:
    """n x n, white + isotropic 1/f + horizontal stripes, 5% disc mask."""
    return make_problem(n, n, seed, **kw)


def fno_init(seed: int, width: int = 32, mx: int = 16, my: int = 16, layers: int = 4, cin: int = 2) -> np.ndarray:
    """Seeded initial parameters of the warm-start network, as one float32
    vector in the order P [width][cin], p [width], per layer W [width][width],
    w [width], R [width][width][2 my][mx] (re, im) pairs, then Q [1][width],
    q [1].  Matrices ~ N(0, 1/fan_in); spectral weights uniform in
    [0, 1/width^2) in both parts; biases 0."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, 1.0 / np.sqrt(cin), (width, cin)).ravel(), np.zeros(width)]
    for _ in range(layers):
        parts += [rng.normal(0.0, 1.0 / np.sqrt(width), (width, width)).ravel(), np.zeros(width),
                  rng.uniform(0.0, 1.0 / (width * width), (width, width, 2 * my, mx, 2)).ravel()]
    parts += [rng.normal(0.0, 1.0 / np.sqrt(width), (1, width)).ravel(), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
