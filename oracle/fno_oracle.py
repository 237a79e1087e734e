"""Plain FP64 CPU reference of the Fourier neural operator (FNO) that warm-starts
the messenger iteration.

TEST INFRASTRUCTURE: imported only by tests/ (and bench.py's CPU baseline).
It shares no code with the CUDA path.

The paper has no network; the warm start is an extension of the method.  What
it computes, written from the definition of a Fourier-neural-operator layer:

* input  x [B, 2, N, N]: the data map and a log noise-weight map;
* lift   h = P x + p                      (pointwise, 2 -> width channels);
* layers h <- act(W_l h + w_l + K_l h),   l = 0 .. L-1, act = GELU except after
                                          the last layer (identity);
* output y = Q h + q                      (pointwise, width -> 1 channel).

K_l is the spectral convolution on the retained modes: the real 2D DFT of
every channel, kept on k_x in [0, mx) and k_y in [0, my) U [N - my, N), mixed
across channels by one complex matrix per mode (R_l[i, o, mode]), every other
mode set to zero, and transformed back (numpy's rfft2 / irfft2 conventions:
unnormalised forward, 1/N^2 inverse, real output).

Pointwise weights are [out, in]; R_l is complex [in, out, 2 my, mx] with the
k_y axis ordered 0 .. my-1, N-my .. N-1.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)


def gelu(z):
    """GELU by its definition, z * Phi(z) with the normal CDF Phi."""
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def ky_index(N: int, my: int) -> np.ndarray:
    return np.concatenate([np.arange(my), np.arange(N - my, N)])


def spectral_conv(h: np.ndarray, R: np.ndarray, mx: int, my: int) -> np.ndarray:
    """K h for h [B, Ci, N, N] real and R [Ci, Co, 2 my, mx] complex."""
    B, Ci, N, _ = h.shape
    Co = R.shape[1]
    H = np.fft.rfft2(h)                                   # [B, Ci, N, N/2+1]
    ky = ky_index(N, my)
    Hm = H[:, :, ky, :mx]                                  # [B, Ci, 2my, mx]
    Ym = np.einsum("bimk,iomk->bomk", Hm, R)
    Y = np.zeros((B, Co, N, N // 2 + 1), np.complex128)
    Y[:, :, ky, :mx] = Ym
    return np.fft.irfft2(Y, s=(N, N))


def pointwise(W: np.ndarray, b: np.ndarray, h: np.ndarray) -> np.ndarray:
    return np.einsum("oi,bipq->bopq", W, h) + b[None, :, None, None]


def forward(params: dict, x: np.ndarray) -> np.ndarray:
    """Network output [B, N, N] for input x [B, 2, N, N]."""
    mx, my = params["mx"], params["my"]
    h = pointwise(params["P"], params["p"], x)
    L = len(params["W"])
    for l in range(L):
        z = pointwise(params["W"][l], params["w"][l], h) + spectral_conv(h, params["R"][l], mx, my)
        h = gelu(z) if l < L - 1 else z
    return pointwise(params["Q"], params["q"], h)[:, 0]


def loss(params: dict, x: np.ndarray, target: np.ndarray) -> float:
    """Mean over the batch of ||y_b - t_b||^2 / ||t_b||^2."""
    y = forward(params, x)
    num = ((y - target) ** 2).sum(axis=(1, 2))
    den = (target ** 2).sum(axis=(1, 2))
    return float(np.mean(num / den))


def flatten(params: dict) -> np.ndarray:
    """Every trainable number in one vector, in the library's order:
    P, p, then per layer W_l, w_l, Re/Im of R_l (interleaved), then Q, q."""
    parts = [params["P"].ravel(), params["p"].ravel()]
    for l in range(len(params["W"])):
        R = params["R"][l]
        parts += [params["W"][l].ravel(), params["w"][l].ravel(),
                  np.stack([R.real, R.imag], axis=-1).ravel()]
    parts += [params["Q"].ravel(), params["q"].ravel()]
    return np.concatenate(parts).astype(np.float64)


def unflatten(theta: np.ndarray, like: dict) -> dict:
    """Inverse of flatten with the shapes of `like`."""
    out = {"mx": like["mx"], "my": like["my"], "W": [], "w": [], "R": []}
    i = 0

    def take(shape):
        nonlocal i
        n = int(np.prod(shape))
        v = theta[i:i + n].reshape(shape)
        i += n
        return v

    out["P"] = take(like["P"].shape)
    out["p"] = take(like["p"].shape)
    for l in range(len(like["W"])):
        out["W"].append(take(like["W"][l].shape))
        out["w"].append(take(like["w"][l].shape))
        ri = take(like["R"][l].shape + (2,))
        out["R"].append(ri[..., 0] + 1j * ri[..., 1])
    out["Q"] = take(like["Q"].shape)
    out["q"] = take(like["q"].shape)
    return out


def template(width: int, mx: int, my: int, layers: int, cin: int = 2) -> dict:
    """Zero parameters with the network's shapes (for unflatten)."""
    return {"mx": mx, "my": my,
            "P": np.zeros((width, cin)), "p": np.zeros(width),
            "W": [np.zeros((width, width)) for _ in range(layers)],
            "w": [np.zeros(width) for _ in range(layers)],
            "R": [np.zeros((width, width, 2 * my, mx), np.complex128) for _ in range(layers)],
            "Q": np.zeros((1, width)), "q": np.zeros(1)}


def features(d: np.ndarray, pixel_var: np.ndarray, mask) -> tuple[np.ndarray, float]:
    """Network input of one map: d / sigma (0 where masked) and
    log(sigma^2 / pixel_var) (log 1e-6 where masked), sigma^2 the mean pixel
    variance over unmasked pixels."""
    m = np.zeros(d.shape, bool) if mask is None else mask.astype(bool)
    v = pixel_var.astype(np.float64)
    sigma = math.sqrt(v[~m].mean())
    x0 = np.where(m, 0.0, d.astype(np.float64) / sigma)
    x1 = np.where(m, math.log(1e-6), np.log(sigma ** 2 / np.where(m, 1.0, v)))
    return np.stack([x0, x1]), sigma


def fd_gradient(params: dict, x: np.ndarray, target: np.ndarray, idx, step: float = 1e-6) -> np.ndarray:
    """Central finite differences of `loss` with respect to the flattened
    parameters at positions idx."""
    theta = flatten(params)
    g = np.empty(len(idx))
    for j, k in enumerate(idx):
        tp = theta.copy()
        tp[k] += step
        tm = theta.copy()
        tm[k] -= step
        g[j] = (loss(unflatten(tp, params), x, target) - loss(unflatten(tm, params), x, target)) / (2 * step)
    return g
