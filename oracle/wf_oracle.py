"""Plain, slow, FP64 reference implementation of the multi-messenger Wiener filter.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline.  It shares no code with the CUDA path.

What it computes (Huffenberger 2017, arXiv:1704.00865):

* ``dense_wf``      -- the Wiener filter by its definition, Sec. 1 eq. (wiener):
                       s = (S^-1 + N^-1)^-1 N^-1 d, dense matrices + Cholesky
                       (tiny maps only).  A mask is infinite noise variance
                       (Sec. 3.2, Sec. 3.3): N^-1 := P^T (P N P^T)^-1 P.
* ``dense_wf_alt``  -- the same by eq. (wiener-alt), s = S (S + N)^-1 d,
                       restricted to unmasked pixels.
* ``closed_form``   -- homogeneous noise: every part is diagonal in 2D Fourier
                       space and s_k = C_k / (C_k + N_k) d_k (Sec. 3.1).
* ``inverse_noise_dense`` -- N^-1 d by its definition (dense, tiny maps): what
                       the S = alpha I Wiener filter of Sec. 4 approximates.
* ``Chain`` / ``messenger_solve`` -- the messenger iteration itself, eqs.
                       (2mess_t1)-(2mess_s) of Sec. 2 generalised to K parts
                       as Sec. 2 and Appendix A describe ("each additional
                       piece ... two additional fields"), with T_i = lambda
                       tau_i I, Nbar_i = N_i - tau_i I fixed while lambda cools
                       (Sec. 2), and the lambda rule of Sec. 3.3.
* ``residual_terms`` -- the reconstructed-data difference Delta d = (I + N
                       S^-1) s - d of Sec. 2 restricted to unmasked pixels,
                       plus S^-1 s on masked pixels.
* ``literal_residual`` / ``pcg_wf`` -- FP64 conjugate gradients for
                       || (S^-1 + N^-1) s - N^-1 d || / || N^-1 d || and for the
                       Wiener solution itself on full-size maps.
* ``chi2`` / ``chi2_aug`` -- the objective of Sec. 1 and the augmented
                       objective of Appendix A eq. (2mess_prob).

Conventions.  Maps are real [ny][nx].  Three noise parts, in chain order from
the signal end: part "2DF" (diagonal in the 2D DFT: isotropic 1/f), part "RF"
(diagonal in the row-wise 1D DFT along x: stripes), part "PX" (diagonal in
pixels: white noise, infinite at masked pixels).  Spectral inputs use the
half-spectrum layout [ny][nx/2+1] and are expanded here to the full grid by
Hermitian symmetry.  Transforms are numpy/scipy FFTs of the full complex
field (unnormalised forward, 1/n inverse); eigenvalues do not depend on the
normalisation.

Readings where the paper is silent (each also listed in the design notes):
* chain order 2DF -> RF -> PX from the signal end; the sweep runs from the
  data end: t_PX, d_RF, t_RF, d_2DF, t_2DF, s;
* tau_i = theta_i * (minimum eigenvalue of part i); theta < 1 for interior
  parts keeps Nbar_i > 0 so no mode is frozen (an interior link with
  Nbar = 0 pins d_i = t_i and neither ever moves);
* a white floor may be moved between parts (white is diagonal in every
  basis), which leaves N and the solution unchanged (Sec. 3.1 splits white
  noise between parts; Sec. 3.3 gives the harmonic part half of it);
* one shared lambda for all parts;
* lambda rule: after each residual evaluation, if the per-iteration
  relative change of Delta d^T Delta d is below ``ratio``, lambda <- lambda^expo,
  snapping to 1 below ``snap``; the reference value of Delta d^T Delta d is
  reset after every change of lambda.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

try:  # scipy.fft is a drop-in library FFT that can use several threads
    import scipy.fft as _sfft
except Exception:  # pragma: no cover
    _sfft = None

__all__ = [
    "FFT_WORKERS", "set_workers", "full_from_half", "full_stripe", "brute_dft",
    "brute_idft", "Parts", "build_parts", "dense_cov_stationary",
    "dense_cov_stripes", "dense_matrices", "dense_wf", "dense_wf_alt",
    "closed_form", "Chain", "messenger_solve", "fixed_schedule",
    "cooling_levels", "apply_N", "apply_Sinv", "residual_terms", "pcg",
    "literal_residual", "pcg_wf", "chi2", "rel_l2", "DEFAULT_THETA",
    "ADAPTIVE_DEFAULT", "DEFAULT_SPLIT_F", "rel_terms", "to_basis", "from_basis",
    "inverse_noise_dense", "chi2_aug_state",
]

FFT_WORKERS = 1
DEFAULT_THETA = (0.9, 0.9, 1.0)          # (2DF, RF, PX)
# Half of the 1/f part's white floor is carried by the stripe part, which
# raises the stripe messenger's tau from the tiny Nyquist stripe power to a
# useful level without changing N (Sec. 3.3 likewise gives the harmonic part
# half of the white noise).
DEFAULT_SPLIT_F = 0.5
# Sec. 3.3: lambda starts near 5e5, lowered by lambda^0.7 when Delta d^T
# Delta d changes by less than 1e-2 per iteration.
ADAPTIVE_DEFAULT = dict(lam0=5e5, ratio=1e-2, expo=0.7, snap=1.01)


def set_workers(n: int) -> None:
    global FFT_WORKERS
    FFT_WORKERS = max(1, int(n))


def _fft2(x):
    if _sfft is not None:
        return _sfft.fft2(x, workers=FFT_WORKERS)
    return np.fft.fft2(x)


def _ifft2(x):
    if _sfft is not None:
        return _sfft.ifft2(x, workers=FFT_WORKERS)
    return np.fft.ifft2(x)


def _fftx(x):
    if _sfft is not None:
        return _sfft.fft(x, axis=1, workers=FFT_WORKERS)
    return np.fft.fft(x, axis=1)


def _ifftx(x):
    if _sfft is not None:
        return _sfft.ifft(x, axis=1, workers=FFT_WORKERS)
    return np.fft.ifft(x, axis=1)


# ----------------------------------------------------------------------------
# spectra on the full grid
# ----------------------------------------------------------------------------

def full_from_half(half: np.ndarray, nx: int) -> np.ndarray:
    """Expand [ny][nx/2+1] eigenvalues to [ny][nx]: e(ky, kx) = e(-ky, -kx)."""
    half = np.asarray(half, dtype=np.float64)
    ny = half.shape[0]
    full = np.empty((ny, nx))
    h = nx // 2
    full[:, : h + 1] = half
    for kx in range(h + 1, nx):
        full[:, kx] = half[(-np.arange(ny)) % ny, nx - kx]
    return full


def full_stripe(Pst: np.ndarray, nx: int) -> np.ndarray:
    """Expand the per-kx stripe eigenvalues [nx/2+1] to [nx]: e(kx) = e(-kx)."""
    Pst = np.asarray(Pst, dtype=np.float64)
    return np.array([Pst[min(k, nx - k)] for k in range(nx)])


def brute_dft(x: np.ndarray, axis: int = -1, inverse: bool = False) -> np.ndarray:
    """O(n^2) DFT along one axis, straight from the definition (pins only)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    j = np.arange(n)
    sgn = 1.0 if inverse else -1.0
    W = np.exp(sgn * 2j * np.pi * np.outer(j, j) / n)
    y = x @ W.T
    if inverse:
        y = y / n
    return np.moveaxis(y, -1, axis)


def brute_idft(X: np.ndarray, axis: int = -1) -> np.ndarray:
    return brute_dft(X, axis=axis, inverse=True)


# ----------------------------------------------------------------------------
# the noise parts and messenger covariances
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Part:
    name: str                 # "2DF" | "RF" | "PX"
    N: np.ndarray             # eigenvalues of this part (after white moves), in its basis
    tau: float                # theta * min eigenvalue
    Nbar: np.ndarray          # N - tau (inf where masked)


@dataclasses.dataclass
class Parts:
    ny: int
    nx: int
    C: np.ndarray             # [ny][nx] signal eigenvalues
    parts: list               # signal end first
    unmasked: np.ndarray      # bool [ny][nx]
    d: np.ndarray             # [ny][nx] float64, 0 at masked pixels
    N0_full: Optional[np.ndarray]   # original parts (before moves), for N itself
    N1_full: Optional[np.ndarray]
    var: np.ndarray           # [ny][nx] pixel variance (unmasked values)
    merge_2df: bool = False   # 2DF block updated jointly (Appendix A shortcut)


def build_parts(prob, theta: Sequence[float] = DEFAULT_THETA, split_f: float = DEFAULT_SPLIT_F,
                split_w: float = 0.0, merge_2df: bool = False, split_fp: float = 0.0) -> Parts:
    """Messenger covariances of Sec. 2: T_i = tau_i I with tau_i = theta_i x the
    minimum eigenvalue of N_i (Sec. 2, Appendix A), Nbar_i = N_i - tau_i.

    ``split_f`` moves split_f * min(P1f) of white floor from the 2DF part to
    the RF part, ``split_fp`` moves split_fp * min(P1f) from the 2DF part to
    the PX part, and ``split_w`` moves split_w * min(pixel_var) from the PX
    part to the RF part.  All leave N = sum_i N_i unchanged.

    ``merge_2df``: the 2DF part needs no messenger covariance of its own (its
    tau is 0 and Nbar is the whole, possibly reduced, 1/f part): the sweep
    updates s, t_0 and d_0 together (see Chain.sweep).
    """
    d = np.asarray(prob.d, dtype=np.float64)
    ny, nx = d.shape
    var = np.asarray(prob.pixel_var, dtype=np.float64)
    mask = None if prob.mask is None else np.asarray(prob.mask).astype(bool)
    unmasked = np.ones((ny, nx), bool) if mask is None else ~mask
    C = full_from_half(prob.C, nx)

    have_f = prob.P1f is not None
    have_s = prob.Pst is not None
    N0 = full_from_half(prob.P1f, nx) if have_f else None
    N1 = None
    if have_s:
        a2 = np.ones(ny) if prob.stripe_amp2 is None else np.asarray(prob.stripe_amp2, np.float64)
        N1 = a2[:, None] * full_stripe(prob.Pst, nx)[None, :]

    vmin = float(var[unmasked].min())
    w_f = split_f * float(N0.min()) if (have_f and have_s) else 0.0
    w_fp = split_fp * float(N0.min()) if have_f else 0.0
    w_w = split_w * vmin if have_s else 0.0

    parts = []
    th_f, th_s, th_p = theta
    if have_f:
        n0 = N0 - w_f - w_fp
        tau = 0.0 if merge_2df else th_f * float(n0.min())
        parts.append(Part("2DF", n0, tau, n0 - tau))
    if have_s:
        n1 = N1 + w_f + w_w
        tau = th_s * float(n1.min())
        parts.append(Part("RF", n1, tau, n1 - tau))
    n2 = np.where(unmasked, var - w_w + w_fp, np.inf)
    tau = th_p * float(n2[unmasked].min())
    parts.append(Part("PX", n2, tau, np.where(unmasked, n2 - tau, np.inf)))
    dd = np.where(unmasked, d, 0.0)
    return Parts(ny, nx, C, parts, unmasked, dd, N0, N1, np.where(unmasked, var, 0.0),
                 merge_2df=bool(merge_2df and have_f))


def to_basis(name: str, x: np.ndarray) -> np.ndarray:
    if name == "PX":
        return np.asarray(x, dtype=np.complex128) if np.iscomplexobj(x) else np.asarray(x, np.float64)
    if name == "RF":
        return _fftx(x)
    if name == "2DF":
        return _fft2(x)
    raise ValueError(name)


def from_basis(name: str, X: np.ndarray) -> np.ndarray:
    if name == "PX":
        return np.real(X)
    if name == "RF":
        return np.real(_ifftx(X))
    if name == "2DF":
        return np.real(_ifft2(X))
    raise ValueError(name)


def _link_mean(A, a, B, b):
    """Mean of x for the Gaussian terms (x-a)^2/A + (x-b)^2/B, i.e.
    (A^-1 + B^-1)^-1 (A^-1 a + B^-1 b) = (B a + A b) / (A + B), the form of
    every update in eqs. (ew_t), (2mess_t1)-(2mess_t0).  A = inf gives b
    (a masked pixel, Sec. 3.3); A = 0 gives a."""
    A = np.asarray(A, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        x = (B * a + A * b) / (A + B)
    if np.any(np.isinf(A)):
        x = np.where(np.isinf(A), b, x)
    return x


# ----------------------------------------------------------------------------
# the messenger iteration
# ----------------------------------------------------------------------------

class Chain:
    """State and sweep of the K-part messenger chain.

    Fields (all kept as real pixel-space maps between updates):
      s, t[i] (messenger of part i), dd[i] (the data-like field on the data
      side of part i; dd[K-1] is the data d itself).
    Chain (Appendix A, eq. 2mess_prob, generalised):
      s -T_0- t_0 -Nbar_0- d_0 -T_1- t_1 -Nbar_1- d_1 ... -T_{K-1}- t_{K-1} -Nbar_{K-1}- d
    """

    def __init__(self, P: Parts):
        self.P = P
        K = len(P.parts)
        z = np.zeros((P.ny, P.nx))
        self.s = z.copy()
        self.t = [z.copy() for _ in range(K)]
        self.dd = [z.copy() for _ in range(K - 1)] + [P.d]
        self.iters = 0

    @property
    def K(self):
        return len(self.P.parts)

    def T(self, i, lam):
        return lam * self.P.parts[i].tau

    def sweep(self, lam: float, on_update=None) -> None:
        """One iteration: eqs. (2mess_t1), (2mess_d0), (2mess_t0), (2mess_s),
        generalised, from the data end to the signal: t_{K-1}, d_{K-2}, ...,
        t_0, s.  Each update is computed in the basis where its covariances
        are diagonal (Sec. 2).

        With ``merge_2df`` the last three updates are replaced by the joint
        conditional mean of (s, t_0, d_0) given t_1 -- possible because S and
        the 2DF part share a basis (Appendix A: the t_0 updates can be combined
        there, and s = (S^-1 + N_0^-1)^-1 N_0^-1 d_0).  Marginalising t_0
        leaves s -N_0- d_0 -T_1- t_1, so
            d_0 = (C + N_0) / (C + N_0 + T_1) t_1,   s = C / (C + N_0) d_0.
        """
        if self.P.merge_2df:
            return self._sweep_merged(lam, on_update)
        P = self.P
        for i in range(self.K - 1, -1, -1):
            part = P.parts[i]
            b = part.name
            data_side = self.dd[i]
            sig_side = self.dd[i - 1] if i > 0 else self.s
            # t_i: link Nbar_i to the data side, link T_i to the signal side
            t = _link_mean(part.Nbar, to_basis(b, data_side), self.T(i, lam), to_basis(b, sig_side))
            self.t[i] = from_basis(b, t)
            if on_update is not None:
                on_update(f"t{i}")
            if i > 0:
                prev = P.parts[i - 1]
                pb = prev.name
                # d_{i-1}: link T_i to t_i, link Nbar_{i-1} to t_{i-1}
                dprev = _link_mean(self.T(i, lam), to_basis(pb, self.t[i]), prev.Nbar,
                                   to_basis(pb, self.t[i - 1]))
                self.dd[i - 1] = from_basis(pb, dprev)
                if on_update is not None:
                    on_update(f"d{i - 1}")
        # eq. (2mess_s): s = (S^-1 + T_0^-1)^-1 T_0^-1 t_0, in 2D Fourier space
        T0 = self.T(0, lam)
        self.s = from_basis("2DF", P.C / (P.C + T0) * to_basis("2DF", self.t[0]))
        self.iters += 1
        if on_update is not None:
            on_update("s")

    def _sweep_merged(self, lam: float, on_update=None) -> None:
        P = self.P
        for i in range(self.K - 1, 0, -1):
            part = P.parts[i]
            b = part.name
            t = _link_mean(part.Nbar, to_basis(b, self.dd[i]), self.T(i, lam), to_basis(b, self.dd[i - 1]))
            self.t[i] = from_basis(b, t)
            if on_update is not None:
                on_update(f"t{i}")
            if i > 1:
                prev = P.parts[i - 1]
                pb = prev.name
                dprev = _link_mean(self.T(i, lam), to_basis(pb, self.t[i]), prev.Nbar,
                                   to_basis(pb, self.t[i - 1]))
                self.dd[i - 1] = from_basis(pb, dprev)
                if on_update is not None:
                    on_update(f"d{i - 1}")
        N0 = P.parts[0].N
        T1 = self.T(1, lam)
        D0 = (P.C + N0) / (P.C + N0 + T1) * to_basis("2DF", self.t[1])
        self.dd[0] = from_basis("2DF", D0)
        self.s = from_basis("2DF", P.C / (P.C + N0) * D0)
        # t_0 is marginalised; keep the field defined as s (its T_0 = 0 limit)
        self.t[0] = self.s
        self.iters += 1
        if on_update is not None:
            on_update("s")

    # --- augmented objective (Appendix A, eq. 2mess_prob) ------------------
    def chi2_aug(self, lam: float) -> float:
        P = self.P
        tot = _quad("2DF", self.s, 1.0 / P.C)
        if P.merge_2df:
            # t_0 marginalised: s -N_0- d_0 replaces s -T_0- t_0 -Nbar_0- d_0
            with np.errstate(divide="ignore"):
                w0 = np.where(P.parts[0].N > 0, 1.0 / P.parts[0].N, 0.0)
            tot += _quad("2DF", self.dd[0] - self.s, w0)
        for i, part in enumerate(P.parts):
            if P.merge_2df and i == 0:
                continue
            sig_side = self.dd[i - 1] if i > 0 else self.s
            tot += _quad("PX", self.t[i] - sig_side, np.full((P.ny, P.nx), 1.0 / self.T(i, lam)))
            # Nbar = inf (masked) contributes nothing; Nbar = 0 pins d = t
            # exactly, so its term is 0 as well.
            with np.errstate(divide="ignore"):
                w = np.where(np.isinf(part.Nbar) | (part.Nbar <= 0), 0.0, 1.0 / part.Nbar)
            tot += _quad(part.name, self.dd[i] - self.t[i], w)
        return tot


def chi2_aug_state(chain: "Chain", lam: float) -> float:
    """The augmented objective (Appendix A, eq. 2mess_prob) of the fields a
    GPU plan keeps, with the two it does not keep at their conditional means:
    s given d_0 (merged 2DF block: s = C/(C + N_0) d_0, which the merged
    sweep already holds) and, when a stripe part sits between them, the pixel
    messenger given its neighbours d_RF and d,
        t_PX = (T_PX d + Nbar_PX d_RF) / (Nbar_PX + T_PX)   (d_RF on masked pixels).
    Minimising over one field cannot raise the objective, so this is at most
    chain.chi2_aug(lam), with equality at the fixed point."""
    P = chain.P
    c = Chain(P)
    c.s = chain.s.copy()
    c.t = [t.copy() for t in chain.t]
    c.dd = [d.copy() for d in chain.dd]
    if P.merge_2df:
        N0 = P.parts[0].N
        c.s = from_basis("2DF", P.C / (P.C + N0) * to_basis("2DF", c.dd[0]))
        c.t[0] = c.s
    names = [part.name for part in P.parts]
    if "RF" in names and names[-1] == "PX":
        i = len(names) - 1
        c.t[i] = _link_mean(P.parts[i].Nbar, c.dd[i], c.T(i, lam), c.dd[i - 1])
    return c.chi2_aug(lam)


def _quad(basis: str, x: np.ndarray, w: np.ndarray) -> float:
    """x^T A x for A diagonal in ``basis`` with eigenvalues w (Parseval)."""
    if basis == "PX":
        return float(np.sum(w * x * x))
    X = to_basis(basis, x)
    n = x.shape[1] if basis == "RF" else x.size
    return float(np.sum(w * np.abs(X) ** 2) / n)


# ----------------------------------------------------------------------------
# operators, residual, chi2
# ----------------------------------------------------------------------------

def apply_Sinv(P: Parts, s: np.ndarray) -> np.ndarray:
    return from_basis("2DF", to_basis("2DF", s) / P.C)


def apply_S(P: Parts, x: np.ndarray) -> np.ndarray:
    return from_basis("2DF", to_basis("2DF", x) * P.C)


def apply_N(P: Parts, x: np.ndarray) -> np.ndarray:
    """N x for N = N_1f + N_stripe + diag(pixel_var) with the ORIGINAL parts;
    x must vanish at masked pixels and the result is meaningful only on
    unmasked pixels."""
    y = P.var * x
    if P.N0_full is not None:
        y = y + from_basis("2DF", to_basis("2DF", x) * P.N0_full)
    if P.N1_full is not None:
        y = y + from_basis("RF", to_basis("RF", x) * P.N1_full)
    return y


def residual_terms(P: Parts, s: np.ndarray):
    """Delta d of Sec. 2 for a masked sky.

    g = S^-1 s.  With N^-1 := P^T (P N P^T)^-1 P the literal residual
    r = S^-1 s - N^-1 (d - s) splits into r_masked = g_masked and
    N_uu r_u = rho_u = [N (P^T P g) + s - d]_u, which is Delta d = (I + N S^-1) s - d
    restricted to unmasked pixels.  Returns (rho_u, g_masked, g) as full maps
    (zeros off their support)."""
    g = apply_Sinv(P, s)
    um = P.unmasked
    gp = np.where(um, g, 0.0)
    rho = np.where(um, apply_N(P, gp) + s - P.d, 0.0)
    gm = np.where(um, 0.0, g)
    return rho, gm, g


def rel_terms(P: Parts, s: np.ndarray):
    rho, gm, g = residual_terms(P, s)
    du = np.linalg.norm(P.d[P.unmasked])
    rel_u = float(np.linalg.norm(rho) / du)
    gn = float(np.linalg.norm(g))
    rel_m = float(np.linalg.norm(gm) / gn) if gn > 0 else 0.0
    return rel_u, rel_m, float(np.sum(rho * rho))


# ----------------------------------------------------------------------------
# schedules and the driver
# ----------------------------------------------------------------------------

def cooling_levels(lam_hi: float, nlev: int):
    """nlev levels geometric from lam_hi down to exactly 1."""
    if nlev <= 1:
        return [1.0]
    return [float(lam_hi ** ((nlev - 1 - j) / (nlev - 1))) for j in range(nlev)]


def fixed_schedule(lams: Sequence[float], iters: Sequence[int]):
    return dict(mode="fixed", lam=list(map(float, lams)), iters=list(map(int, iters)))


def messenger_solve(prob, *, theta=DEFAULT_THETA, split_f=DEFAULT_SPLIT_F, split_w=0.0,
                    schedule=None, tol=1e-6, residual_every=10, max_iters=20000,
                    n_iters: Optional[int] = None, P: Optional[Parts] = None,
                    trace: bool = False, merge_2df: bool = False, split_fp: float = 0.0):
    """Run the messenger iteration (Sec. 2) with a cooling schedule.

    schedule: dict(mode="fixed", lam=[...], iters=[...]) -- each level j runs
    iters[j] iterations at lam[j] (levels change only at residual checkpoints,
    every ``residual_every`` iterations), then lambda = 1 until convergence;
    or dict(mode="adaptive", lam0, ratio, expo, snap) -- the rule of Sec. 3.3.
    Converged when lambda == 1 and ||rho_u||/||d_u|| <= tol and
    ||g_masked||/||g|| <= tol at a checkpoint.
    ``n_iters`` runs exactly that many iterations and ignores tol.
    """
    if P is None:
        P = build_parts(prob, theta, split_f, split_w, merge_2df, split_fp)
    ch = Chain(P)
    if schedule is None:
        schedule = dict(mode="adaptive", **ADAPTIVE_DEFAULT)
    R = max(1, int(residual_every))
    mode = schedule["mode"]
    if mode == "fixed":
        levels = list(zip(schedule["lam"], schedule["iters"]))
        if not levels or levels[-1][0] != 1.0:
            levels.append((1.0, 0))
        lev = 0
        lam = levels[0][0]
    else:
        lam = float(schedule["lam0"])
    in_level = 0
    prev_rho2 = None
    log = []
    status = "maxiter"
    limit = n_iters if n_iters is not None else max_iters
    rel_u = rel_m = float("nan")
    while ch.iters < limit:
        ch.sweep(lam)
        in_level += 1
        if ch.iters % R != 0:
            continue
        rel_u, rel_m, rho2 = rel_terms(P, ch.s)
        if trace:
            log.append(dict(it=ch.iters, lam=lam, rel_u=rel_u, rel_m=rel_m))
        if n_iters is None and lam == 1.0 and rel_u <= tol and rel_m <= tol:
            status = "converged"
            break
        if mode == "fixed":
            if lev < len(levels) - 1 and in_level >= levels[lev][1]:
                lev += 1
                lam = levels[lev][0]
                in_level = 0
        else:
            if lam > 1.0:
                if prev_rho2 is not None and prev_rho2 > 0 and rho2 > 0:
                    rate = abs(1.0 - (rho2 / prev_rho2) ** (1.0 / R))
                    if rate < schedule["ratio"]:
                        lam = lam ** schedule["expo"]
                        if lam < schedule["snap"]:
                            lam = 1.0
                        in_level = 0
                        prev_rho2 = None
                        continue
                prev_rho2 = rho2
    if n_iters is not None:
        status = "fixed"
    return dict(s=ch.s, iters=ch.iters, lam=lam, status=status, rel_u=rel_u,
                rel_m=rel_m, chain=ch, parts=P, log=log)


# ----------------------------------------------------------------------------
# dense definition (tiny maps)
# ----------------------------------------------------------------------------

def dense_cov_stationary(spec_full: np.ndarray) -> np.ndarray:
    """Dense covariance of a stationary field with eigenvalues spec_full:
    N[p, q] = c(y_p - y_q, x_p - x_q), c = inverse DFT of the spectrum
    (computed by brute-force DFT sums)."""
    ny, nx = spec_full.shape
    c = np.real(brute_idft(brute_idft(spec_full, axis=0), axis=1))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    yy = yy.ravel()
    xx = xx.ravel()
    return c[(yy[:, None] - yy[None, :]) % ny, (xx[:, None] - xx[None, :]) % nx]


def dense_cov_stripes(Pst_full: np.ndarray, a2: np.ndarray, ny: int) -> np.ndarray:
    """Dense covariance of independent rows, each stationary along x with
    eigenvalues Pst_full and scaled by a(y)^2."""
    nx = Pst_full.shape[0]
    c = np.real(brute_idft(Pst_full))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    yy = yy.ravel()
    xx = xx.ravel()
    same = yy[:, None] == yy[None, :]
    return np.where(same, a2[yy][:, None] * c[(xx[:, None] - xx[None, :]) % nx], 0.0)


def dense_matrices(prob):
    d = np.asarray(prob.d, np.float64)
    ny, nx = d.shape
    C = full_from_half(prob.C, nx)
    S = dense_cov_stationary(C)
    Sinv = dense_cov_stationary(1.0 / C)
    N = np.diag(np.asarray(prob.pixel_var, np.float64).ravel())
    if prob.P1f is not None:
        N = N + dense_cov_stationary(full_from_half(prob.P1f, nx))
    if prob.Pst is not None:
        a2 = np.ones(ny) if prob.stripe_amp2 is None else np.asarray(prob.stripe_amp2, np.float64)
        N = N + dense_cov_stripes(full_stripe(prob.Pst, nx), a2, ny)
    um = np.ones(ny * nx, bool) if prob.mask is None else ~np.asarray(prob.mask).astype(bool).ravel()
    return S, Sinv, N, um


def dense_wf(prob, return_parts: bool = False):
    """Eq. (wiener): s = (S^-1 + N^-1)^-1 N^-1 d with N^-1 = P^T N_uu^-1 P,
    both inverses by Cholesky."""
    from scipy.linalg import cho_factor, cho_solve
    S, Sinv, N, um = dense_matrices(prob)
    d = np.asarray(prob.d, np.float64).ravel()
    n = d.size
    Nuu = N[np.ix_(um, um)]
    cf = cho_factor(Nuu)
    Ninv = np.zeros((n, n))
    Ninv[np.ix_(um, um)] = cho_solve(cf, np.eye(um.sum()))
    A = Sinv + Ninv
    b = Ninv @ d
    s = cho_solve(cho_factor(A), b)
    s = s.reshape(np.asarray(prob.d).shape)
    if return_parts:
        return s, dict(S=S, Sinv=Sinv, N=N, Ninv=Ninv, um=um, A=A, b=b)
    return s


def inverse_noise_dense(prob) -> np.ndarray:
    """N^-1 d by its definition (Sec. 4, the S = alpha I remark computes it
    approximately): with a mask, P^T (P N P^T)^-1 P d, zero on masked pixels;
    dense Cholesky (tiny maps only)."""
    from scipy.linalg import cho_factor, cho_solve
    _, _, N, um = dense_matrices(prob)
    d = np.asarray(prob.d, np.float64).ravel()
    out = np.zeros(d.size)
    out[um] = cho_solve(cho_factor(N[np.ix_(um, um)]), d[um])
    return out.reshape(np.asarray(prob.d).shape)


def dense_wf_alt(prob):
    """Eq. (wiener-alt) on the unmasked pixels: s = S P^T (P (S + N) P^T)^-1 P d."""
    from scipy.linalg import cho_factor, cho_solve
    S, _, N, um = dense_matrices(prob)
    d = np.asarray(prob.d, np.float64).ravel()
    x = cho_solve(cho_factor((S + N)[np.ix_(um, um)]), d[um])
    return (S[:, um] @ x).reshape(np.asarray(prob.d).shape)


def closed_form(prob) -> np.ndarray:
    """Homogeneous noise (uniform pixel_var, no mask, a(y) = 1): all parts are
    diagonal in 2D Fourier space and s_k = C_k / (C_k + N_k) d_k (Sec. 3.1)."""
    d = np.asarray(prob.d, np.float64)
    ny, nx = d.shape
    var = np.asarray(prob.pixel_var, np.float64)
    assert prob.mask is None or not np.asarray(prob.mask).any()
    assert np.allclose(var, var.flat[0], rtol=1e-6)
    assert prob.stripe_amp2 is None or np.allclose(prob.stripe_amp2, 1.0)
    C = full_from_half(prob.C, nx)
    Nk = np.full((ny, nx), float(var.flat[0]))
    if prob.P1f is not None:
        Nk = Nk + full_from_half(prob.P1f, nx)
    if prob.Pst is not None:
        Nk = Nk + full_stripe(prob.Pst, nx)[None, :]
    return np.real(np.fft.ifft2(C / (C + Nk) * np.fft.fft2(d)))


def chi2(prob, s, Ninv=None, P: Optional[Parts] = None) -> float:
    """chi^2(s) = s^T S^-1 s + (d - s)^T N^-1 (d - s) (Sec. 1), with the
    masked N^-1; dense Ninv if given, else conjugate gradients."""
    s = np.asarray(s, np.float64)
    if P is None:
        P = build_parts(prob)
    r = P.d - s
    t1 = float(np.sum(s * apply_Sinv(P, s)))
    if Ninv is not None:
        rv = np.where(P.unmasked, r, 0.0).ravel()
        return t1 + float(rv @ Ninv @ rv)
    x = _solve_Nuu(P, np.where(P.unmasked, r, 0.0), 1e-13)
    return t1 + float(np.sum(np.where(P.unmasked, r, 0.0) * x))


# ----------------------------------------------------------------------------
# conjugate gradients (full-size checks)
# ----------------------------------------------------------------------------

def pcg(apply_A, b, apply_Minv=None, tol=1e-12, maxiter=20000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel), FP64."""
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_Minv(r) if apply_Minv else r
    p = z.copy()
    rz = float(np.sum(r * z))
    bn = float(np.linalg.norm(b))
    if bn == 0:
        return x, 0
    for it in range(1, maxiter + 1):
        Ap = apply_A(p)
        alpha = rz / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        if float(np.linalg.norm(r)) <= tol * bn:
            return x, it
        z = apply_Minv(r) if apply_Minv else r
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    raise RuntimeError(f"pcg: no convergence in {maxiter} iterations")


def _hom_noise_spectrum(P: Parts) -> np.ndarray:
    v = float(np.mean(P.var[P.unmasked]))
    Nk = np.full((P.ny, P.nx), v)
    if P.N0_full is not None:
        Nk = Nk + P.N0_full
    if P.N1_full is not None:
        Nk = Nk + np.mean(P.N1_full, axis=0)[None, :]
    return Nk


def _solve_Nuu(P: Parts, b: np.ndarray, tol: float) -> np.ndarray:
    """x with x_m = 0 and (N x)_u = b_u (N_uu^-1 b), by PCG."""
    um = P.unmasked
    Nk = _hom_noise_spectrum(P)

    def A(x):
        return np.where(um, apply_N(P, np.where(um, x, 0.0)), 0.0)

    def Minv(r):
        return np.where(um, from_basis("2DF", to_basis("2DF", r) / Nk), 0.0)

    x, _ = pcg(A, np.where(um, b, 0.0), Minv, tol=tol)
    return x


def literal_residual(prob, s, P: Optional[Parts] = None, tol: float = 1e-12):
    """|| (S^-1 + N^-1) s - N^-1 d || / || N^-1 d || with N^-1 = P^T N_uu^-1 P
    (Sec. 1 eq. wiener; Sec. 2 on why N^-1 needs an iterative solve)."""
    if P is None:
        P = build_parts(prob)
    s = np.asarray(s, np.float64)
    g = apply_Sinv(P, s)
    ninv_r = _solve_Nuu(P, np.where(P.unmasked, P.d - s, 0.0), tol)
    ninv_d = _solve_Nuu(P, P.d, tol)
    r = g - ninv_r
    return float(np.linalg.norm(r) / np.linalg.norm(ninv_d))


def pcg_wf(prob, P: Optional[Parts] = None, tol: float = 1e-11) -> np.ndarray:
    """Wiener solution by eq. (wiener-alt) on unmasked pixels:
    (S_uu + N_uu) x = d_u, s = S P^T x, by PCG with a 2D-Fourier diagonal
    preconditioner."""
    if P is None:
        P = build_parts(prob)
    um = P.unmasked
    Nk = _hom_noise_spectrum(P) + P.C

    def A(x):
        xz = np.where(um, x, 0.0)
        return np.where(um, apply_S(P, xz) + apply_N(P, xz), 0.0)

    def Minv(r):
        return np.where(um, from_basis("2DF", to_basis("2DF", r) / Nk), 0.0)

    x, _ = pcg(A, np.where(um, P.d, 0.0), Minv, tol=tol)
    return apply_S(P, np.where(um, x, 0.0))


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
