"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a brute-force DFT, an eigen-decomposition, a covariance written out
as a sum, a closed form, a second formula for the same solution, or an
invariant the mathematics fixes (Huffenberger 2017, Sec. 1-3, Appendix A)."""

import numpy as np
import pytest

import oracle as O
from paper_1704_00865_gb300 import synth


# Tiny maps with flattened 1/f and stripe spectra (knees at 2 cycles per map)
# converge in a few thousand sweeps, which keeps the CPU suite short while
# exercising every part, the mask and per-row stripe amplitudes.
def _prob(n=12, seed=3, **kw):
    kw.setdefault("mask_frac", 0.06)
    kw.setdefault("k_knee", 2.0)
    kw.setdefault("k_knee_x", 2.0)
    return synth.make_problem(n, n, seed, **kw)


def _rect(ny=8, nx=12, seed=5, **kw):
    kw.setdefault("mask_frac", 0.06)
    kw.setdefault("k_knee", 2.0)
    kw.setdefault("k_knee_x", 2.0)
    return synth.make_problem(ny, nx, seed, **kw)


SCHED = O.fixed_schedule(O.cooling_levels(1e2, 5), [10] * 5)


def _converged(p, tol=1e-10, **kw):
    r = O.messenger_solve(p, schedule=SCHED, tol=tol, residual_every=10, max_iters=200000, **kw)
    assert r["status"] == "converged"
    return r


# --------------------------------------------------------------- transforms

def test_bases_match_brute_force_dft():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((6, 10))
    X2 = O.to_basis("2DF", x)
    Xb = O.brute_dft(O.brute_dft(x, axis=0), axis=1)
    assert np.abs(X2 - Xb).max() < 1e-12
    Xr = O.to_basis("RF", x)
    assert np.abs(Xr - O.brute_dft(x, axis=1)).max() < 1e-12
    assert np.abs(O.from_basis("2DF", Xb) - x).max() < 1e-12
    assert np.abs(O.from_basis("RF", Xr) - x).max() < 1e-12


def test_full_from_half_is_hermitian_and_matches_rfft_layout():
    rng = np.random.default_rng(1)
    ny, nx = 6, 8
    x = rng.standard_normal((ny, nx))
    # |rfft2(x)|^2 on the half grid must expand to |fft2(x)|^2 on the full grid
    half = np.abs(np.fft.rfft2(x)) ** 2
    full = O.full_from_half(half, nx)
    assert np.allclose(full, np.abs(O.brute_dft(O.brute_dft(x, 0), 1)) ** 2, rtol=1e-12, atol=1e-12)
    assert np.allclose(O.full_stripe(np.arange(nx // 2 + 1.0), nx), [0, 1, 2, 3, 4, 3, 2, 1])


# --------------------------------------------------------------- covariances

def test_dense_stationary_covariance_written_as_a_sum():
    ny, nx = 4, 6
    rng = np.random.default_rng(2)
    half = rng.uniform(0.5, 2.0, (ny, nx // 2 + 1))
    # make the kx=0 and kx=nx/2 columns symmetric in ky (a real covariance)
    for c in (0, nx // 2):
        half[:, c] = 0.5 * (half[:, c] + half[(-np.arange(ny)) % ny, c])
    full = O.full_from_half(half, nx)
    M = O.dense_cov_stationary(full)
    for p in [(0, 0), (1, 2), (3, 5)]:
        for q in [(0, 0), (2, 1), (3, 4)]:
            dy, dx = p[0] - q[0], p[1] - q[1]
            ref = sum(full[ky, kx] * np.cos(2 * np.pi * (ky * dy / ny + kx * dx / nx))
                      for ky in range(ny) for kx in range(nx)) / (ny * nx)
            assert abs(M[p[0] * nx + p[1], q[0] * nx + q[1]] - ref) < 1e-12


def test_dense_covariances_have_the_given_eigenvalues():
    p = _rect(stripe_rows_vary=True)
    ny, nx = p.shape
    N0 = O.dense_cov_stationary(O.full_from_half(p.P1f, nx))
    ev = np.sort(np.linalg.eigvalsh(N0))
    assert np.allclose(ev, np.sort(O.full_from_half(p.P1f, nx).ravel()), rtol=1e-9)
    N1 = O.dense_cov_stripes(O.full_stripe(p.Pst, nx), p.stripe_amp2.astype(float), ny)
    ev1 = np.sort(np.linalg.eigvalsh(N1))
    ref1 = np.sort((p.stripe_amp2.astype(float)[:, None] * O.full_stripe(p.Pst, nx)[None, :]).ravel())
    assert np.allclose(ev1, ref1, rtol=1e-9)
    S, Sinv, _, _ = O.dense_matrices(p)
    assert np.abs(S @ Sinv - np.eye(S.shape[0])).max() < 1e-8


# --------------------------------------------------------------- the solution

def test_closed_form_equals_dense_in_homogeneous_case():
    p = _prob(homogeneous=True, mask_frac=0.0)
    assert O.rel_l2(O.closed_form(p), O.dense_wf(p)) < 1e-11


def test_wiener_and_wiener_alt_agree_with_mask():
    p = _rect(stripe_rows_vary=True)
    assert O.rel_l2(O.dense_wf_alt(p), O.dense_wf(p)) < 1e-11


def test_dense_solution_minimises_chi2():
    p = _prob(stripe_rows_vary=True)
    s, M = O.dense_wf(p, return_parts=True)
    sv = s.ravel()
    d = np.asarray(p.d, np.float64).ravel()
    grad = M["Sinv"] @ sv - M["Ninv"] @ (d - sv)
    assert np.linalg.norm(grad) / np.linalg.norm(M["Ninv"] @ d) < 1e-10
    c0 = O.chi2(p, s, Ninv=M["Ninv"])
    rng = np.random.default_rng(4)
    for _ in range(5):
        delta = rng.standard_normal(s.shape) * 1e-3 * np.std(s)
        assert O.chi2(p, s + delta, Ninv=M["Ninv"]) > c0


def test_chi2_by_conjugate_gradients_equals_the_dense_value():
    # chi2() without a dense N^-1 solves N_uu x = (d - s)_u by CG (the path a
    # full-size map takes); on a tiny masked map with per-row stripe
    # amplitudes it must give the value the dense masked N^-1 gives, at the
    # solution and away from it
    p = _prob(stripe_rows_vary=True)
    s_d, M = O.dense_wf(p, return_parts=True)
    rng = np.random.default_rng(12)
    for s in (s_d, s_d + 1e-2 * np.std(s_d) * rng.standard_normal(s_d.shape), np.zeros_like(s_d)):
        ref = O.chi2(p, s, Ninv=M["Ninv"])
        assert abs(O.chi2(p, s) - ref) / ref < 1e-9, (O.chi2(p, s), ref)


@pytest.mark.parametrize("shape", [(8, 12), (12, 8)])
def test_messenger_converges_to_dense_three_parts_mask_row_amplitudes(shape):
    p = _rect(*shape, stripe_rows_vary=True)
    s_d = O.dense_wf(p)
    assert O.rel_l2(_converged(p)["s"], s_d) < 1e-8


@pytest.mark.parametrize("split_f", [0.5, 1.0])
def test_merged_2df_block_converges_to_dense(split_f):
    # Appendix A: with S and the 1/f part sharing a basis, (s, t_0, d_0) may be
    # updated jointly; the fixed point must not move.
    p = _rect(stripe_rows_vary=True, seed=9)
    s_d = O.dense_wf(p)
    r = _converged(p, merge_2df=True, split_f=split_f)
    assert O.rel_l2(r["s"], s_d) < 1e-8
    # d_0 is then the Wiener estimate of s + n_0 from t_1: s = C/(C + N_0) d_0
    P = r["parts"]
    N0 = P.parts[0].N
    s_from_d0 = O.from_basis("2DF", P.C / (P.C + N0) * O.to_basis("2DF", r["chain"].dd[0]))
    assert O.rel_l2(s_from_d0, r["s"]) < 1e-12


@pytest.mark.parametrize("parts", [dict(one_over_f=False), dict(stripes=False),
                                   dict(one_over_f=False, stripes=False)])
def test_messenger_converges_with_fewer_parts(parts):
    p = _prob(n=8, seed=11, **parts)
    s_d = O.dense_wf(p)
    assert O.rel_l2(_converged(p)["s"], s_d) < 1e-8


def test_ew_converges_in_one_step_when_tau_is_the_white_level():
    # Sec. 3.1: with uniform white noise and tau = sigma^2 the messenger
    # carries all the noise and one iteration gives the exact solution.
    p = _prob(homogeneous=True, mask_frac=0.0, one_over_f=False, stripes=False)
    P = O.build_parts(p, theta=(0.9, 0.9, 1.0))
    ch = O.Chain(P)
    ch.sweep(1.0)
    assert O.rel_l2(ch.s, O.closed_form(p)) < 1e-12


def test_augmented_chi2_never_increases_under_any_single_update():
    # Appendix A: each update is the exact minimiser of eq. (2mess_prob) over
    # one field, so the augmented objective cannot go up at fixed lambda.
    p = _prob(stripe_rows_vary=True)
    for lam, merge in ((30.0, False), (1.0, False), (30.0, True), (1.0, True)):
        P = O.build_parts(p, merge_2df=merge)
        ch = O.Chain(P)
        vals = [ch.chi2_aug(lam)]
        for _ in range(6):
            ch.sweep(lam, on_update=lambda name: vals.append(ch.chi2_aug(lam)))
        v = np.array(vals)
        assert np.all(np.diff(v) <= 1e-9 * np.abs(v[:-1])), np.diff(v).max()
        assert v[-1] < v[0]


def test_augmented_chi2_equals_chi2_at_the_fixed_point():
    # marginalising the messengers (Appendix A) leaves chi^2(s); at the fixed
    # point every messenger sits at its conditional mean, so the minimum of
    # the augmented objective over them is chi^2(s*).
    p = _rect(seed=13)
    s_d, M = O.dense_wf(p, return_parts=True)
    r = _converged(p, tol=1e-11)
    c = O.chi2(p, s_d, Ninv=M["Ninv"])
    assert abs(r["chain"].chi2_aug(1.0) - c) / c < 1e-9


def test_state_chi2_aug_minimises_the_unkept_fields():
    # chi2_aug_state puts s and (with a stripe part) the pixel messenger at
    # their conditional means: never above chi2_aug of the same state, equal
    # to it after a merged sweep without a stripe part (nothing to minimise:
    # the merged sweep already holds s at its mean), equal to chi^2(s*) at
    # the fixed point, and below it when the pixel messenger is perturbed
    for kw in (dict(), dict(stripes=False), dict(one_over_f=False), dict(one_over_f=False, stripes=False)):
        p = _prob(**kw)
        for merge in (True, False):
            P = O.build_parts(p, merge_2df=merge)
            ch = O.Chain(P)
            for _ in range(3):
                ch.sweep(10.0)
            a, b = O.chi2_aug_state(ch, 10.0), ch.chi2_aug(10.0)
            assert a <= b * (1 + 1e-12), (kw, merge, a, b)
            names = [q.name for q in P.parts]
            if P.merge_2df and "RF" not in names:
                assert abs(a - b) <= 1e-12 * b, (kw, a, b)
    p = _prob()
    P = O.build_parts(p, merge_2df=True)
    ch = O.Chain(P)
    for _ in range(3):
        ch.sweep(10.0)
    base = O.chi2_aug_state(ch, 10.0)
    ch.t[-1] = ch.t[-1] + 0.3 * np.random.default_rng(5).standard_normal(ch.t[-1].shape)
    assert O.chi2_aug_state(ch, 10.0) == pytest.approx(base, rel=1e-12)   # t_PX is minimised out
    assert ch.chi2_aug(10.0) > base
    p = _rect(seed=13)
    s_d, M = O.dense_wf(p, return_parts=True)
    r = _converged(p, tol=1e-11)
    c = O.chi2(p, s_d, Ninv=M["Ninv"])
    assert abs(O.chi2_aug_state(r["chain"], 1.0) - c) / c < 1e-9


def test_interior_link_with_theta_one_freezes_a_mode():
    # Reading: tau = the exact minimum eigenvalue of an interior part makes
    # Nbar = 0 on that mode; d_i = t_i is then pinned and never moves.
    p = _prob(n=12, seed=17, mask_frac=0.0, homogeneous=True, stripes=False)
    s_d = O.dense_wf(p)
    r1 = O.messenger_solve(p, theta=(1.0, 1.0, 1.0), schedule=O.fixed_schedule([1.0], [0]),
                           n_iters=3000, residual_every=100)
    r9 = O.messenger_solve(p, theta=(0.9, 0.9, 1.0), schedule=O.fixed_schedule([1.0], [0]),
                           n_iters=3000, residual_every=100)
    assert O.rel_l2(r1["s"], s_d) > 1e-4
    assert O.rel_l2(r9["s"], s_d) < 1e-6


def test_three_part_chain_equals_merged_two_part_chain_when_rows_are_alike():
    # with a(y) = 1 the stripe covariance is also diagonal in 2D Fourier
    # space; merging it into the 1/f part must give the same fixed point.
    p = _rect(seed=19)
    merged = synth.Problem(**{**p.__dict__})
    merged.P1f = p.P1f.astype(np.float64) + p.Pst.astype(np.float64)[None, :]
    merged.Pst = None
    a = _converged(p)["s"]
    b = _converged(merged)["s"]
    assert O.rel_l2(a, b) < 1e-8


def test_reduces_to_single_messenger_as_extra_parts_vanish():
    p = _rect(seed=23)
    ew = synth.Problem(**{**p.__dict__})
    ew.P1f = None
    ew.Pst = None
    s_ew = O.dense_wf(ew)
    errs = []
    for eps in (1e-4, 1e-5, 1e-6):
        q = synth.Problem(**{**p.__dict__})
        q.P1f = p.P1f.astype(np.float64) * eps
        q.Pst = p.Pst.astype(np.float64) * eps
        errs.append(O.rel_l2(O.dense_wf(q), s_ew))
    # O(eps): each decade of eps removes about a decade of difference.  (The
    # messenger itself cannot run at tiny eps: an almost empty part has an
    # almost zero tau, which Sec. 3.1 notes makes the method fail; with the
    # parts omitted the chain is the single-messenger one, pinned above.)
    assert 0.05 < errs[1] / errs[0] < 0.2 and 0.05 < errs[2] / errs[1] < 0.2


def test_masked_data_values_do_not_matter():
    p = _prob(stripe_rows_vary=True)
    q = synth.Problem(**{**p.__dict__})
    q.d = p.d.copy()
    q.d[p.mask.astype(bool)] = 123.0
    assert O.rel_l2(O.dense_wf(q), O.dense_wf(p)) < 1e-12
    sch = O.fixed_schedule([10.0, 1.0], [10, 10])
    a = O.messenger_solve(p, schedule=sch, n_iters=40, residual_every=10)["s"]
    b = O.messenger_solve(q, schedule=sch, n_iters=40, residual_every=10)["s"]
    assert O.rel_l2(a, b) < 1e-13


def test_iteration_is_linear_in_the_data():
    p = _prob(stripe_rows_vary=True)
    q = synth.Problem(**{**p.__dict__})
    q.d = np.roll(p.s_true, 3, axis=1).astype(np.float64)
    r = synth.Problem(**{**p.__dict__})
    r.d = 2.0 * p.d.astype(np.float64) - 0.5 * q.d
    sch = O.fixed_schedule([10.0, 1.0], [10, 10])
    a = O.messenger_solve(p, schedule=sch, n_iters=30, residual_every=10)["s"]
    b = O.messenger_solve(q, schedule=sch, n_iters=30, residual_every=10)["s"]
    c = O.messenger_solve(r, schedule=sch, n_iters=30, residual_every=10)["s"]
    assert O.rel_l2(c, 2.0 * a - 0.5 * b) < 1e-12


def test_homogeneous_problem_is_shift_equivariant():
    p = _rect(homogeneous=True, mask_frac=0.0)
    q = synth.Problem(**{**p.__dict__})
    q.d = np.roll(p.d, (2, 5), axis=(0, 1))
    sch = O.fixed_schedule([10.0, 1.0], [10, 10])
    a = O.messenger_solve(p, schedule=sch, n_iters=25, residual_every=5)["s"]
    b = O.messenger_solve(q, schedule=sch, n_iters=25, residual_every=5)["s"]
    assert np.abs(np.roll(a, (2, 5), axis=(0, 1)) - b).max() < 1e-12 * np.abs(a).max()


# --------------------------------------------------------------- residuals

def test_residual_terms_are_the_literal_residual_times_N():
    p = _prob(stripe_rows_vary=True)
    s_d, M = O.dense_wf(p, return_parts=True)
    rng = np.random.default_rng(6)
    s = s_d + 1e-3 * np.std(s_d) * rng.standard_normal(s_d.shape)
    rho, gm, g = O.residual_terms(O.build_parts(p), s)
    d = np.asarray(p.d, np.float64).ravel()
    r = M["Sinv"] @ s.ravel() - M["Ninv"] @ (d - s.ravel())
    um = M["um"]
    Nuu = M["N"][np.ix_(um, um)]
    assert np.allclose(Nuu @ r[um], rho.ravel()[um], rtol=1e-9, atol=1e-12 * np.abs(rho).max())
    assert np.allclose(r[~um], gm.ravel()[~um], rtol=1e-9, atol=1e-12 * np.abs(gm).max())


def test_cg_literal_residual_and_cg_solution_match_dense():
    p = _prob(stripe_rows_vary=True)
    s_d, M = O.dense_wf(p, return_parts=True)
    rng = np.random.default_rng(8)
    s = s_d + 1e-4 * np.std(s_d) * rng.standard_normal(s_d.shape)
    d = np.asarray(p.d, np.float64).ravel()
    r = M["Sinv"] @ s.ravel() - M["Ninv"] @ (d - s.ravel())
    ref = np.linalg.norm(r) / np.linalg.norm(M["Ninv"] @ d)
    assert abs(O.literal_residual(p, s) - ref) / ref < 1e-7
    assert O.rel_l2(O.pcg_wf(p), s_d) < 1e-9
    assert O.literal_residual(p, s_d) < 1e-9


# --------------------------------------------------------------- cooling rule

def test_adaptive_rule_lowers_lambda_by_the_paper_power_to_exactly_one():
    p = _rect(seed=29)
    r = O.messenger_solve(p, schedule=dict(mode="adaptive", **O.ADAPTIVE_DEFAULT), tol=1e-8,
                          residual_every=1, max_iters=400000, trace=True)
    lams = []
    for e in r["log"]:
        if not lams or e["lam"] != lams[-1]:
            lams.append(e["lam"])
    assert lams[0] == 5e5 and lams[-1] == 1.0
    for a, b in zip(lams[:-2], lams[1:-1]):
        assert abs(b - a ** 0.7) < 1e-9 * b
    assert lams[-2] ** 0.7 < 1.01
    assert r["status"] == "converged"


def test_fixed_schedule_levels_and_paper_constants():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    assert O.ADAPTIVE_DEFAULT["lam0"] == g["cooling_lambda_start"]["value"]
    assert O.ADAPTIVE_DEFAULT["ratio"] == g["cooling_plateau_fraction"]["value"]
    assert O.ADAPTIVE_DEFAULT["expo"] == g["cooling_exponent"]["value"]
    lv = O.cooling_levels(1e3, 20)
    assert lv[0] == 1e3 and lv[-1] == 1.0 and len(lv) == 20


# --------------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("mutation", ["swap_link", "mask_takes_data", "transpose_rf"])
def test_pins_catch_planted_mistakes(monkeypatch, mutation):
    """A plausible slip planted in the oracle must break the dense pin."""
    p = _rect(ny=8, nx=12, seed=31, stripe_rows_vary=True)
    s_d = O.dense_wf(p)
    import oracle.wf_oracle as W
    if mutation == "swap_link":
        orig = W._link_mean
        monkeypatch.setattr(W, "_link_mean", lambda A, a, B, b: orig(B, a, A, b))
    elif mutation == "mask_takes_data":
        orig = W._link_mean

        def wrong(A, a, B, b):
            x = orig(A, a, B, b)
            A = np.asarray(A, dtype=np.float64)
            return np.where(np.isinf(A), a, x) if np.any(np.isinf(A)) else x
        monkeypatch.setattr(W, "_link_mean", wrong)
    else:
        orig_to, orig_from = W.to_basis, W.from_basis

        def to_b(name, x):
            if name == "RF":
                return np.fft.fft(x, axis=0)
            return orig_to(name, x)

        def from_b(name, X):
            if name == "RF":
                return np.real(np.fft.ifft(X, axis=0))
            return orig_from(name, X)
        monkeypatch.setattr(W, "to_basis", to_b)
        monkeypatch.setattr(W, "from_basis", from_b)
    r = W.messenger_solve(p, schedule=W.fixed_schedule([30.0, 3.0], [20, 20]), tol=1e-12,
                          residual_every=10, max_iters=20000)
    assert r["status"] != "converged" or W.rel_l2(r["s"], s_d) > 1e-6


def test_inverse_noise_weighting_definition():
    # white noise only: N is diagonal, N^-1 d = d / pixel_var on unmasked pixels
    prob = synth.make_problem(16, 16, 71, one_over_f=False, stripes=False, mask_frac=0.1)
    w = O.inverse_noise_dense(prob)
    m = prob.mask.astype(bool)
    assert np.allclose(w[~m], prob.d[~m].astype(np.float64) / prob.pixel_var[~m], rtol=1e-12)
    assert np.all(w[m] == 0.0)
    # all parts: N (N^-1 d) = d on the unmasked pixels, and the S = alpha I
    # Wiener filter divided by alpha approaches it at rate alpha
    prob = synth.make_problem(16, 16, 72, mask_frac=0.1, k_knee=4.0, k_knee_x=4.0)
    w = O.inverse_noise_dense(prob)
    _, _, N, um = O.dense_matrices(prob)
    assert np.allclose((N[np.ix_(um, um)] @ w.ravel()[um]), prob.d.ravel()[um].astype(np.float64), rtol=1e-9)
    errs = []
    lmin = np.linalg.eigvalsh(N[np.ix_(um, um)]).min()
    for alpha in (1e-2 * lmin, 1e-3 * lmin):
        q = synth.make_problem(16, 16, 72, mask_frac=0.1, k_knee=4.0, k_knee_x=4.0)
        q.C[...] = alpha
        errs.append(np.linalg.norm(O.dense_wf(q) / alpha - w) / np.linalg.norm(w))
    assert errs[0] < 2e-2 and errs[1] < 2e-3 and errs[1] < 0.2 * errs[0]
