"""Pins of the oracle's shift-variant preconditioner, this project's form of
the one Sec. 5 mentions (approximating D = (tau A A^T + W^-1)^-1 of Eq. 23
better than Eq. 24, with no published details):

    D = T_lo + S T_hi S,   S = diag(sqrt(kappa w)),

T_lo and T_hi the convolutions with the taps of the low and high bands
H_lo + H_hi = H (Eq. 24).  Pinned against the paper's equations and the
mathematics: the bands add up to Eq. 24; the low band tends to the pure ramp
of Eq. 32 (the FBP filter) at low frequency; with uniform variances the form
is Eq. 24 exactly; as tau -> 0 it tends to W, the tau -> 0 limit of Eq. 23;
it is symmetric positive definite; and the Theorem of Sec. 2.2 holds: the
iteration converges to the same minimiser as with Eq. 24."""
import math

import numpy as np

import oracle as O
import synth


def full_period(t, half, P):
    per = np.zeros(P)
    for k in range(-(half - 1), half):
        per[k % P] = t[half - 1 + k]
    per[P // 2] = t[half - 1 + P // 2]
    return per


def test_bands_add_up_to_smoothed_ramp():
    B, V, tau, kappa = 95, 90, 0.3, 0.02
    t0 = O.ramp_taps(0, V, B, tau, kappa)
    t2 = O.ramp_taps(2, V, B, tau, kappa)
    t3 = O.ramp_taps(3, V, B, tau, kappa)
    np.testing.assert_allclose(t2 + t3, t0, rtol=0, atol=1e-13 * np.abs(t0).max())


def test_band_responses_limits():
    # over a full period: the low band approaches the pure ramp |w|/(2 m tau)
    # (Eq. 32) as w -> 0, the high band vanishes there and approaches
    # 1/kappa = the high-frequency limit of Eq. 24 as 2 m tau / kappa -> 0
    B, V, tau, kappa = 95, 90, 1e-4, 0.02
    P = O.fft_len(B)
    half = P // 2 + 1
    j = np.arange(P)
    w = 2 * math.pi * np.minimum(j, P - j) / P
    lo = np.fft.fft(full_period(O.ramp_taps(2, V, B, tau, kappa, half=half, period=P), half, P)).real
    hi = np.fft.fft(full_period(O.ramp_taps(3, V, B, tau, kappa, half=half, period=P), half, P)).real
    ramp = np.fft.fft(full_period(O.ramp_taps(1, V, B, tau, 0.0, half=half, period=P), half, P)).real
    assert abs(lo[0]) < 1e-12 and abs(hi[0]) < 1e-12
    # w_1 = 2 pi / P: 2 m tau / (kappa w_1) = 0.73; a looser tau makes the low band the ramp
    t_small = 1.0
    lo_s = np.fft.fft(full_period(O.ramp_taps(2, V, B, t_small, kappa, half=half, period=P), half, P)).real
    ramp_s = np.fft.fft(full_period(O.ramp_taps(1, V, B, t_small, 0.0, half=half, period=P), half, P)).real
    assert abs(lo_s[1] / ramp_s[1] - 1.0) < 2 * kappa * w[1] / (2 * V * t_small)
    # tiny tau: the high band is 1/kappa at every non-zero frequency
    hi_t = np.fft.fft(full_period(O.ramp_taps(3, V, B, 1e-12, kappa, half=half, period=P), half, P)).real
    np.testing.assert_allclose(hi_t[1:], 1.0 / kappa, rtol=1e-6)
    for r in (lo, hi, ramp):
        assert np.all(r >= -1e-12 * r.max())


def test_uniform_variance_gives_eq24():
    V, B, tau = 6, 41, 0.05
    kappa = 0.01
    w = np.full((V, B), 1.0 / kappa)
    s = O.shift_variant_scale(w)
    np.testing.assert_allclose(s, 1.0, rtol=1e-15)
    y = synth.random_sinogram(V, B, 7)
    d_sv = O.apply_d(y, O.ramp_taps(2, 60, B, tau, kappa), O.ramp_taps(3, 60, B, tau, kappa), s)
    d_24 = O.filt(y, O.ramp_taps(0, 60, B, tau, kappa))
    np.testing.assert_allclose(d_sv, d_24, rtol=0, atol=1e-12 * np.abs(d_24).max())


def test_tends_to_w_as_tau_vanishes():
    # Eq. 23 with tau -> 0 is D = W.  The high band tends to (1/kappa)(1 - [w = 0]),
    # whose taps are (1/kappa)(delta_k - 1/P): D y -> w y - s (s . y) / (kappa P) per view
    V, B = 4, 37
    rng = np.random.default_rng(3)
    w = rng.uniform(20.0, 400.0, (V, B))
    s = O.shift_variant_scale(w)
    kappa = float(np.mean(1 / w))
    P = O.fft_len(B)
    y = synth.random_sinogram(V, B, 4)
    d = O.apply_d(y, O.ramp_taps(2, 30, B, 1e-13, kappa), O.ramp_taps(3, 30, B, 1e-13, kappa), s)
    ref = w * y - s * np.sum(s * y, axis=1, keepdims=True) / (kappa * P)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-7 * np.abs(ref).max())


def test_symmetric_positive_definite():
    V, B, tau = 1, 31, 0.02
    rng = np.random.default_rng(9)
    w = rng.uniform(10.0, 1000.0, (V, B))
    s = O.shift_variant_scale(w)
    kappa = float(np.mean(1 / w))
    tl, th = O.ramp_taps(2, 40, B, tau, kappa), O.ramp_taps(3, 40, B, tau, kappa)
    M = np.zeros((B, B))
    for e in range(B):
        u = np.zeros((V, B))
        u[0, e] = 1.0
        M[:, e] = O.apply_d(u, tl, th, s)[0]
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-13 * np.abs(M).max())
    np.linalg.cholesky(M)


def problem(N, V, B, seed, spread):
    rng = np.random.default_rng(seed)
    xt = synth.ellipse_phantom(N, 4, seed)
    b = O.project(xt, V, B) + 0.2 * rng.standard_normal((V, B))
    w = np.exp(rng.uniform(-spread, spread, (V, B)))
    return b, w


def test_same_limit_as_eq24():
    # Theorem (Sec. 2.2): any symmetric positive definite D gives the minimiser
    N, V, B = 12, 18, 17
    b, w = problem(N, V, B, 4, 2.0)
    beta = 0.3
    kappa = float(np.mean(1 / w))
    tau = O.default_tau(0, V, kappa)
    t0 = O.ramp_taps(0, V, B, tau, kappa)
    tl, th = O.ramp_taps(2, V, B, tau, kappa), O.ramp_taps(3, V, B, tau, kappa)
    s = O.shift_variant_scale(w)
    sig0, _, _ = O.step_sizes(0, N, V, B, t0, w, tau)
    sig2, _, _ = O.step_sizes(0, N, V, B, tl, w, tau, taps_hi=th, s=s)
    x0 = O.pdtv(b, w, t0, 0, beta, tau, sig0, 50, 3000, N)[0].x
    x2 = O.pdtv(b, w, tl, 0, beta, tau, sig2, 50, 3000, N, taps_hi=th, s=s)[0].x
    assert np.linalg.norm(x2 - x0) / np.linalg.norm(x0) < 1e-6


def test_faster_with_spread_weights():
    # the purpose of the form: transmission data whose counts span two
    # decades (dense object, Poisson statistics); after 20 iterations the
    # iterate is closer to the minimiser than with Eq. 24 (0.63x measured)
    N, V, B = 32, 45, 47
    xt = synth.ellipse_phantom(N, 6, 2) * (2.0 / N) * 8.0
    b, w = synth.poisson_data(O.project(xt, V, B), 1e4, 5)
    assert w.max() / w.min() > 100
    beta = 0.01
    kappa = float(np.mean(1 / w))
    tau = O.default_tau(0, V, kappa)
    t0 = O.ramp_taps(0, V, B, tau, kappa)
    tl, th = O.ramp_taps(2, V, B, tau, kappa), O.ramp_taps(3, V, B, tau, kappa)
    s = O.shift_variant_scale(w)
    sig0, _, _ = O.step_sizes(0, N, V, B, t0, w, tau)
    sig2, _, _ = O.step_sizes(0, N, V, B, tl, w, tau, taps_hi=th, s=s)
    xs = O.pdtv(b, w, t0, 0, beta, tau, sig0, 20, 3000, N)[0].x
    d0 = np.linalg.norm(O.pdtv(b, w, t0, 0, beta, tau, sig0, 20, 20, N)[0].x - xs)
    d2 = np.linalg.norm(O.pdtv(b, w, tl, 0, beta, tau, sig2, 20, 20, N, taps_hi=th, s=s)[0].x - xs)
    assert d2 < 0.8 * d0
