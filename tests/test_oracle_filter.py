"""Pins of the oracle's preconditioner D = F^-1 H F (Eq. 24 smoothed ramp,
Eq. 32 pure ramp): DFT of a full period equals H (numpy FFT), the direct
convolution equals numpy.convolve, D is symmetric positive definite on the
detector (Cholesky), and tau A^T D A reproduces a smooth image (D inverts
tau A A^T, i.e. filtered backprojection, Sec. 3)."""
import math

import numpy as np
import pytest

import oracle as O
import synth


def H(mode, w, m, tau, kappa):
    return np.abs(w) / (2 * m * tau + kappa * np.abs(w)) if mode == 0 else np.abs(w) / (2 * m * tau)


@pytest.mark.parametrize("mode", [0, 1])
def test_fft_of_full_period_is_H(mode):
    B, V, tau, kappa = 95, 90, 0.3, 0.02
    P = O.fft_len(B)
    assert P == 256
    half = P // 2 + 1
    t = O.ramp_taps(mode, V, B, tau, kappa, half=half, period=P)
    per = np.zeros(P)
    for k in range(-(half - 1), half):
        per[k % P] = t[half - 1 + k]           # k = +-P/2 land on the same slot
    per[P // 2] = t[half - 1 + P // 2]
    j = np.arange(P)
    w = 2 * math.pi * np.minimum(j, P - j) / P
    np.testing.assert_allclose(np.fft.fft(per).real, H(mode, w, V, tau, kappa), rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.fft.fft(per).imag, 0.0, atol=1e-12)


def test_fft_length_rule():
    assert [O.fft_len(b) for b in (95, 368, 369, 553, 736, 738)] == [256, 1024, 1024, 2048, 2048, 2048]


def test_filter_is_numpy_convolve():
    B, V = 37, 5
    t = O.ramp_taps(0, 60, B, 0.1, 0.05)
    y = synth.random_sinogram(V, B, 3)
    out = O.filt(y, t)
    for v in range(V):
        full = np.convolve(y[v], t)            # length B + 2B-1 - 1
        np.testing.assert_allclose(out[v], full[B - 1:2 * B - 1], rtol=0, atol=1e-13)


def test_impulse_response_is_taps():
    B = 21
    t = O.ramp_taps(1, 30, B, 0.5)
    e = np.zeros((1, B))
    e[0, 10] = 1.0
    out = O.filt(e, t)[0]
    np.testing.assert_allclose(out, t[B - 1 - 10:B - 1 - 10 + B], atol=0)


@pytest.mark.parametrize("mode", [0, 1])
def test_D_symmetric_positive_definite(mode):
    B = 95
    t = O.ramp_taps(mode, 90, B, 0.2, 0.05)
    D = np.array([[t[B - 1 + (i - j)] for j in range(B)] for i in range(B)])
    np.testing.assert_allclose(D, D.T, atol=0)
    np.linalg.cholesky(D)                      # raises if not positive definite
    # smallest eigenvalue is positive but small (H(0) = 0 on the period)
    assert np.linalg.eigvalsh(D).min() > 0


def test_fbp_identity_scale():
    # D = (tau A A^T)^-1 (Eq. 32) makes tau A^T D A the identity on smooth
    # images up to the interpolation blur of the projector.  A wrong factor
    # (2, pi, m) in H or in the frequency axis breaks this by far more.
    N, V, B = 64, 180, 95
    c = (N - 1) / 2
    yy, xx = np.meshgrid(np.arange(N) - c, np.arange(N) - c, indexing="ij")
    x = np.exp(-(xx ** 2 + yy ** 2) / (2 * 8.0 ** 2)) + 0.5 * np.exp(-((xx - 10) ** 2 + (yy + 5) ** 2) / 32.0)
    for tau in (1.0, 0.05):
        t = O.ramp_taps(1, V, B, tau)
        y = tau * O.backproject(O.filt(O.project(x, V, B), t), N)
        m = (xx ** 2 + yy ** 2) < 25 ** 2
        assert np.linalg.norm((y - x)[m]) / np.linalg.norm(x[m]) < 0.02


def test_smoothed_ramp_tends_to_pure_ramp():
    # kappa -> 0 in Eq. 24 gives Eq. 32.
    t0 = O.ramp_taps(0, 32, 50, 0.7, 0.0)
    t1 = O.ramp_taps(1, 32, 50, 0.7)
    np.testing.assert_allclose(t0, t1, rtol=1e-12, atol=1e-15)
