"""The host FP64 eigendecomposition behind the error-tolerant few-view form
(ct_sym_toeplitz_eig): eigenvalues equal numpy's, the eigenvectors are
orthonormal and reconstruct the matrix, for random symmetric Toeplitz
matrices and the per-view matrices of the paper's ramp filters."""
import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def P():
    from conftest import build_library
    build_library()
    from paper_1609_06041_gb300 import ctpd
    return ctpd


def toeplitz(t):
    n = t.size
    i = np.arange(n)
    return t[np.abs(i[:, None] - i[None, :])]


def check(P, t):
    T = toeplitz(t)
    q, lam = P.ct_sym_toeplitz_eig(t)
    n = t.size
    scale = max(1.0, np.abs(T).max())
    ref = np.linalg.eigvalsh(T)
    assert np.allclose(np.sort(lam), ref, rtol=0, atol=1e-12 * n * scale)
    assert np.abs(q.T @ q - np.eye(n)).max() < 1e-12 * n
    assert np.abs(q @ np.diag(lam) @ q.T - T).max() < 1e-12 * n * scale


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 33, 64, 95, 150])
def test_random_symmetric_toeplitz(P, n):
    rng = np.random.default_rng(n)
    check(P, rng.standard_normal(n))


@pytest.mark.parametrize("n,mode", [(95, 1), (96, 0), (200, 1), (369, 0)])
def test_ramp_filter_matrices(P, n, mode):
    # the taps of Eq. 32 (few-view) and Eq. 24 (with kappa) as T's first row
    taps = O.ramp_taps(mode, 32, n, 0.01, 0.0 if mode == 1 else 0.5)
    check(P, taps[n - 1:])


def test_degenerate_and_bad_arguments(P):
    check(P, np.zeros(6))                     # all eigenvalues 0
    check(P, np.r_[1.0, np.zeros(9)])          # the identity
    with pytest.raises(P.CTError):
        P.ct_sym_toeplitz_eig(np.zeros(0))
    P.ct_sym_toeplitz_eig(np.ones(3))          # a good call clears the message
    assert P.ct_last_error() == ""
