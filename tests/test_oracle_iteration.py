"""Pins of the oracle's Algorithm 1 / 1' / 2 (Eqs. 18-20, 29-31) against what
the paper and the mathematics fix: the first iterate is filtered
backprojection followed by the TV prox (Sec. 2.2, Sec. 3), the beta = 0 limit
is the weighted least-squares solution (closed form), the few-view limit
with an injective A is x_true, the limit does not depend on D or tau (the
Theorem of Sec. 2.2) and equals an independent Chambolle-Pock run on
K = [A; grad], and the dual fixed point is mu* = W(Ax* - b) (Eq. 20)."""
import numpy as np
import pytest

import oracle as O
import synth


def explicit_A(N, V, B):
    A = np.zeros((V * B, N * N))
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        A[:, j] = O.project(e.reshape(N, N), V, B).ravel()
    return A


def lowdose_problem(N=8, V=16, B=13, seed=1, noise=0.01):
    rng = np.random.default_rng(seed)
    xt = 0.5 + 0.5 * rng.uniform(size=(N, N))
    b = O.project(xt, V, B) + noise * rng.standard_normal((V, B))
    w = rng.uniform(0.5, 2.0, (V, B))
    return xt, b, w


def test_first_iterate_is_fbp_then_tv():
    # x^0 = mu^0 = 0: x^1 = prox_{tau g}(sigma tau A^T D b).
    N, V, B = 16, 20, 23
    xt = synth.ellipse_phantom(N, 3, 0)
    b = O.project(xt, V, B)
    tau, sigma, beta, ntv = 0.05, 0.8, 0.02, 7
    for mode in (0, 1):
        w = np.full((V, B), 2.0) if mode == 0 else None
        taps = O.ramp_taps(mode, V, B, tau, 0.5 if mode == 0 else 0.0)
        st, _ = O.pdtv(b, w, taps, mode, beta, tau, sigma, ntv, 1, N)
        z = sigma * tau * O.backproject(O.filt(b, taps), N)
        lam = tau * beta if mode == 0 else tau
        x1, _, _ = O.tv_prox(z, lam, ntv)
        np.testing.assert_allclose(st.x, x1, rtol=0, atol=1e-13)


def test_beta_zero_limit_is_weighted_least_squares():
    # Algorithm 1' converges to argmin_{x>=0} 1/2||Ax-b||_W^2; with a
    # positive unconstrained solution that is (A^T W A)^-1 A^T W b.
    N, V, B = 8, 16, 13
    xt, b, w = lowdose_problem(N, V, B)
    A = explicit_A(N, V, B)
    xw = np.linalg.solve(A.T @ (w.ravel()[:, None] * A), A.T @ (w.ravel() * b.ravel()))
    assert xw.min() > 0
    kappa = float(np.mean(1 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau)
    st, _ = O.pdtv(b, w, taps, 0, 0.0, tau, sigma, 10, 20000, N)
    assert np.linalg.norm(st.x.ravel() - xw) / np.linalg.norm(xw) < 1e-10
    # dual fixed point of Eq. 20: mu* = W (A x* - b)
    r = w * (O.project(st.x, V, B) - b)
    assert np.linalg.norm(st.mu - r) / np.linalg.norm(r) < 1e-8


def test_fewview_injective_limit_is_truth():
    # I > J and A injective: Ax = b, x >= 0 has the single point x_true.
    N, V, B = 8, 16, 13
    xt, _, _ = lowdose_problem(N, V, B)
    b = O.project(xt, V, B)
    tau = 0.01
    taps = O.ramp_taps(1, V, B, tau)
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    st, tr = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, 3000, N, trace=True)
    assert np.linalg.norm(st.x - xt) / np.linalg.norm(xt) < 1e-8
    assert tr[-1] < 1e-7 and tr[-1] < tr[0]


def test_tv_limit_matches_chambolle_pock_and_plain_iteration():
    # Theorem (Sec. 2.2): the saddle point gives the minimiser of Eq. 1 for
    # any non-singular D.  Three routes: ramp-preconditioned Algorithm 1,
    # unpreconditioned (D = I) Algorithm 1, and Chambolle-Pock on K = [A; grad].
    N, V, B = 16, 24, 23
    rng = np.random.default_rng(5)
    xt = synth.ellipse_phantom(N, 4, 3)
    b = O.project(xt, V, B) + 0.3 * rng.standard_normal((V, B))
    w = rng.uniform(0.5, 2.0, (V, B))
    beta = 0.5
    kappa = float(np.mean(1 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau)
    st, tr = O.pdtv(b, w, taps, 0, beta, tau, sigma, 50, 1500, N, trace=True)
    xa = st.x
    # plain iteration, same problem
    tau1 = 0.01
    sig1, _, _ = O.step_sizes(0, N, V, B, np.ones(1), w, tau1)
    st1, _ = O.pdtv(b, w, np.ones(1), 0, beta, tau1, sig1, 50, 4000, N)
    assert np.linalg.norm(st1.x - xa) / np.linalg.norm(xa) < 1e-10
    # Chambolle-Pock on [A; grad]
    L = np.sqrt(O.power_norm(0, N, V, B, iters=300) + 8.0)
    xr = O.cp_reference(b, w, 0, beta, 0.99 / (0.2 * L), 0.99 * 0.2 / L, 60000, N)
    assert np.linalg.norm(xr - xa) / np.linalg.norm(xa) < 2e-5
    fa, fr = O.cost(xa, b, w, beta), O.cost(xr, b, w, beta)
    assert fa <= fr + 1e-9 * abs(fr)
    assert tr[-1] == pytest.approx(fa, rel=1e-12)


def test_limit_independent_of_tau():
    N, V, B = 12, 18, 17
    rng = np.random.default_rng(2)
    xt = synth.ellipse_phantom(N, 3, 1)
    b = O.project(xt, V, B) + 0.2 * rng.standard_normal((V, B))
    w = rng.uniform(0.5, 2.0, (V, B))
    beta = 0.3
    kappa = float(np.mean(1 / w))
    xs = []
    for f in (0.25, 1.0, 4.0):
        tau = f * O.default_tau(0, V, kappa)
        taps = O.ramp_taps(0, V, B, tau, kappa)
        sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau)
        st, _ = O.pdtv(b, w, taps, 0, beta, tau, sigma, 50, 3000, N)
        xs.append(st.x)
    for x in xs[1:]:
        assert np.linalg.norm(x - xs[0]) / np.linalg.norm(xs[0]) < 1e-6


def test_resume_is_bit_exact():
    N, V, B = 10, 12, 15
    xt, b, w = lowdose_problem(N, V, B, seed=4)
    taps = O.ramp_taps(0, V, B, 0.05, 0.7)
    st, _ = O.pdtv(b, w, taps, 0, 0.1, 0.05, 0.5, 5, 7, N)
    sa, _ = O.pdtv(b, w, taps, 0, 0.1, 0.05, 0.5, 5, 3, N)
    sa, _ = O.pdtv(b, w, taps, 0, 0.1, 0.05, 0.5, 5, 4, N, state=sa)
    np.testing.assert_array_equal(sa.x, st.x)
    np.testing.assert_array_equal(sa.mu, st.mu)


def test_power_norm_matches_matrix_norm():
    N, V, B = 8, 10, 13
    A = explicit_A(N, V, B)
    taps = O.ramp_taps(0, V, B, 0.1, 0.3)
    D = np.array([[taps[B - 1 + (i - j)] for j in range(B)] for i in range(B)])
    DD = np.kron(np.eye(V), D)
    M = A.T @ DD @ A
    assert O.power_norm(0, N, V, B, taps=taps, iters=500) == pytest.approx(np.linalg.norm(M, 2), rel=1e-6)
    w = np.random.default_rng(0).uniform(0.5, 2.0, V * B)
    Mw = np.diag(w ** -0.5) @ DD @ np.diag(w ** -0.5)
    got = O.power_norm(1, N, V, B, taps=taps, w=w.reshape(V, B), iters=2000)
    assert got == pytest.approx(np.linalg.norm(Mw, 2), rel=1e-6)


def test_fgp_prox_keeps_the_limit():
    # the prox by fast gradient projection (warm-started, momentum restarted
    # at every outer iteration) reaches the same minimiser of Eq. 1
    N, V, B = 12, 18, 17
    rng = np.random.default_rng(2)
    xt = synth.ellipse_phantom(N, 3, 1)
    b = O.project(xt, V, B) + 0.2 * rng.standard_normal((V, B))
    w = rng.uniform(0.5, 2.0, (V, B))
    beta = 0.3
    kappa = float(np.mean(1 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau)
    xg = O.pdtv(b, w, taps, 0, beta, tau, sigma, 10, 3000, N)[0].x
    xf = O.pdtv(b, w, taps, 0, beta, tau, sigma, 10, 3000, N, fgp=True)[0].x
    assert np.linalg.norm(xf - xg) / np.linalg.norm(xg) < 1e-6


def test_fewview_ell_is_mean_diagonal_of_AAt():
    # l of the few-view smoothed ramp against the explicit matrix: the mean
    # over the rays that meet the image of sum_j a_ij^2, times the hit fraction
    N, V, B = 16, 24, 23
    A = explicit_A(N, V, B)
    diag = (A ** 2).sum(axis=1)
    assert O.fewview_ell(N, V, B) == pytest.approx(diag.mean(), rel=0.05)


def fewview_problem(N, V, B, seed):
    x = synth.ellipse_phantom(N, 8, seed)
    return x, O.project(x, V, B)


def test_fewview_smoothed_ramp_keeps_the_limit():
    # Theorem (Sec. 2.2): injective few-view (N = 8, V = 16, B = 13): the
    # smoothed ramp with kappa = tau l also converges to x_true
    N, V, B = 8, 16, 13
    rng = np.random.default_rng(3)
    xt = 0.5 + 0.5 * rng.uniform(size=(N, N))
    b = O.project(xt, V, B)
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    st, _ = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, 12000, N)
    assert np.linalg.norm(st.x - xt) / np.linalg.norm(xt) < 1e-8


def test_fewview_smoothed_ramp_converges_faster_than_eq32():
    # 64^2 from 32 views: the pure ramp of Eq. 32 over-amplifies the detector
    # frequencies that sparse views leave to the same-view part of A A^T
    N, V, B = 64, 32, 95
    x, b = fewview_problem(N, V, B, 0)
    tau = O.default_tau(1, V, 0.0)
    t32 = O.ramp_taps(1, V, B, tau)
    tsm = O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    s32, n32, _ = O.step_sizes(1, N, V, B, t32, None, tau)
    ssm, nsm, _ = O.step_sizes(1, N, V, B, tsm, None, tau)
    assert tau * nsm < 0.5 * tau * n32          # the step-size bound is far less restrictive
    xs = O.pdtv(b, None, t32, 1, 0.0, tau, s32, 10, 2000, N)[0].x
    d32 = np.linalg.norm(O.pdtv(b, None, t32, 1, 0.0, tau, s32, 10, 30, N)[0].x - xs)
    dsm = np.linalg.norm(O.pdtv(b, None, tsm, 1, 0.0, tau, ssm, 10, 30, N)[0].x - xs)
    assert dsm < 0.5 * d32


def test_extrapolation_agrees_with_the_first_form_of_eq18_and_eq29():
    # Eq. 18 states Step 1 of Algorithm 1 in two forms,
    #   mu^k + sigma D (A x^k - b - W^-1 mu^k)                    (APP's own step)
    #   2 mu^k - mu^{k-1} - sigma D W^-1 (mu^k - mu^{k-1})        (the box form),
    # equal because mu^k - mu^{k-1} is the previous dual update; Eq. 29 is the
    # same without W^-1 (Algorithm 2).  The oracle runs the box form; here
    # the first form is formed from its state at k = 0 .. 5 with the oracle's
    # A, D and W, so a dropped term, a wrong sign or a stale mu^{k-1} in the
    # box form shows up as a mismatch.
    N, V, B = 12, 18, 17
    xt, b, w = lowdose_problem(N, V, B, seed=7, noise=0.05)
    for mode in (0, 1):
        ww = w if mode == 0 else None
        kappa = float(np.mean(1 / w)) if mode == 0 else 0.0
        tau = O.default_tau(mode, V, kappa)
        taps = O.ramp_taps(mode, V, B, tau, kappa)
        sigma, _, _ = O.step_sizes(mode, N, V, B, taps, ww, tau)
        st = None
        for k in range(6):
            x_k = np.zeros((N, N)) if st is None else st.x.copy()
            mu_k = np.zeros((V, B)) if st is None else st.mu.copy()
            r = O.project(x_k, V, B) - b
            if mode == 0:
                r = r - mu_k / w
            first = mu_k + sigma * O.filt(r, taps)
            mb = np.empty((V, B))
            st, _ = O.pdtv(b, ww, taps, mode, 0.05, tau, sigma, 5, 1, N, state=st, mubar=mb)
            assert np.linalg.norm(mb - first) <= 1e-12 * np.linalg.norm(first)
        # the low-dose correction term is not negligible here: dropping it
        # (Algorithm 2's Step 1 on Algorithm 1's state) misses the first form
        if mode == 0:
            st2, _ = O.pdtv(b, ww, taps, mode, 0.05, tau, sigma, 5, 3, N)
            mu_prev = st2.mu_prev.copy()
            mu_k = st2.mu.copy()
            first = mu_k + sigma * O.filt(O.project(st2.x, V, B) - b - mu_k / w, taps)
            no_corr = 2 * mu_k - mu_prev
            assert np.linalg.norm(no_corr - first) > 1e-3 * np.linalg.norm(first)


def test_cost_of_eq1_has_the_half():
    # Eq. 1: f(x) = beta psi(x) + 1/2 ||Ax - b||_W^2.  At the unconstrained
    # beta = 0 minimiser x* (normal equations, numpy solve) the gradient
    # vanishes, so f(x* + e d) - f(x*) = 1/2 e^2 ||A d||_W^2 exactly, with A
    # the explicit matrix; a missing 1/2 doubles it.
    N, V, B = 8, 16, 13
    xt, b, w = lowdose_problem(N, V, B, seed=3)
    A = explicit_A(N, V, B)
    wv = w.ravel()
    xs = np.linalg.solve(A.T @ (wv[:, None] * A), A.T @ (wv * b.ravel())).reshape(N, N)
    d = np.random.default_rng(11).standard_normal((N, N))
    Ad = A @ d.ravel()
    for eps in (0.1, 0.5):
        df = O.cost(xs + eps * d, b, w, 0.0) - O.cost(xs, b, w, 0.0)
        assert df == pytest.approx(0.5 * eps ** 2 * float(Ad @ (wv * Ad)), rel=1e-8)
    # and the penalty term: b = A x gives zero fidelity, so f = beta psi(x);
    # a vertical step of height h across all N rows has psi = N h (Eq. 2
    # with forward differences)
    h, beta = 0.7, 0.3
    x = np.zeros((N, N))
    x[:, N // 2:] = h
    assert O.cost(x, O.project(x, V, B), w, beta) == pytest.approx(beta * N * h, rel=1e-12)
    # unit weights (W = I, the few-view residual's norm): f = 1/2 ||Ax - b||^2
    bb = b + 0.1
    r = O.residual(x, bb)
    assert O.cost(x, bb, None, 0.0) == pytest.approx(0.5 * r * r, rel=1e-12)
