"""Pins of the oracle's epsilon-constrained few-view form (min TV(x) subject
to ||Ax - b|| <= eps, x >= 0; Sec. 5 names it without giving its steps:
the eps-ball's support function takes h's place, so the dual step is a
proximal map).  Its dual step is checked
against a brute-force minimisation of its variational definition and its
closed forms; its limit against the independent Chambolle-Pock run on
K = [A; grad] with the Euclidean ball projection, the constraint being
active at the limit, and the eps -> 0 and eps >= |b| ends."""
import numpy as np
import pytest

import oracle as O


def toeplitz(taps, B):
    """The B x B matrix of the per-view convolution D (centre tap at half-1)."""
    half = (taps.size + 1) // 2
    T = np.zeros((B, B))
    for i in range(B):
        for j in range(B):
            if abs(i - j) < half:
                T[i, j] = taps[half - 1 + i - j]
    return T


def prox_objective(nu, q, Tinv, se):
    d = nu - q
    return se * np.linalg.norm(nu) + 0.5 * sum(d[v] @ Tinv @ d[v] for v in range(q.shape[0]))


@pytest.mark.parametrize("kind", ["ramp_eq32", "smoothed"])
def test_eps_prox_minimises_its_definition(kind):
    scipy_opt = pytest.importorskip("scipy.optimize")
    V, B, tau = 3, 7, 0.05
    taps = O.ramp_taps(1, 8, B, tau) if kind == "ramp_eq32" else O.ramp_taps(0, 8, B, tau, 0.3)
    T = toeplitz(taps, B)
    Tinv = np.linalg.inv(T)
    rng = np.random.default_rng(4)
    for trial in range(3):
        q = rng.standard_normal((V, B))
        bound = np.linalg.norm(np.linalg.solve(T, q.T))    # |T^-1 q|: nu = 0 at and above
        se = (0.15 + 0.3 * trial) * bound
        nu = O.eps_prox(q, taps, se)
        f = lambda v: prox_objective(v.reshape(V, B), q, Tinv, se)
        best = scipy_opt.minimize(f, q.ravel(), method="BFGS", options={"gtol": 1e-11, "maxiter": 20000}).x
        assert f(nu.ravel()) <= f(best) + 1e-10 * abs(f(best))
        assert np.linalg.norm(nu.ravel() - best) <= 1e-4 * np.linalg.norm(q)
        # no direction decreases the objective from nu
        for _ in range(20):
            d = rng.standard_normal(V * B)
            assert f(nu.ravel() + 1e-6 * d) >= f(nu.ravel()) - 1e-14


def test_eps_prox_ends_and_identity():
    V, B = 2, 9
    taps = O.ramp_taps(1, 8, B, 0.05)
    T = toeplitz(taps, B)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((V, B))
    # eps = 0: the equality form's dual step (q itself)
    assert np.array_equal(O.eps_prox(q, taps, 0.0), q)
    # se >= |T^-1 q|: nu = 0; just below it: not
    bound = np.linalg.norm(np.linalg.solve(T, q.T))
    assert not O.eps_prox(q, taps, 1.0001 * bound).any()
    assert np.linalg.norm(O.eps_prox(q, taps, 0.999 * bound)) > 0
    # D = I: the conjugate of the Euclidean ball's indicator shrinks radially
    for se in (0.1, 0.5 * np.linalg.norm(q), 2.0 * np.linalg.norm(q)):
        want = max(0.0, 1.0 - se / np.linalg.norm(q)) * q
        assert np.allclose(O.eps_prox(q, np.ones(1), se), want, rtol=1e-12, atol=1e-12)


def noisy_fewview(N=8, V=16, B=13, seed=6, rel_noise=0.02):
    rng = np.random.default_rng(seed)
    xt = 0.5 + 0.5 * rng.uniform(size=(N, N))
    clean = O.project(xt, V, B)
    noise = rel_noise * np.abs(clean).mean() * rng.standard_normal((V, B))
    return xt, clean + noise, float(np.linalg.norm(noise))


def test_eps_limit_equals_chambolle_pock_and_is_active():
    # the ramp-preconditioned eps-form and plain Chambolle-Pock on [A; grad]
    # with the Euclidean ball reach the same minimiser; the constraint is
    # active there and the phantom (feasible) has no smaller TV
    N, V, B = 8, 16, 13
    xt, b, nn = noisy_fewview(N, V, B)
    eps = nn
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    st, _ = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 20, 2000, N, eps=eps)
    xp = st.x
    L = np.sqrt(O.power_norm(0, N, V, B, iters=300) + 8.0)
    xr = O.cp_reference(b, None, 1, 0.0, 0.99 / (0.2 * L), 0.99 * 0.2 / L, 40000, N, eps=eps)
    assert np.linalg.norm(xp - xr) / np.linalg.norm(xr) < 1e-8
    assert np.linalg.norm(O.project(xp, V, B) - b) == pytest.approx(eps, rel=1e-9)
    assert O.tv(xp) < 0.9 * O.tv(xt)
    # the equality form (no tolerance) has another limit
    xe = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 20, 2000, N)[0].x
    assert np.linalg.norm(xe - xr) / np.linalg.norm(xr) > 0.05


def test_eps_above_data_norm_gives_a_flat_image():
    # eps >= |b|: x = 0 is feasible, so the minimum TV is 0 (a constant image)
    N, V, B = 8, 16, 13
    xt, b, _ = noisy_fewview(N, V, B, seed=7)
    eps = 1.5 * np.linalg.norm(b)
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(1, V, B, tau)
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    x = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 20, 2000, N, eps=eps)[0].x
    assert O.tv(x) <= 1e-6 * O.tv(xt)
    assert np.linalg.norm(O.project(x, V, B) - b) <= eps * (1 + 1e-9)


def test_eps_to_zero_recovers_the_equality_limit():
    # noiseless data, injective A: the equality form's limit is x_true; a
    # tiny eps moves the limit by O(eps)
    N, V, B = 8, 16, 13
    rng = np.random.default_rng(3)
    xt = 0.5 + 0.5 * rng.uniform(size=(N, N))
    b = O.project(xt, V, B)
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    x = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, 12000, N, eps=1e-7 * np.linalg.norm(b))[0].x
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) < 1e-5
