"""GPU parity of the shift-variant preconditioner D = T_lo + S T_hi S
(precond = 2) against the FP64 oracle: the band taps, the filter itself
(ct_ramp_filter_split), the whole low-dose iteration with the same tau,
sigma and taps, and the step sizes against the 2-norms of the explicitly
built operators."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL_PASS = 1e-4
TOL = 1e-3


def lowdose_case(N, V, B, seed, n_ell=10, i0=1e4, scale=1.0):
    x = synth.ellipse_phantom(N, n_ell, seed) * (2.0 / N) * scale
    b, w = synth.poisson_data(O.project(x, V, B), i0, seed + 100)
    return x, f32(b), f32(w)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("B,V", [(95, 90), (736, 32), (53, 13)])
def test_band_taps_parity(mode, B, V):
    P = need_gpu()
    g = P.Geometry(16, V, B)
    tau, kappa = 0.02, 0.4
    got = to_np(P.ct_ramp_taps(g, mode, tau, kappa))
    ref = O.ramp_taps(mode, V, B, tau, kappa)
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("V,B,half,batch", [(90, 95, 95, 1), (13, 53, 53, 2), (8, 300, 40, 1),
                                            (5, 1100, 1100, 1), (1, 1, 1, 1), (3, 2, 2, 1)])
def test_split_filter_parity(V, B, half, batch):
    P = need_gpu()
    g = P.Geometry(16, V, B)
    rng = np.random.default_rng(V + B)
    w = f32(rng.uniform(50.0, 8000.0, (V, B)))
    kappa = float(np.mean(1.0 / w))
    tl = f32(O.ramp_taps(2, V, B, 0.05, kappa, half=half))
    th = f32(O.ramp_taps(3, V, B, 0.05, kappa, half=half))
    s = f32(O.shift_variant_scale(w))
    ys = [f32(synth.random_sinogram(V, B, 4 + k)) for k in range(batch)]
    got = to_np(P.ct_ramp_filter_split(g, to_gpu(tl), to_gpu(th), to_gpu(s), to_gpu(np.stack(ys))))
    for k in range(batch):
        assert rel_l2(got[k], O.apply_d(ys[k], tl, th, s)) <= TOL_PASS


def test_split_filter_rejects_large_detectors():
    P = need_gpu()
    g = P.Geometry(16, 2, 4200)
    t = to_gpu(np.zeros(2 * 4200 - 1))
    y = to_gpu(np.zeros((2, 4200)))
    with pytest.raises(P.CTError):
        P.ct_ramp_filter_split(g, t, t, y, y)


@pytest.mark.parametrize("N,V,B,scale,iters", [(64, 90, 95, 1.0, 20), (48, 60, 70, 6.0, 25)])
def test_solve_parity(N, V, B, scale, iters):
    # low-dose Algorithm 1 with the shift-variant D, 10 TV steps, explicit tau
    # and sigma, against the oracle with the same band taps and s
    P = need_gpu()
    x, b, w = lowdose_case(N, V, B, 1, scale=scale)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    beta, sigma = 0.01, 0.4
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=iters, tv_iters=10, precond=2, beta=beta, tau=tau, sigma=sigma)
    ws = P.workspace_for(g, prm)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm, workspace=ws)
    tl, th = O.ramp_taps(2, V, B, tau, kappa), O.ramp_taps(3, V, B, tau, kappa)
    st, _ = O.pdtv(b, w, tl, 0, beta, tau, sigma, 10, iters, N, taps_hi=th, s=O.shift_variant_scale(w))
    assert rel_l2(to_np(xg), st.x) <= TOL
    # resume continues the same iteration
    prm2 = P.PDTVParams(**{**prm.__dict__, "iters": 3, "resume": 1})
    xg2, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm2, x_out=xg, workspace=ws)   # x lives in x_out
    st2, _ = O.pdtv(b, w, tl, 0, beta, tau, sigma, 10, 3, N, state=st, taps_hi=th, s=O.shift_variant_scale(w))
    assert rel_l2(to_np(xg2), st2.x) <= TOL


def test_step_sizes_match_matrix_norms():
    P = need_gpu()
    N, V, B = 24, 36, 37
    x, b, w = lowdose_case(N, V, B, 2, n_ell=5, scale=6.0)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=1, beta=0.01, norm_iters=40, precond=2)
    _, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    tl, th = O.ramp_taps(2, V, B, tau, kappa), O.ramp_taps(3, V, B, tau, kappa)
    s = O.shift_variant_scale(w)
    cols = []
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        cols.append(O.backproject(O.apply_d(O.project(e.reshape(N, N), V, B), tl, th, s), N).ravel())
    nada = np.linalg.norm(np.stack(cols, axis=1), 2)
    Tl = np.array([[tl[B - 1 + (i - j)] for j in range(B)] for i in range(B)])
    Th = np.array([[th[B - 1 + (i - j)] for j in range(B)] for i in range(B)])
    nwdw = 0.0
    for v in range(V):
        D = Tl + s[v][:, None] * Th * s[v][None, :]
        q = 1.0 / np.sqrt(w[v])
        nwdw = max(nwdw, np.linalg.norm(q[:, None] * D * q[None, :], 2))
    assert nada * (1 - 2e-4) <= rep["norm_ADA"] <= nada * 1.01
    assert nwdw * (1 - 2e-4) <= rep["norm_WDW"] <= nwdw * 1.01
    assert rep["sigma"] == pytest.approx(0.95 * min(2.0 / rep["norm_WDW"], 1.0 / (tau * rep["norm_ADA"])), rel=1e-6)


def test_rejects_fewview_and_bad_precond():
    P = need_gpu()
    N, V, B = 16, 8, 23
    g = P.Geometry(N, V, B)
    b = to_gpu(np.zeros((V, B)))
    with pytest.raises(P.CTError):
        P.ct_pdtv_solve(g, b, None, P.PDTVParams(mode=1, iters=1, precond=2))
    with pytest.raises(P.CTError):
        P.ct_pdtv_solve(g, b, to_gpu(np.ones((V, B))), P.PDTVParams(mode=0, iters=1, precond=3))
