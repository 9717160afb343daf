"""The boundary's input checks and the optional per-iteration trace of
ct_pdtv_solve.

Eq. 1 needs W = diag(w) positive definite (W^-1 enters every dual step of
Algorithm 1), and b and w finite; a solve given a zero weight (a
photon-starved ray), a negative one, or NaN / infinity must return
CT_ERR_ARG or CT_ERR_NONFINITE instead of CT_OK with a NaN image.  The
trace is f(x^{k+1}) of Eq. 1 (low-dose) or ||A x^{k+1} - b|| (few-view,
Eq. 25) after every iteration, checked against the oracle's orc_cost /
orc_residual of its own iterates."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu


def lowdose(N, V, B, seed):
    x = synth.ellipse_phantom(N, 8, seed) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x, V, B), 1e4, seed + 7)
    return f32(b), f32(w)


def test_bad_weights_and_data_return_error_codes():
    P = need_gpu()
    C = P.ctpd
    N, V, B = 32, 30, 47
    b, w = lowdose(N, V, B, 1)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=3, beta=0.01, sigma=0.5)
    cases = []
    w0 = w.copy()
    w0[3, 7] = 0.0                       # a ray with no counts
    cases.append((b, w0, C.CT_ERR_ARG))
    wn = w.copy()
    wn[0, 0] = -2.0
    cases.append((b, wn, C.CT_ERR_ARG))
    bn = b.copy()
    bn[5, 11] = np.nan
    cases.append((bn, w, C.CT_ERR_NONFINITE))
    wi = w.copy()
    wi[9, 2] = np.inf
    cases.append((b, wi, C.CT_ERR_NONFINITE))
    for bb, ww, code in cases:
        with pytest.raises(P.CTError) as e:
            P.ct_pdtv_solve(g, to_gpu(bb), to_gpu(ww), prm)
        assert e.value.status == code, str(e.value)
    # clean inputs still pass on the same geometry
    x, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    assert rep["k"] == 3 and np.isfinite(to_np(x)).all()


def test_status_without_report_and_in_a_solve_graph():
    # no report: the flags stay in the workspace, ct_pdtv_status reads them;
    # the repeated call replays the library's solve graph, which checks too
    P = need_gpu()
    C = P.ctpd
    N, V, B = 32, 30, 47
    b, w = lowdose(N, V, B, 2)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=2, beta=0.01, sigma=0.5)
    ws = P.workspace_for(g, prm)
    tb, tw = to_gpu(b), to_gpu(w)
    x = P.ct_pdtv_solve(g, tb, tw, prm, workspace=ws, report=False)[0]
    P.ct_pdtv_status(ws)
    tw[4, 4] = 0.0
    P.ct_pdtv_solve(g, tb, tw, prm, x_out=x, workspace=ws, report=False)
    with pytest.raises(P.CTError) as e:
        P.ct_pdtv_status(ws)
    assert e.value.status == C.CT_ERR_ARG
    tw.copy_(to_gpu(w))
    P.ct_pdtv_solve(g, tb, tw, prm, x_out=x, workspace=ws, report=False)
    P.ct_pdtv_status(ws)


def test_fewview_nan_and_divergent_step_sizes():
    P = need_gpu()
    C = P.ctpd
    N, V, B = 40, 12, 58
    b = f32(O.project(synth.ellipse_phantom(N, 6, 3), V, B))
    g = P.Geometry(N, V, B)
    bn = b.copy()
    bn[1, 30] = np.inf
    with pytest.raises(P.CTError) as e:
        P.ct_pdtv_solve(g, to_gpu(bn), None, P.PDTVParams(mode=P.CT_FEWVIEW, iters=2))
    assert e.value.status == C.CT_ERR_NONFINITE
    # a step size far beyond the Alg. 2 bound overflows the iterate to
    # infinity / NaN: reported, not returned as CT_OK
    with pytest.raises(P.CTError) as e:
        P.ct_pdtv_solve(g, to_gpu(b), None, P.PDTVParams(mode=P.CT_FEWVIEW, iters=60, tau=1e6, sigma=1e30))
    assert e.value.status == C.CT_ERR_NONFINITE


def test_batched_names_the_bad_slice():
    P = need_gpu()
    C = P.ctpd
    b1, w1 = lowdose(32, 30, 47, 4)
    b2, w2 = lowdose(24, 20, 35, 5)
    w2[0, 3] = 0.0
    s = [(P.Geometry(32, 30, 47), to_gpu(b1), to_gpu(w1), P.PDTVParams(mode=0, iters=2, beta=0.01, sigma=0.5)),
         (P.Geometry(24, 20, 35), to_gpu(b2), to_gpu(w2), P.PDTVParams(mode=0, iters=2, beta=0.01, sigma=0.5))]
    with pytest.raises(P.CTError) as e:
        P.ct_pdtv_solve_batched(s)
    assert e.value.status == C.CT_ERR_ARG and "slice 1" in str(e.value)


def test_lowdose_trace_is_the_cost_of_eq1():
    P = need_gpu()
    N, V, B = 64, 90, 95
    b, w = lowdose(N, V, B, 6)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau)
    beta, K = 0.01, 12
    g = P.Geometry(N, V, B)
    _, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w),
                             P.PDTVParams(mode=0, iters=K, beta=beta, tau=tau, sigma=sigma), trace=True)
    _, tr = O.pdtv(b, w, taps, 0, beta, tau, sigma, 10, K, N, trace=True)
    got = np.array(rep["trace"])
    assert got.shape == (K,)
    np.testing.assert_allclose(got, tr, rtol=1e-4)


def test_fewview_trace_is_the_residual():
    P = need_gpu()
    N, V, B = 96, 16, 137
    b = f32(O.project(synth.ellipse_phantom(N, 8, 4), V, B))
    tau = 0.01
    taps = O.ramp_taps(1, V, B, tau)
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    K = 15
    g = P.Geometry(N, V, B)
    _, rep = P.ct_pdtv_solve(g, to_gpu(b), None, P.PDTVParams(mode=1, iters=K, tau=tau, sigma=sigma), trace=True)
    _, tr = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, K, N, trace=True)
    got = np.array(rep["trace"])
    # the residual shrinks towards 0 (Eq. 25); compare against |b| as well
    assert np.all(np.abs(got - tr) <= 1e-4 * tr + 1e-6 * np.linalg.norm(b))
    assert tr[-1] < 0.5 * tr[0]
