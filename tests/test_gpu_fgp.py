"""GPU parity of the TV prox by fast gradient projection (tv_accel = 1)
inside the whole iteration, against the FP64 oracle run with the same tau,
sigma, taps and FGP prox: relative L2 <= 1e-3 after the stated iterations,
for several inner step counts and TV tile shapes (the temporally blocked
tiles must reproduce the whole-image FGP exactly, momentum included)."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-3


def lowdose_case(N, V, B, seed, n_ell=10, i0=1e4):
    x = synth.ellipse_phantom(N, n_ell, seed) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x, V, B), i0, seed + 100)
    return x, f32(b), f32(w)


@pytest.mark.parametrize("ntv,rows", [(10, 0), (1, 4), (5, 16), (16, 64), (16, 4)])
def test_lowdose_fgp_parity(ntv, rows):
    P = need_gpu()
    N, V, B = 64, 90, 95
    x, b, w = lowdose_case(N, V, B, 0)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    beta, sigma = 2e4, 0.5   # lambda = tau beta ~ 0.01: a prox that does real work on x ~ 0.03
    g = P.Geometry(N, V, B)
    g.set_tuning(tv_rows=rows)
    prm = P.PDTVParams(mode=0, iters=20, tv_iters=ntv, precond=1, beta=beta, tau=tau, sigma=sigma, tv_accel=1)
    xg, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    st, _ = O.pdtv(b, w, taps, 0, beta, tau, sigma, ntv, 20, N, fgp=True)
    assert rel_l2(to_np(xg), st.x) <= TOL
    # and it is not the projected-gradient prox
    sg, _ = O.pdtv(b, w, taps, 0, beta, tau, sigma, ntv, 20, N)
    if ntv > 1:
        assert rel_l2(sg.x, st.x) > 10 * rel_l2(to_np(xg), st.x)


def test_fewview_fgp_parity():
    P = need_gpu()
    N, V, B = 48, 16, 70
    x = synth.ellipse_phantom(N, 6, 2)
    b = f32(O.project(x, V, B))
    tau = O.default_tau(1, V, 0.0)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=1, iters=15, tv_iters=10, precond=1, tau=tau, sigma=0.02, tv_accel=1)
    xg, _ = P.ct_pdtv_solve(g, to_gpu(b), None, prm)
    st, _ = O.pdtv(b, None, O.ramp_taps(1, V, B, tau), 1, 0.0, tau, 0.02, 10, 15, N, fgp=True)
    assert rel_l2(to_np(xg), st.x) <= TOL


@pytest.mark.parametrize("bad", [dict(tv_accel=2), dict(tv_accel=1, tv_iters=17)])
def test_fgp_rejects_bad_parameters(bad):
    P = need_gpu()
    N, V, B = 16, 8, 23
    g = P.Geometry(N, V, B)
    b = to_gpu(np.zeros((V, B)))
    w = to_gpu(np.ones((V, B)))
    with pytest.raises(P.CTError):
        P.ct_pdtv_solve(g, b, w, P.PDTVParams(mode=0, iters=1, **bad))
