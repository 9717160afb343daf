"""GPU parity of the whole iteration (Algorithm 1 / 1' / 2) against the FP64
oracle run with the same tau, sigma, n_tv and taps: relative L2 <= 1e-3 on
the image after the stated iterations (and on the dual variable)."""
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


def run_both(P, N, V, B, b, w, mode, beta, iters, ntv, tau, sigma, precond=1, kappa=None):
    g = P.Geometry(N, V, B)
    if precond:
        kap = float(np.mean(1.0 / w)) if mode == 0 else 0.0
        taps = O.ramp_taps(mode, V, B, tau, kap)
    else:
        taps = np.ones(1)
    prm = P.PDTVParams(mode=mode, iters=iters, tv_iters=ntv, precond=precond, beta=beta,
                       tau=tau, sigma=sigma)
    ws = P.workspace_for(g, prm)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), None if w is None else to_gpu(w), prm, workspace=ws)
    st, _ = O.pdtv(b, w, taps, mode, beta, tau, sigma, ntv, iters, N)
    return to_np(xg), st, rep, ws, g


def test_lowdose_64_parity():
    # 64^2, 90 views, 95 bins, Poisson I0 = 1e4, beta = 0.01, 20 iterations.
    P = need_gpu()
    N, V, B = 64, 90, 95
    x, b, w = lowdose_case(N, V, B, 0)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    xg, st, rep, _, _ = run_both(P, N, V, B, b, w, 0, 0.01, 20, 10, tau, 0.5)
    assert rel_l2(xg, st.x) <= TOL
    assert rep["k"] == 20 and rep["tau"] == pytest.approx(tau) and rep["sigma"] == pytest.approx(0.5)
    assert rep["kappa"] == pytest.approx(kappa, rel=1e-5)


def test_lowdose_beta_zero_parity():
    # Algorithm 1': the prox reduces to max(0, .)
    P = need_gpu()
    N, V, B = 48, 60, 70
    x, b, w = lowdose_case(N, V, B, 3)
    tau = O.default_tau(0, V, float(np.mean(1.0 / w)))
    xg, st, _, _, _ = run_both(P, N, V, B, b, w, 0, 0.0, 15, 10, tau, 0.6)
    assert rel_l2(xg, st.x) <= TOL


def test_fewview_parity():
    # noiseless few-view data, Algorithm 2
    P = need_gpu()
    N, V, B = 96, 16, 137
    x = f32(synth.ellipse_phantom(N, 8, 4))
    b = f32(O.project(x, V, B))
    xg, st, rep, _, _ = run_both(P, N, V, B, b, None, 1, 0.0, 25, 10, 0.01, 0.9)
    assert rel_l2(xg, st.x) <= TOL


def test_plain_iteration_parity():
    # D = I: the unpreconditioned iteration on the same problem
    P = need_gpu()
    N, V, B = 40, 30, 57
    x = f32(synth.ellipse_phantom(N, 6, 9))
    b = f32(O.project(x, V, B))
    xg, st, _, _, _ = run_both(P, N, V, B, b, None, 1, 0.0, 30, 10, 0.01, 0.5, precond=0)
    assert rel_l2(xg, st.x) <= TOL


def test_many_tv_steps_chunked():
    # n_tv larger than one launch's temporal-blocking depth
    P = need_gpu()
    N, V, B = 70, 40, 101
    x, b, w = lowdose_case(N, V, B, 5)
    tau = O.default_tau(0, V, float(np.mean(1.0 / w)))
    xg, st, _, _, _ = run_both(P, N, V, B, b, w, 0, 0.05, 6, 53, tau, 0.5)
    assert rel_l2(xg, st.x) <= TOL


def test_resume_matches_single_run():
    P = need_gpu()
    N, V, B = 64, 90, 95
    x, b, w = lowdose_case(N, V, B, 1)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=12, beta=0.01, sigma=0.5)
    ws = P.workspace_for(g, prm)
    x_all, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm, workspace=ws)
    prm5 = P.PDTVParams(mode=0, iters=5, beta=0.01, sigma=0.5)
    ws2 = P.workspace_for(g, prm5)
    xr, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm5, workspace=ws2)
    prm7 = P.PDTVParams(mode=0, iters=7, beta=0.01, sigma=0.5, resume=1)
    xr, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm7, x_out=xr, workspace=ws2)
    assert rep["k"] == 12
    assert np.array_equal(to_np(x_all), to_np(xr))


def test_auto_step_sizes_match_matrix_norms():
    # sigma of the Alg. 1 box from Lanczos estimates on the GPU, against the
    # 2-norms (numpy) of the explicitly built operators A^T D A and
    # W^-1/2 D W^-1/2 (columns from the FP64 oracle).
    P = need_gpu()
    N, V, B = 32, 45, 48
    x, b, w = lowdose_case(N, V, B, 2, n_ell=5)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=1, beta=0.01, norm_iters=40)
    _, rep = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    cols = []
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        cols.append(O.backproject(O.filt(O.project(e.reshape(N, N), V, B), taps), N).ravel())
    nada = np.linalg.norm(np.stack(cols, axis=1), 2)
    D = np.array([[taps[B - 1 + (i - j)] for j in range(B)] for i in range(B)])
    s = 1.0 / np.sqrt(w)
    nwdw = max(np.linalg.norm(s[v][:, None] * D * s[v][None, :], 2) for v in range(V))
    # the estimates (Ritz value + residual norm) lie at or just above the norms
    assert nada * (1 - 2e-4) <= rep["norm_ADA"] <= nada * 1.01
    assert nwdw * (1 - 2e-4) <= rep["norm_WDW"] <= nwdw * 1.01
    assert rep["sigma"] == pytest.approx(0.95 * min(2.0 / rep["norm_WDW"], 1.0 / (tau * rep["norm_ADA"])), rel=1e-6)
    assert rep["sigma"] <= 0.95 * min(2.0 / nwdw, 1.0 / (tau * nada)) * (1 + 2e-4)


@pytest.mark.parametrize("N,V,B", [(512, 720, 736), (384, 90, 553)])
def test_default_step_sizes_are_valid_at_scale(N, V, B):
    # the default Lanczos depth (12 steps from a +-1 start, Ritz value plus
    # residual norm): the estimates lie above the 64-step ones and close to
    # them, so sigma keeps the step conditions of the Alg. 1 box
    P = need_gpu()
    x, b, w = lowdose_case(N, V, B, 0, n_ell=20, i0=5e3)
    g = P.Geometry(N, V, B)
    _, rep16 = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), P.PDTVParams(mode=0, iters=0, beta=0.005))   # default depth
    _, rep64 = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), P.PDTVParams(mode=0, iters=0, beta=0.005, norm_iters=64))
    for key in ("norm_ADA", "norm_WDW"):
        assert rep16[key] >= rep64[key] * (1 - 1e-3)
        assert rep16[key] <= rep64[key] * 1.05
    assert rep16["sigma"] * rep16["tau"] * rep64["norm_ADA"] <= 0.95 * (1 + 1e-3)
    assert rep16["sigma"] * rep64["norm_WDW"] <= 2 * 0.95 * (1 + 1e-3)


def test_solve_converges_on_gpu():
    # long run: the few-view residual falls and the image approaches x_true
    P = need_gpu()
    N, V, B = 64, 32, 95
    x = f32(synth.ellipse_phantom(N, 6, 11))
    b = f32(O.project(x, V, B))
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=1, iters=300)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), None, prm)
    xg = to_np(xg)
    res = np.linalg.norm(O.project(xg, V, B) - b) / np.linalg.norm(b)
    assert res < 1e-2
    assert rel_l2(xg, x) < 0.2


def test_full_size_two_iterations():
    # 512^2, 720 views, 736 bins, I0 = 5e3, beta = 0.005: two iterations
    # against the oracle (the oracle needs a few seconds per iteration).
    P = need_gpu()
    N, V, B = 512, 720, 736
    x, b, w = lowdose_case(N, V, B, 0, n_ell=20, i0=5e3)
    tau = O.default_tau(0, V, float(np.mean(1.0 / w)))
    xg, st, _, _, _ = run_both(P, N, V, B, b, w, 0, 0.005, 2, 10, tau, 0.5)
    assert rel_l2(xg, st.x) <= TOL


def test_fewview_smoothed_ramp_parity():
    # precond 3: Eq. 24's form with kappa = tau l (the few-view smoothed ramp),
    # against the oracle with the same taps, tau, sigma; and its automatic
    # sigma against the oracle's power-method bound
    P = need_gpu()
    N, V, B = 48, 16, 70
    x = synth.ellipse_phantom(N, 6, 2)
    b = f32(O.project(x, V, B))
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=1, iters=20, tv_iters=10, precond=3, tau=tau, sigma=0.3)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), None, prm)
    assert rep["kappa"] == pytest.approx(tau * O.fewview_ell(N, V, B), rel=1e-6)
    st, _ = O.pdtv(b, None, taps, 1, 0.0, tau, 0.3, 10, 20, N)
    assert rel_l2(to_np(xg), st.x) <= TOL
    # automatic sigma: rho / (tau ||A^T D A||), the norm against the 2-norm of
    # the explicitly built operator (a smaller case)
    N2, V2, B2 = 24, 16, 35
    g2 = P.Geometry(N2, V2, B2)
    b2 = f32(O.project(synth.ellipse_phantom(N2, 4, 1), V2, B2))
    _, rep = P.ct_pdtv_solve(g2, to_gpu(b2), None, P.PDTVParams(mode=1, iters=1, precond=3, norm_iters=40))
    t2 = O.ramp_taps(0, V2, B2, tau, tau * O.fewview_ell(N2, V2, B2))
    cols = []
    for j in range(N2 * N2):
        e = np.zeros(N2 * N2)
        e[j] = 1.0
        cols.append(O.backproject(O.filt(O.project(e.reshape(N2, N2), V2, B2), t2), N2).ravel())
    nada = np.linalg.norm(np.stack(cols, axis=1), 2)
    assert nada * (1 - 2e-4) <= rep["norm_ADA"] <= nada * 1.01
    assert rep["sigma"] == pytest.approx(0.95 / (tau * rep["norm_ADA"]), rel=1e-6)
    with pytest.raises(P.CTError):
        P.ct_pdtv_solve(g, to_gpu(b), to_gpu(np.ones((V, B))), P.PDTVParams(mode=0, iters=1, precond=3))


def test_repeated_solves_replay_a_graph():
    # a call with a workspace and no report is captured as a CUDA graph the
    # first time and replayed by the same call later: the results equal the
    # eager solve (report requested: kernels launched one by one), new data in
    # the same buffers is solved, each replay counts its kernels, and other
    # parameters get their own graph
    P = need_gpu()
    import torch
    N, V, B = 64, 90, 95
    _, b1, w1 = lowdose_case(N, V, B, 0)
    _, b2, w2 = lowdose_case(N, V, B, 1)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=10, beta=0.01)
    ws = P.workspace_for(g, prm)
    bd, wd = to_gpu(b1), to_gpu(w1)
    x = torch.empty(N, N, device="cuda")
    ref1, _ = P.ct_pdtv_solve(g, bd, wd, prm, workspace=ws)
    n0 = P.ct_kernel_launches()
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=x, workspace=ws, report=False)
    n1 = P.ct_kernel_launches()
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=x, workspace=ws, report=False)
    n2 = P.ct_kernel_launches()
    torch.cuda.synchronize()
    assert torch.equal(x, ref1)
    assert n1 - n0 > 100 and n2 - n1 == n1 - n0
    bd.copy_(to_gpu(b2))
    wd.copy_(to_gpu(w2))
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=x, workspace=ws, report=False)
    ref2, _ = P.ct_pdtv_solve(g, bd, wd, prm, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(x, ref2) and not torch.equal(ref1, ref2)
    prm3 = P.PDTVParams(mode=0, iters=7, beta=0.02)
    for _ in range(2):
        P.ct_pdtv_solve(g, bd, wd, prm3, x_out=x, workspace=ws, report=False)
    ref3, _ = P.ct_pdtv_solve(g, bd, wd, prm3, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(x, ref3)
    # and the first parameters still replay their own graph
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=x, workspace=ws, report=False)
    torch.cuda.synchronize()
    assert torch.equal(x, ref2)
    # new launch shapes drop the cached graphs: the next call is captured anew
    g.set_tuning(orbit_slices=2, tv_rows=8)
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=x, workspace=ws, report=False)
    ref4, _ = P.ct_pdtv_solve(g, bd, wd, prm, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(x, ref4)


def test_custom_angles_solve_parity():
    # irregular angles: the projector and backprojector without symmetry
    # sharing (k_project_mirror, k_backproject_tiles) inside the whole solve
    P = need_gpu()
    N, V, B = 48, 40, 71
    rng = np.random.default_rng(12)
    ang = np.sort(rng.uniform(0.0, np.pi, V))
    x = synth.ellipse_phantom(N, 6, 2) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x, V, B, angles=ang), 1e4, 3)
    b, w = f32(b), f32(w)
    tau = O.default_tau(0, V, float(np.mean(1.0 / w)))
    g = P.Geometry(N, V, B, angles=ang)
    prm = P.PDTVParams(mode=0, iters=15, beta=0.01, tau=tau, sigma=0.5)
    xg, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    taps = O.ramp_taps(0, V, B, tau, float(np.mean(1.0 / w)))
    st, _ = O.pdtv(b, w, taps, 0, 0.01, tau, 0.5, 10, 15, N, angles=ang)
    assert rel_l2(to_np(xg), st.x) <= TOL


@pytest.mark.parametrize("case", [dict(mode=0, precond=0), dict(mode=0, precond=2), dict(mode=1, precond=3),
                                  dict(mode=0, precond=1, tv_accel=1)],
                         ids=["plain_cp", "shift_variant", "fewview_smoothed", "fgp"])
def test_graph_replay_equals_eager_for_every_form(case):
    P = need_gpu()
    import torch
    N, V, B = 48, 60, 70
    x, b, w = lowdose_case(N, V, B, 4)
    if case["mode"] == 1:
        b, w = f32(O.project(synth.ellipse_phantom(N, 6, 4), V, B)), None
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(iters=9, beta=0.01, **case)
    ws = P.workspace_for(g, prm)
    bd = to_gpu(b)
    wd = None if w is None else to_gpu(w)
    ref, _ = P.ct_pdtv_solve(g, bd, wd, prm, workspace=ws)
    xo = torch.empty(N, N, device="cuda")
    for _ in range(3):
        P.ct_pdtv_solve(g, bd, wd, prm, x_out=xo, workspace=ws, report=False)
    torch.cuda.synchronize()
    assert torch.equal(xo, ref)


def test_solve_inside_a_callers_graph_capture():
    # inside the caller's own stream capture the library enqueues the kernels
    # (no graph of its own); replaying the caller's graph gives the eager result
    P = need_gpu()
    import torch
    N, V, B = 48, 60, 70
    x, b, w = lowdose_case(N, V, B, 5)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=6, beta=0.01)
    ws = P.workspace_for(g, prm)
    bd, wd = to_gpu(b), to_gpu(w)
    ref, _ = P.ct_pdtv_solve(g, bd, wd, prm, workspace=ws)
    xo = torch.zeros(N, N, device="cuda")
    P.ct_pdtv_solve(g, bd, wd, prm, x_out=xo, workspace=ws, report=False)   # warm (creates the fork stream)
    torch.cuda.synchronize()
    xo.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        P.ct_pdtv_solve(g, bd, wd, prm, x_out=xo, workspace=ws, report=False)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(xo, ref)
