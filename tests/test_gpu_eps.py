"""GPU parity of the error-tolerant few-view form (min TV(x) s.t.
||Ax - b|| <= eps, x >= 0; Sec. 5 names it without its steps: the dual step
is the proximal map of the eps-ball's support function) against the FP64 oracle, whose
dual step is computed independently (bisection with dense Cholesky solves
instead of the eigenbasis): relative L2 <= 1e-3 on the image after the
stated iterations, for the paper's ramp, the few-view smoothed ramp and
D = I; plus the ends of eps, resume, the eigenbasis cache and argument
checks."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-3


def noisy_fewview(N, V, B, seed, rel_noise=0.02):
    x = synth.ellipse_phantom(N, 8, seed)
    clean = O.project(x, V, B)
    rng = np.random.default_rng(seed + 40)
    noise = rel_noise * np.abs(clean).mean() * rng.standard_normal((V, B))
    b = f32(clean + noise)
    return x, b, float(np.linalg.norm(b - clean))


def oracle_taps(precond, N, V, B, tau):
    if precond == 1:
        return O.ramp_taps(1, V, B, tau)
    if precond == 3:
        return O.ramp_taps(0, V, B, tau, tau * O.fewview_ell(N, V, B))
    return np.ones(1)


def solve_both(P, N, V, B, b, eps, precond, iters, tau, sigma, ntv=10, g=None):
    g = g or P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=iters, tv_iters=ntv, precond=precond, tau=tau, sigma=sigma,
                       eps=eps)
    ws = P.workspace_for(g, prm)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), None, prm, workspace=ws)
    st, _ = O.pdtv(b, None, oracle_taps(precond, N, V, B, tau), 1, 0.0, tau, sigma, ntv, iters, N, eps=eps)
    return to_np(xg), st, g, prm, ws


@pytest.mark.parametrize("precond", [1, 3, 0])
def test_eps_form_parity(precond):
    P = need_gpu()
    N, V, B = 32, 16, 47
    x, b, nn = noisy_fewview(N, V, B, 1)
    tau = O.default_tau(1, V, 0.0)
    sigma, _, _ = O.step_sizes(1, N, V, B, oracle_taps(precond, N, V, B, tau), None, tau)
    xg, st, _, _, _ = solve_both(P, N, V, B, b, nn, precond, 20, tau, sigma)
    assert rel_l2(xg, st.x) <= TOL
    # the tolerance matters: the equality form's iterate is far away
    se, _ = O.pdtv(b, None, oracle_taps(precond, N, V, B, tau), 1, 0.0, tau, sigma, 10, 20, N)
    assert rel_l2(se.x, st.x) > 20 * TOL


def test_eps_form_ends():
    P = need_gpu()
    N, V, B = 24, 12, 35
    x, b, nn = noisy_fewview(N, V, B, 2)
    tau = O.default_tau(1, V, 0.0)
    sigma, _, _ = O.step_sizes(1, N, V, B, oracle_taps(1, N, V, B, tau), None, tau)
    # eps above |b|: every dual step is 0, x stays 0
    xg, st, _, _, _ = solve_both(P, N, V, B, b, 1.5 * float(np.linalg.norm(b)), 1, 8, tau, sigma)
    assert not st.x.any() and not xg.any()
    # a tiny eps: next to the equality form
    xg, st, _, _, _ = solve_both(P, N, V, B, b, 1e-6 * nn, 1, 8, tau, sigma)
    assert rel_l2(xg, st.x) <= TOL


def test_eps_form_resume_and_cache():
    P = need_gpu()
    N, V, B = 32, 16, 47
    x, b, nn = noisy_fewview(N, V, B, 3)
    g = P.Geometry(N, V, B)
    tau = O.default_tau(1, V, 0.0)
    sigma, _, _ = O.step_sizes(1, N, V, B, oracle_taps(1, N, V, B, tau), None, tau)
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=12, precond=1, tau=tau, sigma=sigma, eps=nn)
    ws = P.workspace_for(g, prm)
    x12, _ = P.ct_pdtv_solve(g, to_gpu(b), None, prm, workspace=ws)
    half = P.PDTVParams(**{**prm.__dict__, "iters": 5})
    ws2 = P.workspace_for(g, half)
    xr, _ = P.ct_pdtv_solve(g, to_gpu(b), None, half, workspace=ws2)
    xr, _ = P.ct_pdtv_solve(g, to_gpu(b), None, P.PDTVParams(**{**prm.__dict__, "iters": 7, "resume": 1}),
                            x_out=xr, workspace=ws2)
    assert np.array_equal(to_np(xr), to_np(x12))
    # another tau on the same geometry gets its own eigenbasis; the first stays right
    tau2 = 2.0 * tau
    s2, _, _ = O.step_sizes(1, N, V, B, oracle_taps(1, N, V, B, tau2), None, tau2)
    xg2, st2, _, _, _ = solve_both(P, N, V, B, b, nn, 1, 10, tau2, s2, g=g)
    assert rel_l2(xg2, st2.x) <= TOL
    xg1, st1, _, _, _ = solve_both(P, N, V, B, b, nn, 1, 10, tau, sigma, g=g)
    assert rel_l2(xg1, st1.x) <= TOL


def test_eps_form_paper_fewview_shape():
    # 256^2 from 32 views, 369 bins (the paper's few-view shape), 3 iterations
    P = need_gpu()
    N, V, B = 256, 32, 369
    x, b, nn = noisy_fewview(N, V, B, 4, rel_noise=0.01)
    tau = O.default_tau(1, V, 0.0)
    g = P.Geometry(N, V, B)
    sigma, _, _ = O.step_sizes(1, N, V, B, oracle_taps(3, N, V, B, tau), None, tau)
    xg, st, _, _, _ = solve_both(P, N, V, B, b, nn, 3, 3, tau, sigma, g=g)
    assert rel_l2(xg, st.x) <= TOL


def test_eps_form_argument_checks():
    P = need_gpu()
    N, V, B = 16, 8, 23
    g = P.Geometry(N, V, B)
    b = to_gpu(np.zeros((V, B)))
    w = to_gpu(np.ones((V, B)))
    for prm, ww in [(P.PDTVParams(mode=P.CT_FEWVIEW, iters=1, eps=-1.0), None),
                    (P.PDTVParams(mode=P.CT_LOWDOSE, iters=1, eps=1.0, beta=0.1), w),
                    (P.PDTVParams(mode=P.CT_FEWVIEW, iters=1, eps=float("inf")), None),
                    (P.PDTVParams(mode=P.CT_FEWVIEW, iters=1, eps=1.0, precond=2), None)]:
        with pytest.raises(P.CTError):
            P.ct_pdtv_solve(g, b, ww, prm)


def test_eps_form_in_batched_solve_and_graph():
    # an error-tolerant slice beside an equality slice in one batched call:
    # each equals its own single solve bit for bit; once its eigenbasis is
    # cached, the call replays from a CUDA graph
    P = need_gpu()
    import torch
    N, V, B = 32, 16, 47
    x1, b1, nn1 = noisy_fewview(N, V, B, 5)
    x2, b2, _ = noisy_fewview(N, V, B, 6)
    g1, g2 = P.Geometry(N, V, B), P.Geometry(N, V, B)
    tau = O.default_tau(1, V, 0.0)
    p1 = P.PDTVParams(mode=P.CT_FEWVIEW, iters=10, precond=3, tau=tau, eps=nn1)
    p2 = P.PDTVParams(mode=P.CT_FEWVIEW, iters=10, precond=3, tau=tau)
    s1, _ = P.ct_pdtv_solve(g1, to_gpu(b1), None, p1)
    s2, _ = P.ct_pdtv_solve(g2, to_gpu(b2), None, p2)
    bs = P.BatchedSolve([(g1, to_gpu(b1), None, p1), (g2, to_gpu(b2), None, p2)])
    xs, _ = bs.run()
    torch.cuda.synchronize()
    assert np.array_equal(to_np(xs[0]), to_np(s1)) and np.array_equal(to_np(xs[1]), to_np(s2))
    for x in bs.x:
        x.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bs.run()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_np(bs.x[0]), to_np(s1)) and np.array_equal(to_np(bs.x[1]), to_np(s2))


def test_eps_form_first_solve_refuses_capture():
    # the first solve for a (geometry, precond, tau) reads the taps back to the
    # host for the eigendecomposition: inside stream capture it returns an
    # error instead
    P = need_gpu()
    import torch
    N, V, B = 24, 12, 35
    _, b, nn = noisy_fewview(N, V, B, 8)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=2, precond=1, tau=0.0123, eps=nn)
    ws = P.workspace_for(g, prm)
    bg = to_gpu(b)
    x = torch.empty(N, N, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(P.CTError):
        with torch.cuda.graph(graph):
            P.ct_pdtv_solve(g, bg, None, prm, x_out=x, workspace=ws, report=False)
    torch.cuda.synchronize()
    # uncaptured it runs, and then capture works
    P.ct_pdtv_solve(g, bg, None, prm, x_out=x, workspace=ws, report=False)
    torch.cuda.synchronize()
    ref = to_np(x).copy()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        P.ct_pdtv_solve(g, bg, None, prm, x_out=x, workspace=ws, report=False)
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_np(x), ref)


@pytest.mark.parametrize("precond", [3, 0])
def test_eps_form_replayed_solves_equal_eager(precond):
    # once the eigenbasis is cached, a call with a workspace and no report is
    # captured and replayed by the library; the results equal the eager solve
    P = need_gpu()
    import torch
    N, V, B = 32, 16, 47
    _, b, nn = noisy_fewview(N, V, B, 9)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=12, precond=precond, tau=O.default_tau(1, V, 0.0), eps=nn)
    ws = P.workspace_for(g, prm)
    bg = to_gpu(b)
    ref, _ = P.ct_pdtv_solve(g, bg, None, prm, workspace=ws)       # eager (report): caches the basis
    x = torch.empty(N, N, device="cuda")
    n0 = P.ct_kernel_launches()
    for _ in range(3):
        P.ct_pdtv_solve(g, bg, None, prm, x_out=x, workspace=ws, report=False)
    n1 = P.ct_kernel_launches()
    torch.cuda.synchronize()
    assert torch.equal(x, ref)
    assert (n1 - n0) % 3 == 0 and n1 > n0


def test_eps_form_custom_angles():
    P = need_gpu()
    N, V, B = 32, 14, 47
    rng = np.random.default_rng(14)
    ang = np.sort(rng.uniform(0.0, np.pi, V))
    x = synth.ellipse_phantom(N, 8, 10)
    clean = O.project(x, V, B, angles=ang)
    noise = 0.02 * np.abs(clean).mean() * np.random.default_rng(15).standard_normal((V, B))
    b = f32(clean + noise)
    nn = float(np.linalg.norm(b - clean))
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(1, V, B, tau)
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau, angles=ang)
    g = P.Geometry(N, V, B, angles=ang)
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=15, precond=1, tau=tau, sigma=sigma, eps=nn)
    xg, _ = P.ct_pdtv_solve(g, to_gpu(b), None, prm)
    st, _ = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, 15, N, angles=ang, eps=nn)
    assert rel_l2(to_np(xg), st.x) <= TOL
