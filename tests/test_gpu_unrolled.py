"""The differentiable form: the unrolled solve's forward against the FP64
oracle, and its hand-written backward (dL/dtaps, dL/dbeta) against FP64
central finite differences of the oracle's loss."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu


def make_batch(N, V, B, S, seed, i0=1e4):
    xs, bs, ws = [], [], []
    for s in range(S):
        x = synth.ellipse_phantom(N, 5, seed + s) * (2.0 / N)
        b, w = synth.poisson_data(O.project(x, V, B), i0, seed + 50 + s)
        xs.append(x)
        bs.append(f32(b))
        ws.append(f32(w))
    return np.stack(xs), np.stack(bs), np.stack(ws)


def steps_for(V, B, bs, ws, half):
    kappa = float(np.mean(1.0 / ws))
    tau = O.default_tau(0, V, kappa)
    taps = f32(O.ramp_taps(0, V, B, tau, kappa, half=half))
    return tau, taps


def oracle_loss(bs, ws, xt, taps, beta, tau, sigma, K, ntv, N):
    L = 0.0
    for s in range(bs.shape[0]):
        st, _ = O.pdtv(bs[s], ws[s], taps, 0, beta, tau, sigma, ntv, K, N)
        L += float(((st.x - xt[s]) ** 2).sum())
    return L / (bs.shape[0] * N * N)


def test_unrolled_forward_matches_oracle():
    P = need_gpu()
    N, V, B, S, K, ntv, half = 32, 45, 47, 2, 5, 6, 16
    xt, bs, ws = make_batch(N, V, B, S, 3)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.02
    g = P.Geometry(N, V, B)
    work = P.ct_pdtv_workspace_bytes  # noqa: F841  (keeps the binding import visible)
    import torch
    wsp = torch.empty(P.ct_unrolled_workspace_bytes(g, S, half, K, ntv), dtype=torch.uint8, device="cuda")
    x = P.ct_unrolled_forward(g, to_gpu(bs), to_gpu(ws), to_gpu(taps), tau, sigma, beta, 0, K, ntv, wsp)
    for s in range(S):
        st, _ = O.pdtv(bs[s], ws[s], taps, 0, beta, tau, sigma, ntv, K, N)
        assert rel_l2(to_np(x[s]), st.x) <= 1e-3


def test_unrolled_gradients_match_fp64_finite_differences():
    P = need_gpu()
    import torch
    N, V, B, S, K, ntv, half = 24, 30, 35, 2, 4, 5, 8
    xt, bs, ws = make_batch(N, V, B, S, 7)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.05
    g = P.Geometry(N, V, B)
    t = to_gpu(taps).requires_grad_(True)
    bt = torch.tensor(beta, device="cuda", requires_grad=True)
    x = P.UnrolledPDTV.apply(t, bt, g, to_gpu(bs), to_gpu(ws), tau, sigma, 0, K, ntv)
    loss = ((x - to_gpu(xt)) ** 2).sum() / (S * N * N)
    loss.backward()
    gt, gb = to_np(t.grad), float(bt.grad)
    L0 = oracle_loss(bs, ws, xt, taps, beta, tau, sigma, K, ntv, N)
    assert abs(float(loss.detach()) - L0) <= 1e-4 * L0
    # beta
    hb = 1e-3 * beta
    fd_b = (oracle_loss(bs, ws, xt, taps, beta + hb, tau, sigma, K, ntv, N) -
            oracle_loss(bs, ws, xt, taps, beta - hb, tau, sigma, K, ntv, N)) / (2 * hb)
    assert gb == pytest.approx(fd_b, rel=1e-4)
    # taps: two random directions and the centre tap
    rng = np.random.default_rng(0)
    dirs = [rng.standard_normal(taps.size), np.eye(taps.size)[half - 1]]
    for d in dirs:
        eps = 1e-4 * np.abs(taps).max() / np.abs(d).max()
        fd = (oracle_loss(bs, ws, xt, taps + eps * d, beta, tau, sigma, K, ntv, N) -
              oracle_loss(bs, ws, xt, taps - eps * d, beta, tau, sigma, K, ntv, N)) / (2 * eps)
        got = float(gt @ d)
        assert got == pytest.approx(fd, rel=3e-3)


@pytest.mark.parametrize("case", [
    # 150 taps: 299 lags, two passes of the correlation's lag loop
    dict(mode=0, N=20, V=24, B=170, S=2, K=3, ntv=4, half=150),
    # Algorithm 2: one correlation pair per iteration, lambda = tau
    dict(mode=1, N=24, V=12, B=35, S=2, K=4, ntv=5, half=8),
    # no prox steps: the whole-image single-step path instead of the tiled one
    dict(mode=0, N=24, V=30, B=35, S=1, K=4, ntv=0, half=8),
    # 64^2: prox-adjoint tiles inside the image (the path without bounds tests) and at its edges
    dict(mode=0, N=64, V=24, B=95, S=1, K=3, ntv=4, half=8),
], ids=["lowdose_299_lags", "fewview", "no_tv_steps", "interior_tiles_64"])
def test_unrolled_gradients_more_cases(case):
    P = need_gpu()
    import torch
    c = case
    N, V, B, S, K, ntv, half, mode = c["N"], c["V"], c["B"], c["S"], c["K"], c["ntv"], c["half"], c["mode"]
    xt, bs, ws = make_batch(N, V, B, S, 11)
    tau, taps = steps_for(V, B, bs, ws, half)
    if mode == 1:   # noiseless data of the phantoms, no weights
        bs = np.stack([f32(O.project(xt[s], V, B)) for s in range(S)])
    sigma, beta = 0.5, 0.05
    g = P.Geometry(N, V, B)
    t = to_gpu(taps).requires_grad_(True)
    bt = torch.tensor(beta, device="cuda", requires_grad=True)
    wg = to_gpu(ws) if mode == 0 else None
    x = P.UnrolledPDTV.apply(t, bt, g, to_gpu(bs), wg, tau, sigma, mode, K, ntv)
    loss = ((x - to_gpu(xt)) ** 2).sum() / (S * N * N)
    loss.backward()
    gt = to_np(t.grad)

    def oloss(tp, be):
        L = 0.0
        for s in range(S):
            st, _ = O.pdtv(bs[s], ws[s] if mode == 0 else None, tp, mode, be, tau, sigma, ntv, K, N)
            L += float(((st.x - xt[s]) ** 2).sum())
        return L / (S * N * N)

    L0 = oloss(taps, beta)
    assert abs(float(loss.detach()) - L0) <= 1e-4 * L0
    if mode == 0 and ntv > 0:
        hb = 1e-3 * beta
        fd_b = (oloss(taps, beta + hb) - oloss(taps, beta - hb)) / (2 * hb)
        assert float(bt.grad) == pytest.approx(fd_b, rel=1e-4)
    rng = np.random.default_rng(1)
    for d in [rng.standard_normal(taps.size), np.eye(taps.size)[half - 1], np.eye(taps.size)[0],
              np.eye(taps.size)[-1]]:
        eps = 1e-4 * np.abs(taps).max() / np.abs(d).max()
        fd = (oloss(taps + eps * d, beta) - oloss(taps - eps * d, beta)) / (2 * eps)
        assert float(gt @ d) == pytest.approx(fd, rel=3e-3, abs=1e-4 * np.abs(gt).max())


def test_project_backproject_autograd_are_adjoint():
    P = need_gpu()
    import torch
    N, V, B = 40, 30, 57
    g = P.Geometry(N, V, B)
    x = to_gpu(synth.random_image(N, 1)).requires_grad_(True)
    y = to_gpu(synth.random_sinogram(V, B, 2))
    (P.project(g, x) * y).sum().backward()
    assert rel_l2(to_np(x.grad), to_np(P.ct_backproject(g, y))) < 1e-6
    y2 = y.clone().requires_grad_(True)
    (P.backproject(g, y2) * x.detach()).sum().backward()
    assert rel_l2(to_np(y2.grad), to_np(P.ct_project(g, x.detach()))) < 1e-6


def test_unrolled_module_at_scale():
    # batch 16 of 256^2, 180 views, 368 bins, 10 unrolled iterations,
    # learnable log beta and 128 one-sided taps: forward and backward run and
    # give finite gradients of the MSE loss.
    P = need_gpu()
    import torch
    N, V, B, S = 256, 180, 368, 16
    g = P.Geometry(N, V, B)
    xt = torch.from_numpy(np.stack([synth.ellipse_phantom(N, 10, s) * (2.0 / N) for s in range(S)]).astype(np.float32)).cuda()
    p = P.ct_project(g, xt).cpu().numpy()
    b, w = synth.poisson_data(p, 1e4, 1)
    b, w = to_gpu(b), to_gpu(w)
    _, rep = P.ct_pdtv_solve(g, b[0], w[0], P.PDTVParams(mode=0, iters=0, beta=0.01))
    taps0 = P.ct_ramp_taps(g, 0, rep["tau"], rep["kappa"])
    m = P.UnrolledReconstructor(g, taps0, 0.01, rep["tau"], 0.9 * rep["sigma"], iters=10, tv_iters=10, half=128)
    x = m(b, w)
    loss = ((x - xt) ** 2).mean()
    loss.backward()
    assert torch.isfinite(loss)
    assert torch.isfinite(m.taps_half.grad).all() and torch.isfinite(m.log_beta.grad)
    assert float(m.taps_half.grad.abs().max()) > 0


def test_unrolled_full_size_sampled_slices_match_oracle():
    # the differentiable configuration as the bench runs it (16 x 256^2,
    # 180 views, 368 bins, K = 10, n_tv = 10, 128 one-sided taps): slices
    # 0 and 11 of the batch against the oracle
    P = need_gpu()
    N, V, B, S, K, ntv, half = 256, 180, 368, 16, 10, 10, 128
    xt, bs, ws = make_batch(N, V, B, S, 21)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.01
    g = P.Geometry(N, V, B)
    import torch
    x = P.UnrolledPDTV.apply(to_gpu(taps), torch.tensor(beta, device="cuda"), g, to_gpu(bs), to_gpu(ws), tau,
                             sigma, 0, K, ntv)
    for s in (0, 11):
        st, _ = O.pdtv(bs[s], ws[s], taps, 0, beta, tau, sigma, ntv, K, N)
        assert rel_l2(to_np(x[s]), st.x) <= 1e-3


def test_unrolled_full_size_gradients_match_fp64_finite_differences():
    # one full-size slice (256^2, 180 views, 368 bins, K = 10, 128 taps):
    # dL/dbeta and one random tap direction against central differences of
    # the oracle's loss
    P = need_gpu()
    import torch
    N, V, B, S, K, ntv, half = 256, 180, 368, 1, 10, 10, 128
    xt, bs, ws = make_batch(N, V, B, S, 31)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.01
    g = P.Geometry(N, V, B)
    t = to_gpu(taps).requires_grad_(True)
    bt = torch.tensor(beta, device="cuda", requires_grad=True)
    x = P.UnrolledPDTV.apply(t, bt, g, to_gpu(bs), to_gpu(ws), tau, sigma, 0, K, ntv)
    loss = ((x - to_gpu(xt)) ** 2).sum() / (S * N * N)
    loss.backward()
    hb = 1e-3 * beta
    fd_b = (oracle_loss(bs, ws, xt, taps, beta + hb, tau, sigma, K, ntv, N) -
            oracle_loss(bs, ws, xt, taps, beta - hb, tau, sigma, K, ntv, N)) / (2 * hb)
    assert float(bt.grad) == pytest.approx(fd_b, rel=1e-3)
    d = np.random.default_rng(2).standard_normal(taps.size)
    eps = 1e-4 * np.abs(taps).max() / np.abs(d).max()
    fd = (oracle_loss(bs, ws, xt, taps + eps * d, beta, tau, sigma, K, ntv, N) -
          oracle_loss(bs, ws, xt, taps - eps * d, beta, tau, sigma, K, ntv, N)) / (2 * eps)
    assert float(to_np(t.grad) @ d) == pytest.approx(fd, rel=3e-3)


def test_unrolled_custom_angles_gradients():
    # irregular angles: the unrolled solve on the projector and backprojector
    # without symmetry sharing; forward against the oracle, dL/dbeta and a
    # tap direction against FP64 central differences
    P = need_gpu()
    import torch
    N, V, B, S, K, ntv, half = 24, 20, 35, 2, 3, 4, 8
    rng = np.random.default_rng(13)
    ang = np.sort(rng.uniform(0.0, np.pi, V))
    xs, bs, ws = [], [], []
    for s in range(S):
        x = synth.ellipse_phantom(N, 5, 60 + s) * (2.0 / N)
        b, w = synth.poisson_data(O.project(x, V, B, angles=ang), 1e4, 70 + s)
        xs.append(x)
        bs.append(f32(b))
        ws.append(f32(w))
    xt, bs, ws = np.stack(xs), np.stack(bs), np.stack(ws)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.05
    g = P.Geometry(N, V, B, angles=ang)
    t = to_gpu(taps).requires_grad_(True)
    bt = torch.tensor(beta, device="cuda", requires_grad=True)
    x = P.UnrolledPDTV.apply(t, bt, g, to_gpu(bs), to_gpu(ws), tau, sigma, 0, K, ntv)
    loss = ((x - to_gpu(xt)) ** 2).sum() / (S * N * N)
    loss.backward()

    def oloss(tp, be):
        L = 0.0
        for s in range(S):
            st, _ = O.pdtv(bs[s], ws[s], tp, 0, be, tau, sigma, ntv, K, N, angles=ang)
            L += float(((st.x - xt[s]) ** 2).sum())
        return L / (S * N * N)

    assert abs(float(loss.detach()) - oloss(taps, beta)) <= 1e-4 * oloss(taps, beta)
    hb = 1e-3 * beta
    fd_b = (oloss(taps, beta + hb) - oloss(taps, beta - hb)) / (2 * hb)
    assert float(bt.grad) == pytest.approx(fd_b, rel=1e-4)
    d = np.random.default_rng(3).standard_normal(taps.size)
    eps = 1e-4 * np.abs(taps).max() / np.abs(d).max()
    fd = (oloss(taps + eps * d, beta) - oloss(taps - eps * d, beta)) / (2 * eps)
    assert float(to_np(t.grad) @ d) == pytest.approx(fd, rel=3e-3)


@pytest.mark.parametrize("mode", [0, 1])
def test_unrolled_backward_is_deterministic_and_capturable(mode):
    # the tap correlations run on a side stream beside the other adjoints:
    # repeated calls give the same gradients bit for bit, on another caller
    # stream too, and forward + backward captured in a CUDA graph replay to
    # the eager results
    P = need_gpu()
    import torch
    N, V, B, S, K, ntv, half = 64, 90, 95, 4, 3, 5, 16
    xt, bs, ws = make_batch(N, V, B, S, 21)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.02
    g = P.Geometry(N, V, B)
    bd, td = to_gpu(bs), to_gpu(taps)
    wd = to_gpu(ws) if mode == 0 else None
    wsp = torch.empty(P.ct_unrolled_workspace_bytes(g, S, half, K, ntv), dtype=torch.uint8, device="cuda")
    gx = to_gpu(np.random.default_rng(5).standard_normal((S, N, N)))

    def run():
        x = P.ct_unrolled_forward(g, bd, wd, td, tau, sigma, beta, mode, K, ntv, wsp)
        return x, P.ct_unrolled_backward(g, bd, wd, td, tau, sigma, beta, mode, K, ntv, gx, wsp)

    x0, g0 = run()
    x1, g1 = run()
    torch.cuda.synchronize()
    assert torch.equal(x0, x1) and torch.equal(g0, g1)
    assert float(g0[:2 * half - 1].abs().max()) > 0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        x2, g2 = run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    assert torch.equal(x0, x2) and torch.equal(g0, g2)
    xo = torch.zeros(S, N, N, device="cuda")
    go = torch.zeros(2 * half, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        xc, gc = run()
        xo.copy_(xc)
        go.copy_(gc)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(xo, x0) and torch.equal(go, g0)


def test_unrolled_with_one_and_two_orbit_slices():
    # the orbit backprojector writes A^T y (forward: z = x - tau A^T mubar;
    # backward: gz = gx - tau A^T gr) itself when the base views form one
    # slice, and through the slice reduction with two: both give the same
    # x_K and gradients to rounding, and the single-slice gradients match
    # FP64 central differences of the oracle's loss
    P = need_gpu()
    import torch
    N, V, B, S, K, ntv, half = 32, 40, 47, 2, 4, 5, 8
    xt, bs, ws = make_batch(N, V, B, S, 13)
    tau, taps = steps_for(V, B, bs, ws, half)
    sigma, beta = 0.5, 0.03
    g = P.Geometry(N, V, B)
    out = {}
    for nsl in (1, 2):
        g.set_tuning(orbit_slices=nsl)
        t = to_gpu(taps).requires_grad_(True)
        bt = torch.tensor(beta, device="cuda", requires_grad=True)
        x = P.UnrolledPDTV.apply(t, bt, g, to_gpu(bs), to_gpu(ws), tau, sigma, 0, K, ntv)
        loss = ((x - to_gpu(xt)) ** 2).sum() / (S * N * N)
        loss.backward()
        out[nsl] = (to_np(x), to_np(t.grad), float(bt.grad))
    x1, gt1, gb1 = out[1]
    x2, gt2, gb2 = out[2]
    assert rel_l2(x1, x2) <= 1e-5
    assert rel_l2(gt1, gt2) <= 1e-4 and gb1 == pytest.approx(gb2, rel=1e-4)
    hb = 1e-3 * beta
    fd_b = (oracle_loss(bs, ws, xt, taps, beta + hb, tau, sigma, K, ntv, N) -
            oracle_loss(bs, ws, xt, taps, beta - hb, tau, sigma, K, ntv, N)) / (2 * hb)
    assert gb1 == pytest.approx(fd_b, rel=1e-4)
    d = np.random.default_rng(5).standard_normal(taps.size)
    eps = 1e-4 * np.abs(taps).max() / np.abs(d).max()
    fd = (oracle_loss(bs, ws, xt, taps + eps * d, beta, tau, sigma, K, ntv, N) -
          oracle_loss(bs, ws, xt, taps - eps * d, beta, tau, sigma, K, ntv, N)) / (2 * eps)
    assert float(gt1 @ d) == pytest.approx(fd, rel=3e-3)
