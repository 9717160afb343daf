"""Whole-solve parity at the benchmarked workloads, for their full
iteration counts and in the launch configuration the benchmark times:
launch shapes from ct_geometry_autotune, workspace given and no report, so
that repeated calls replay the library's solve graph.

  * low-dose 512^2, 720 views, 736 bins, I0 = 5e3, beta = 0.005, 30
    iterations of Algorithm 1 (the headline workload);
  * few-view 512^2, 32 views, 736 bins, noiseless, 100 iterations of
    Algorithm 2 (its projector runs the four-deep staging variant).

tau is the default of each form and sigma comes from the oracle's power
method, both passed explicitly to both sides; the oracle (FP64, OpenMP over
views / image rows) runs the same iterations.  Bar: relative L2 <= 1e-3 on
x^K; the element-wise maximum error is reported beside it."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-3


def solve_like_the_bench(P, g, b, w, prm):
    # the timed path: explicit workspace, no report; the second identical
    # call replays the solve graph captured by the first
    ws = P.workspace_for(g, prm)
    tb, tw = to_gpu(b), (None if w is None else to_gpu(w))
    x, _ = P.ct_pdtv_solve(g, tb, tw, prm, workspace=ws, report=False)
    x.zero_()
    P.ct_pdtv_solve(g, tb, tw, prm, x_out=x, workspace=ws, report=False)
    P.ct_pdtv_status(ws)
    return to_np(x)


def report(record_property, name, xg, xo):
    r = rel_l2(xg, xo)
    mx = float(np.abs(xg - xo).max() / np.abs(xo).max())
    record_property(name + "_rel_l2", r)
    record_property(name + "_max_err_rel_to_max", mx)
    print(f"{name}: rel L2 {r:.3e}, max |dx| / max |x| {mx:.3e}")
    return r, mx


def test_lowdose_512_v720_30_iterations(record_property):
    P = need_gpu()
    cfg = synth.CONFIGS["lowdose_512"]
    N, V, B = cfg["n"], cfg["views"], cfg["bins"]
    x = synth.ellipse_phantom(N, cfg["ellipses"], 0) * cfg["scale"]
    b, w = synth.poisson_data(O.project(x, V, B), cfg["i0"], 100)
    b, w = f32(b), f32(w)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(0, N, V, B, taps, w, tau, iters=20)
    g = P.Geometry(N, V, B)
    g.autotune()
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=cfg["iters"], tv_iters=10, beta=cfg["beta"], tau=tau, sigma=sigma)
    xg = solve_like_the_bench(P, g, b, w, prm)
    st, _ = O.pdtv(b, w, taps, 0, cfg["beta"], tau, sigma, 10, cfg["iters"], N)
    r, mx = report(record_property, "lowdose_512", xg, st.x)
    assert r <= TOL
    assert mx <= 10 * TOL


def test_fewview_512_v32_100_iterations(record_property):
    P = need_gpu()
    cfg = synth.CONFIGS["fewview_512"]
    N, V, B = cfg["n"], cfg["views"], cfg["bins"]
    b = f32(O.project(synth.ellipse_phantom(N, cfg["ellipses"], 0), V, B))
    tau = O.default_tau(1, V, 0.0)
    taps = O.ramp_taps(1, V, B, tau)
    sigma, _, _ = O.step_sizes(1, N, V, B, taps, None, tau)
    g = P.Geometry(N, V, B)
    tun = g.autotune()
    prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=cfg["iters"], tv_iters=10, tau=tau, sigma=sigma)
    xg = solve_like_the_bench(P, g, b, None, prm)
    st, _ = O.pdtv(b, None, taps, 1, 0.0, tau, sigma, 10, cfg["iters"], N)
    r, mx = report(record_property, "fewview_512", xg, st.x)
    record_property("fewview_512_tuning", str(tun))
    assert r <= TOL
    assert mx <= 10 * TOL


def test_batched_64_mixed_slices_sampled(record_property):
    # the batched workload as the benchmark builds it: 64 slices of mixed
    # N (256, 384, 512), views (32, 90, 360, 720), bins ceil(1.44 N) and
    # mode, 30 iterations each, launch shapes tuned per geometry, one
    # ct_pdtv_solve_batched call in the persistent form and in the
    # stream-pool form.  Every slice agrees bit for bit between the two
    # forms; four sampled slices (few-view 256^2/32 and 384^2/90, low-dose
    # 384^2/720 and 512^2/720), whose tau and sigma are set from the
    # oracle, match the oracle's 30 iterations.
    P = need_gpu()
    import torch
    shapes = synth.mixed_slices(64, 0)
    sampled = [2, 1, 5, 27]
    slices, geoms, cases = [], {}, {}
    for i, (n, v, nb, mode, sd) in enumerate(shapes):
        g = geoms.setdefault((n, v, nb), P.Geometry(n, v, nb))
        x = synth.ellipse_phantom(n, 10, sd) * ((2.0 / n) if mode == 0 else 1.0)
        p = O.project(x, v, nb)
        if mode == 0:
            b, w = synth.poisson_data(p, 1e4, sd)
            b, w = f32(b), f32(w)
        else:
            b, w = f32(p), None
        prm = P.PDTVParams(mode=mode, iters=30, tv_iters=10, beta=0.005)
        if i in sampled:
            kappa = float(np.mean(1.0 / w)) if mode == 0 else 0.0
            prm.tau = O.default_tau(mode, v, kappa)
            taps = O.ramp_taps(mode, v, nb, prm.tau, kappa)
            prm.sigma, _, _ = O.step_sizes(mode, n, v, nb, taps, w, prm.tau, iters=20)
            cases[i] = (b, w, taps, mode, prm.tau, prm.sigma, n)
        slices.append((g, to_gpu(b), None if w is None else to_gpu(w), prm))
    bs = P.BatchedSolve(slices, autotune=True)
    bs.form = P.CT_BATCH_AUTO            # the persistent launch (every slice qualifies)
    xs, _ = bs.run()
    torch.cuda.synchronize()
    persistent = [to_np(x).copy() for x in xs]
    bs.form = P.CT_BATCH_POOL
    xs, _ = bs.run()
    torch.cuda.synchronize()
    for i, x in enumerate(xs):
        assert np.array_equal(to_np(x), persistent[i]), i
    for i, (b, w, taps, mode, tau, sigma, n) in cases.items():
        st, _ = O.pdtv(b, w, taps, mode, 0.005 if mode == 0 else 0.0, tau, sigma, 10, 30, n)
        r, mx = report(record_property, f"batched_slice_{i}", persistent[i], st.x)
        assert r <= TOL, i
        assert mx <= 10 * TOL, i
