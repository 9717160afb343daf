"""The batched form: many slices of mixed geometry and mode in one call
(ct_pdtv_solve_batched).  Each slice must equal its single-slice solve bit
for bit, match the FP64 oracle, and replay identically from a CUDA graph."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu


def make_slices(P, shapes, iters, oracle_data=True, explicit_steps=False):
    """Slices of the given shapes; with explicit_steps, tau and sigma are set
    from the oracle (default tau, sigma by the oracle's power method), so an
    oracle run with the same values needs nothing from the GPU."""
    out = []
    for n, v, b, mode, sd in shapes:
        g = P.Geometry(n, v, b)
        if mode == 0:
            x = synth.ellipse_phantom(n, 6, sd) * (2.0 / n)
            bb, w = synth.poisson_data(O.project(x, v, b), 1e4, sd)
            w = to_gpu(f32(w))
        else:
            bb = O.project(synth.ellipse_phantom(n, 6, sd), v, b)
            w = None
        prm = P.PDTVParams(mode=mode, iters=iters, beta=0.01)
        if explicit_steps:
            wh = None if w is None else to_np(w)
            kappa = float(np.mean(1.0 / wh)) if mode == 0 else 0.0
            prm.tau = O.default_tau(mode, v, kappa)
            taps = O.ramp_taps(mode, v, b, prm.tau, kappa)
            prm.sigma, _, _ = O.step_sizes(mode, n, v, b, taps, wh, prm.tau)
        out.append((g, to_gpu(f32(bb)), w, prm))
    return out


def test_batched_equals_single_slice_solves():
    P = need_gpu()
    shapes = [(48, 60, 70, 0, 1), (32, 8, 47, 1, 2), (64, 90, 95, 0, 3), (40, 12, 58, 1, 4), (48, 60, 70, 0, 5),
              (17, 30, 25, 0, 6)]
    slices = make_slices(P, shapes, 6)
    xs, reps = P.ct_pdtv_solve_batched(slices)
    for (g, b, w, prm), xb, rep in zip(slices, xs, reps):
        x1, rep1 = P.ct_pdtv_solve(g, b, w, prm)
        assert np.array_equal(to_np(xb), to_np(x1))
        assert rep["sigma"] == rep1["sigma"] and rep["k"] == 6


def test_batched_matches_oracle():
    P = need_gpu()
    shapes = [(32, 45, 47, 0, 11), (40, 10, 58, 1, 12), (24, 36, 35, 0, 13)]
    slices = make_slices(P, shapes, 8, explicit_steps=True)
    xs, reps = P.ct_pdtv_solve_batched(slices)
    for (g, b, w, prm), xb, rep, (n, v, nb, mode, sd) in zip(slices, xs, reps, shapes):
        bh = to_np(b)
        wh = None if w is None else to_np(w)
        kappa = float(np.mean(1.0 / wh)) if mode == 0 else 0.0
        taps = O.ramp_taps(mode, v, nb, prm.tau, kappa)
        st, _ = O.pdtv(bh, wh, taps, mode, 0.01, prm.tau, prm.sigma, 10, 8, n)
        assert rel_l2(to_np(xb), st.x) <= 1e-3


def test_batched_graph_replay():
    P = need_gpu()
    import torch
    shapes = synth.mixed_slices(8, 7, sizes=(32, 48, 64), views=(16, 45, 90))
    slices = make_slices(P, shapes, 5)
    bs = P.BatchedSolve(slices)
    xs, _ = bs.run()                      # eager (creates the stream pool)
    torch.cuda.synchronize()
    ref = [to_np(x).copy() for x in xs]
    for x in bs.x:
        x.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bs.run()
    graph.replay()
    torch.cuda.synchronize()
    for x, r in zip(bs.x, ref):
        assert np.array_equal(to_np(x), r)


def test_batched_rejects_bad_slices():
    P = need_gpu()
    slices = make_slices(P, [(16, 20, 24, 0, 1)], 2)
    g, b, w, prm = slices[0]
    with pytest.raises(P.CTError):
        P.ct_pdtv_solve_batched([(g, b, None, prm)])


# ---------------------------------------------------------------------------
# The persistent form: when every slice qualifies (default angles, N a
# multiple of 32, V even, the same iteration count), the batched call runs
# the slices' setups on the stream pool and all their iterations in one
# persistent launch.  Its item bodies are the single-slice kernels' bodies
# with the same launch shapes, so each slice equals its single solve bit
# for bit; the stream-pool form and the oracle are checked beside it.
PERSISTENT_SHAPES = [(64, 90, 95, 0, 21), (32, 8, 47, 1, 22), (96, 30, 137, 0, 23), (64, 16, 93, 1, 24),
                     (128, 60, 185, 0, 25), (32, 180, 47, 0, 26), (64, 90, 95, 1, 27)]


def test_persistent_batched_equals_single_solves_and_pool():
    P = need_gpu()
    slices = make_slices(P, PERSISTENT_SHAPES, 7)
    P.ct_batched_options(P.CT_BATCH_AUTO)
    xs, reps = P.ct_pdtv_solve_batched(slices)
    got = [to_np(x).copy() for x in xs]
    try:
        P.ct_batched_options(P.CT_BATCH_POOL)
        xp, _ = P.ct_pdtv_solve_batched(slices)
        pool = [to_np(x).copy() for x in xp]
    finally:
        P.ct_batched_options(P.CT_BATCH_AUTO)
    for (g, b, w, prm), xg, xq, rep in zip(slices, got, pool, reps):
        x1, rep1 = P.ct_pdtv_solve(g, b, w, prm)
        assert np.array_equal(xg, to_np(x1))
        assert np.array_equal(xg, xq)
        assert rep["k"] == 7 and rep["sigma"] == rep1["sigma"]


def test_persistent_batched_matches_oracle():
    P = need_gpu()
    shapes = [(32, 46, 47, 0, 31), (64, 12, 93, 1, 32), (32, 36, 47, 0, 33), (64, 64, 93, 0, 34)]
    slices = make_slices(P, shapes, 9, explicit_steps=True)
    xs, _ = P.ct_pdtv_solve_batched(slices)
    for (g, b, w, prm), xb, (n, v, nb, mode, sd) in zip(slices, xs, shapes):
        bh = to_np(b)
        wh = None if w is None else to_np(w)
        kappa = float(np.mean(1.0 / wh)) if mode == 0 else 0.0
        taps = O.ramp_taps(mode, v, nb, prm.tau, kappa)
        st, _ = O.pdtv(bh, wh, taps, mode, 0.01, prm.tau, prm.sigma, 10, 9, n)
        assert rel_l2(to_np(xb), st.x) <= 1e-3


def test_persistent_batched_graph_replay_and_prox_forms():
    # one CUDA graph of the whole call (setups on the pool, then the
    # persistent launch), with FGP and D = I slices, replays to the eager result
    P = need_gpu()
    import torch
    slices = make_slices(P, PERSISTENT_SHAPES[:5], 6)
    slices[1][3].tv_accel = 1
    slices[2][3].precond = 0
    slices[3][3].tv_iters = 16
    bs = P.BatchedSolve(slices)
    xs, _ = bs.run()
    torch.cuda.synchronize()
    ref = [to_np(x).copy() for x in xs]
    for (g, b, w, prm), r in zip(slices, ref):
        assert np.array_equal(r, to_np(P.ct_pdtv_solve(g, b, w, prm)[0]))
    for x in bs.x:
        x.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bs.run()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for x, r in zip(bs.x, ref):
        assert np.array_equal(to_np(x), r)


def test_persistent_wait_limit_reports_timeout():
    # a zero wait limit: the first item that finds its slice's previous
    # phase unfinished gives up at once; the launch ends and the call
    # reports CT_ERR_TIMEOUT.  No GPU fault: every wait is bounded.
    P = need_gpu()
    slices = make_slices(P, PERSISTENT_SHAPES, 5)
    try:
        P.ct_batched_options(P.CT_BATCH_AUTO, 0.0)
        with pytest.raises(P.CTError) as e:
            P.ct_pdtv_solve_batched(slices)
        assert e.value.status == P.ctpd.CT_ERR_TIMEOUT
    finally:
        P.ct_batched_options(P.CT_BATCH_AUTO)
    # the device and the library are fine afterwards
    xs, reps = P.ct_pdtv_solve_batched(slices)
    for (g, b, w, prm), x in zip(slices, xs):
        assert np.array_equal(to_np(x), to_np(P.ct_pdtv_solve(g, b, w, prm)[0]))


def test_batched_options_reject_bad_values():
    P = need_gpu()
    for form, ws in [(2, -1.0), (0, float("nan")), (1, 1e6)]:
        with pytest.raises(P.CTError):
            P.ct_batched_options(form, ws)
