"""ct_pdtv_solve with page-locked host buffers: b, w and x_out in host
memory are copied through the workspace's staging area around the same
device solve, so the results equal the device-buffer solve bit for bit, on
the direct path, on the library's replayed solve graph and when resuming;
pageable host memory is refused."""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu


def lowdose(N, V, B, seed):
    x = synth.ellipse_phantom(N, 10, seed) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x, V, B), 1e4, seed + 100)
    return f32(b), f32(w)


def pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()


def test_host_buffers_equal_device_buffers_and_the_oracle():
    P = need_gpu()
    import torch
    N, V, B = 64, 90, 96
    b, w = lowdose(N, V, B, 0)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=15, tv_iters=10, beta=0.01, tau=tau, sigma=0.5)
    xd, rep_d = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    xh, rep_h = P.ct_pdtv_solve(g, pinned(b), pinned(w), prm)   # report: x ready at return
    assert not xh.is_cuda and xh.is_pinned()
    assert np.array_equal(xh.numpy(), to_np(xd))
    assert rep_h == rep_d
    st, _ = O.pdtv(b, w, O.ramp_taps(0, V, B, tau, kappa), 0, 0.01, tau, 0.5, 10, 15, N)
    assert rel_l2(xh.numpy(), st.x) <= 1e-3
    # mixed: device b and w, host x_out
    xm = torch.empty(N, N).pin_memory()
    P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm, x_out=xm)
    assert np.array_equal(xm.numpy(), to_np(xd))


def test_host_buffers_on_the_replayed_solve_graph_and_resume():
    # repeated calls with a workspace and no report replay the library's
    # graph, whose copies read the host buffers when it runs: new contents
    # of the same buffers are solved as usual
    P = need_gpu()
    import torch
    N, V, B = 48, 60, 72
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=0, iters=10, tv_iters=10, beta=0.01)
    ws = P.workspace_for(g, prm)
    bh, wh, xh = torch.empty(V, B).pin_memory(), torch.empty(V, B).pin_memory(), torch.empty(N, N).pin_memory()
    for seed in (1, 2, 3):
        b, w = lowdose(N, V, B, seed)
        bh.numpy()[:] = b
        wh.numpy()[:] = w
        P.ct_pdtv_solve(g, bh, wh, prm, x_out=xh, workspace=ws, report=False)
        torch.cuda.synchronize()
        xd, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
        assert np.array_equal(xh.numpy(), to_np(xd)), seed
    # resume: 4 + 6 iterations with a host x_out equal 10 in one call
    b, w = lowdose(N, V, B, 4)
    bh.numpy()[:] = b
    wh.numpy()[:] = w
    ws2 = P.workspace_for(g, prm)
    P.ct_pdtv_solve(g, bh, wh, P.PDTVParams(**{**prm.__dict__, "iters": 4}), x_out=xh, workspace=ws2)
    P.ct_pdtv_solve(g, bh, wh, P.PDTVParams(**{**prm.__dict__, "iters": 6, "resume": 1}), x_out=xh, workspace=ws2)
    xd, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    assert np.array_equal(xh.numpy(), to_np(xd))


def test_fewview_host_b_and_pageable_refused():
    P = need_gpu()
    import torch
    N, V, B = 64, 16, 92
    x = f32(synth.ellipse_phantom(N, 6, 2))
    b = f32(O.project(x, V, B))
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=1, iters=20, tv_iters=10, tau=0.01, sigma=0.5)
    xh, _ = P.ct_pdtv_solve(g, pinned(b), None, prm)
    xd, _ = P.ct_pdtv_solve(g, to_gpu(b), None, prm)
    assert np.array_equal(xh.numpy(), to_np(xd))
    # the binding refuses a pageable CPU tensor ...
    with pytest.raises(ValueError):
        P.ct_pdtv_solve(g, torch.from_numpy(b), None, prm)
    # ... and the library refuses pageable memory itself
    from paper_1609_06041_gb300 import ctpd as C
    bp = np.ascontiguousarray(b)
    xo = torch.empty(N, N, device="cuda")
    p = prm.to_c()
    st = C._lib.ct_pdtv_solve(g.handle, ctypes.c_void_p(bp.ctypes.data), None, ctypes.byref(p),
                              ctypes.c_void_p(xo.data_ptr()), None, None, C._stream())
    assert st == C.CT_ERR_ARG and "page-locked" in C.ct_last_error()
