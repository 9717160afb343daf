"""A seeded sweep of random geometries against the FP64 oracle.

The fixed-shape parity tests pick the shapes that reach each kernel path
(the view-pair projector for N a multiple of 32, the rotation-orbit
backprojector for N and V even with the default angles, the fallbacks for
custom angles, odd sizes and narrow detectors).  This sweep draws sizes,
angle sets and batch counts at random, weighted so that every path is hit
several times, and holds each draw to the same bars: relative L2 <= 1e-4
per A, A^T and D pass, and <= 1e-3 on the image after a short solve of
either algorithm (Alg. 1 low-dose, Alg. 2 few-view) run with the oracle's
tau and sigma."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL_PASS = 1e-4
TOL_SOLVE = 1e-3


def draw(seed):
    """One geometry: N, V, B, angles (None = the default v pi / V), batch."""
    r = np.random.default_rng(seed)
    kind = seed % 4
    if kind == 0:      # view-pair projector, orbit backprojector
        N = int(32 * r.integers(1, 6))
        V = int(2 * r.integers(1, 50))
    elif kind == 1:    # odd or unaligned sizes, default angles
        N = int(r.integers(1, 170))
        V = int(r.integers(1, 100))
    elif kind == 2:    # N a multiple of 32 with odd V (no orbit), or custom angles below
        N = int(32 * r.integers(1, 5))
        V = int(2 * r.integers(0, 45) + 1)
    else:              # custom angles: any order of magnitude of spacing, unsorted
        N = int(r.integers(2, 150))
        V = int(r.integers(1, 80))
    angles = None
    if kind == 3 or (kind == 2 and seed % 8 == 6):
        angles = r.uniform(0.0, np.pi, V)
    diag = int(np.ceil(N * np.sqrt(2.0)))
    B = int(max(1, r.integers(max(1, diag // 3), diag + 24)))   # narrower and wider than the diagonal
    batch = int(r.integers(1, 4))
    return N, V, B, angles, batch


SEEDS = list(range(48))


@pytest.mark.parametrize("seed", SEEDS)
def test_random_operators(seed):
    P = need_gpu()
    N, V, B, angles, batch = draw(seed)
    g = P.Geometry(N, V, B, angles=angles)
    xs = np.stack([f32(synth.ellipse_phantom(N, 5, 40 + seed + i) if N > 4 else
                       synth.random_image(N, seed + i, positive=True)) for i in range(batch)])
    sino = to_np(P.ct_project(g, to_gpu(xs)))
    assert sino.shape == (batch, V, B)
    for i in range(batch):
        assert rel_l2(sino[i], O.project(xs[i], V, B, angles=angles)) <= TOL_PASS, (N, V, B, i)
    ys = np.stack([f32(synth.random_sinogram(V, B, 70 + seed + i)) for i in range(batch)])
    back = to_np(P.ct_backproject(g, to_gpu(ys)))
    assert back.shape == (batch, N, N)
    for i in range(batch):
        assert rel_l2(back[i], O.backproject(ys[i], N, angles=angles)) <= TOL_PASS, (N, V, B, i)
    taps = f32(O.ramp_taps(seed % 2, V, B, 0.02, 0.3))
    fl = to_np(P.ct_ramp_filter(g, to_gpu(taps), to_gpu(ys)))
    for i in range(batch):
        assert rel_l2(fl[i], O.filt(ys[i], taps)) <= TOL_PASS, (N, V, B, i)


@pytest.mark.parametrize("seed", SEEDS[::3])
def test_random_solves(seed):
    P = need_gpu()
    N, V, B, angles, _ = draw(seed)
    if N < 4:
        N = 4
        B = max(B, 6)
    mode = seed % 2
    x = synth.ellipse_phantom(N, 5, 90 + seed) * (2.0 / N)
    if mode == 0:
        b, w = synth.poisson_data(O.project(x, V, B, angles=angles), 1e4, seed + 7)
        b, w = f32(b), f32(w)
        kappa = float(np.mean(1.0 / w))
        tau = O.default_tau(0, V, kappa)
        beta = 0.01
    else:
        b, w = f32(O.project(f32(x), V, B, angles=angles)), None
        kappa = 0.0
        tau = O.default_tau(1, V, 0.0)
        beta = 0.0
    taps = O.ramp_taps(mode, V, B, tau, kappa)
    sigma, _, _ = O.step_sizes(mode, N, V, B, taps, w, tau, iters=30, angles=angles)
    iters, ntv = 6, 10
    g = P.Geometry(N, V, B, angles=angles)
    prm = P.PDTVParams(mode=mode, iters=iters, tv_iters=ntv, precond=1, beta=beta, tau=tau, sigma=sigma)
    xg, rep = P.ct_pdtv_solve(g, to_gpu(b), None if w is None else to_gpu(w), prm,
                              workspace=P.workspace_for(g, prm))
    st, _ = O.pdtv(b, w, taps, mode, beta, tau, sigma, ntv, iters, N, angles=angles)
    assert rep["k"] == iters
    assert rel_l2(to_np(xg), st.x) <= TOL_SOLVE, (N, V, B, mode)
