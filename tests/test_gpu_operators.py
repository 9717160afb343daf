"""GPU parity of the operators against the FP64 oracle: A, A^T (exact
transpose), the taps and the filter D.  Tolerance: relative L2 <= 1e-4 per
pass, the bound set for one projector / backprojector / filter pass."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-4

SHAPES = [
    (64, 90, 95),      # low-dose 64^2 workload
    (37, 13, 53),      # ragged: odd N, odd V, tails of every tile
    (33, 7, 40),       # bins narrower than the diagonal
    (5, 3, 9),         # tiny
    (1, 1, 1),         # single pixel, single ray
    (130, 32, 190),    # several 128-bin tiles + tail
    # N a multiple of 32: the view-pair projector; V = 33 (odd), 12 (V/4 a
    # row pair, V/2 a single), 16; even N and V: the orbit backprojector,
    # with B % 4 = 0 (aligned window copies) and not
    (96, 33, 140),
    (32, 12, 47),
    (64, 16, 92),
]


@pytest.mark.parametrize("N,V,B", SHAPES)
def test_project_parity(N, V, B):
    P = need_gpu()
    g = P.Geometry(N, V, B)
    x = f32(synth.ellipse_phantom(N, 6, N) if N > 4 else synth.random_image(N, 1, positive=True))
    got = to_np(P.ct_project(g, to_gpu(x)))
    ref = O.project(x, V, B)
    assert rel_l2(got, ref) <= TOL


@pytest.mark.parametrize("N,V,B", SHAPES)
def test_backproject_parity(N, V, B):
    P = need_gpu()
    g = P.Geometry(N, V, B)
    y = f32(synth.random_sinogram(V, B, 5))
    got = to_np(P.ct_backproject(g, to_gpu(y)))
    ref = O.backproject(y, N)
    assert rel_l2(got, ref) <= TOL


def test_custom_angles_parity():
    P = need_gpu()
    N, V, B = 48, 17, 70
    ang = np.sort(np.random.default_rng(3).uniform(0, math.pi, V))
    g = P.Geometry(N, V, B, angles=ang)
    x = f32(synth.ellipse_phantom(N, 5, 2))
    assert rel_l2(to_np(P.ct_project(g, to_gpu(x))), O.project(x, V, B, angles=ang)) <= TOL
    y = f32(synth.random_sinogram(V, B, 2))
    assert rel_l2(to_np(P.ct_backproject(g, to_gpu(y))), O.backproject(y, N, angles=ang)) <= TOL


def test_batched_operators():
    P = need_gpu()
    N, V, B = 40, 24, 60
    g = P.Geometry(N, V, B)
    xs = np.stack([f32(synth.ellipse_phantom(N, 4, s)) for s in range(3)])
    sino = to_np(P.ct_project(g, to_gpu(xs)))
    for i in range(3):
        assert rel_l2(sino[i], O.project(xs[i], V, B)) <= TOL
    back = to_np(P.ct_backproject(g, to_gpu(sino)))
    for i in range(3):
        assert rel_l2(back[i], O.backproject(f32(sino[i]), N)) <= TOL
    # empty batch is a no-op
    import torch
    e = torch.empty(0, N, N, device="cuda")
    assert P.ct_project(g, e).shape == (0, V, B)


def test_transpose_to_coordinate_rounding():
    # The matrix of A (columns from unit images) and of A^T (columns from
    # unit sinograms) are transposes of each other up to the float rounding
    # of the Joseph coordinates (A evaluates weights from the ray side, A^T
    # from the pixel side); both agree with the oracle's FP64 matrix.
    P = need_gpu()
    import torch
    N, V, B = 8, 12, 13
    g = P.Geometry(N, V, B)
    E = torch.eye(N * N, device="cuda").reshape(N * N, N, N).contiguous()
    A = P.ct_project(g, E).reshape(N * N, V * B).T.cpu().numpy()          # (I, J)
    F = torch.eye(V * B, device="cuda").reshape(V * B, V, B).contiguous()
    AT = P.ct_backproject(g, F).reshape(V * B, N * N).T.cpu().numpy()     # (J, I)
    assert np.abs(A.T - AT).max() < 4e-6
    Ao = np.stack([O.project(np.eye(N * N)[j].reshape(N, N), V, B).ravel() for j in range(N * N)], axis=1)
    assert np.abs(A - Ao).max() < 4e-6
    assert np.abs(AT.T - Ao).max() < 4e-6


def test_adjoint_identity_gpu():
    P = need_gpu()
    N, V, B = 96, 60, 140
    g = P.Geometry(N, V, B)
    x = synth.random_image(N, 7)
    y = synth.random_sinogram(V, B, 8)
    ax = to_np(P.ct_project(g, to_gpu(x)))
    aty = to_np(P.ct_backproject(g, to_gpu(y)))
    lhs = float((ax * f32(y)).sum())
    rhs = float((f32(x) * aty).sum())
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt((ax ** 2).sum() * (f32(y) ** 2).sum())


@pytest.mark.parametrize("mode,B,V", [(0, 95, 90), (1, 736, 32), (0, 53, 13), (1, 1, 1)])
def test_taps_parity(mode, B, V):
    P = need_gpu()
    g = P.Geometry(16, V, B)
    tau, kappa = 0.02, 0.4
    got = to_np(P.ct_ramp_taps(g, mode, tau, kappa))
    ref = O.ramp_taps(mode, V, B, tau, kappa)
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("V,B,half", [(90, 95, 95), (13, 53, 53), (8, 300, 40), (5, 1100, 1100),
                                      (3, 4200, 4200), (1, 1, 1), (2, 2, 2)])
def test_filter_parity(V, B, half):
    P = need_gpu()
    g = P.Geometry(16, V, B)
    t = f32(O.ramp_taps(0, V, B, 0.05, 0.3, half=half))
    y = f32(synth.random_sinogram(V, B, 4))
    got = to_np(P.ct_ramp_filter(g, to_gpu(t), to_gpu(y)))
    assert rel_l2(got, O.filt(y, t)) <= TOL


def test_full_size_operators():
    # 512^2 image, 720 views, 736 bins: the low-dose workload at scale.
    P = need_gpu()
    N, V, B = 512, 720, 736
    g = P.Geometry(N, V, B)
    x = f32(synth.ellipse_phantom(N, 20, 2) * (2.0 / N))
    assert rel_l2(to_np(P.ct_project(g, to_gpu(x))), O.project(x, V, B)) <= TOL
    y = f32(synth.random_sinogram(V, B, 3))
    assert rel_l2(to_np(P.ct_backproject(g, to_gpu(y))), O.backproject(y, N)) <= TOL
    t = f32(O.ramp_taps(0, V, B, 1e-3, 0.5))
    assert rel_l2(to_np(P.ct_ramp_filter(g, to_gpu(t), to_gpu(y))), O.filt(y, t)) <= TOL


def test_bad_arguments_raise():
    P = need_gpu()
    import torch
    g = P.Geometry(16, 8, 20)
    with pytest.raises(ValueError):
        P.ct_project(g, torch.zeros(15, 16, device="cuda"))
    with pytest.raises(TypeError):
        P.ct_project(g, torch.zeros(16, 16, device="cuda", dtype=torch.float64))
    with pytest.raises(P.CTError):
        P.ct_ramp_taps(g, 0, -1.0, 0.1)


@pytest.mark.parametrize("N,V,B,angles,batch", [(64, 90, 95, None, 1), (96, 30, 140, None, 3),
                                                (64, 33, 93, "custom", 2), (37, 13, 53, "custom", 1),
                                                (512, 720, 736, None, 1)])
def test_project_bands_add_up_to_the_projection(N, V, B, angles, batch):
    # ct_project_bands: the band partial sums, which scaled by each view's
    # path length |a_v| and added over the bands give A img (ct_project)
    P = need_gpu()
    import torch
    ang = np.sort(np.random.default_rng(5).uniform(0.0, np.pi, V)) if angles == "custom" else None
    g = P.Geometry(N, V, B, angles=ang)
    xs = np.stack([f32(synth.ellipse_phantom(N, 6, 11 + i)) for i in range(batch)])
    xg = to_gpu(xs)
    parts = P.ct_project_bands(g, xg)
    nb = P.ct_project_bands_count(g)
    assert parts.shape == (batch, nb, V, B) and nb == (N + 31) // 32
    t = np.arange(V) * np.pi / V if ang is None else ang
    a = (1.0 / np.maximum(np.abs(np.cos(t)), np.abs(np.sin(t)))).astype(np.float32)
    sino = to_np(P.ct_project(g, xg))
    summed = to_np(parts).astype(np.float64).sum(axis=1) * a[None, :, None]
    assert rel_l2(summed, sino) <= 1e-6
    assert rel_l2(summed[0], O.project(xs[0], V, B, angles=ang)) <= TOL
    # an output 4 bytes off a 16-byte boundary is refused
    unaligned = torch.empty(batch * nb * V * B + 1, device="cuda")[1:].view(batch, nb, V, B)
    with pytest.raises(P.CTError):
        P.ct_project_bands(g, xg, out=unaligned)
