"""Launch-shape tuning (ct_geometry_autotune / set / get): every shape must
give the same operators and the same solve as the oracle, within the
per-pass and per-solve tolerances; out-of-range shapes are rejected."""
import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.mark.parametrize("N,V,B", [(64, 90, 95), (96, 12, 140), (64, 33, 93)])
@pytest.mark.parametrize("items,rows,slices", [(4, 2, 1), (7, 4, 2), (13, 2, 8), (16, 2, 4), (12, 4, 4)])
@pytest.mark.parametrize("form", [1, 2])
def test_operator_shapes_parity(N, V, B, items, rows, slices, form):
    P = need_gpu()
    g = P.Geometry(N, V, B)
    if V % 2:
        slices = 0   # odd V: no orbit backprojector
    g.set_tuning(items_per_block=items, orbit_slices=slices, proj_rows=rows, proj_form=form)
    assert g.tuning == {"items_per_block": items, "proj_rows": rows, "orbit_slices": slices, "tv_rows": 0,
                        "proj_form": form}
    x = f32(synth.ellipse_phantom(N, 6, 3))
    assert rel_l2(to_np(P.ct_project(g, to_gpu(x))), O.project(x, V, B)) <= TOL
    y = f32(synth.random_sinogram(V, B, 4))
    assert rel_l2(to_np(P.ct_backproject(g, to_gpu(y))), O.backproject(y, N)) <= TOL


@pytest.mark.parametrize("N,V,B,batch", [(64, 90, 95, 1), (96, 12, 140, 3), (64, 33, 93, 2), (128, 360, 185, 2),
                                         (512, 720, 736, 1), (256, 180, 368, 5), (64, 1, 96, 2), (32, 3, 47, 1)])
def test_projector_forms_agree_bit_for_bit(N, V, B, batch):
    # the work-balanced projector forms every band sum exactly as the
    # band-pair-per-block form does, whatever the items per block, the steps
    # per pass of a ray walk (a pass of four steps is two passes of two with
    # their loads issued together) or the batch: the projections are equal
    # bit for bit
    P = need_gpu()
    import torch
    g = P.Geometry(N, V, B)
    xs = np.stack([f32(synth.ellipse_phantom(N, 6, 3 + i)) for i in range(batch)])
    xg = to_gpu(xs)
    outs = []
    for rows, shapes in [(2, [(8, 1), (16, 2), (8, 2), (13, 1), (12, 2)]), (4, [(10, 1), (12, 2), (8, 2)])]:
        for items, form in shapes:
            g.set_tuning(items_per_block=items, proj_rows=rows, proj_form=form)
            outs.append(P.ct_project(g, xg).clone())
            # each slice of the batch equals its own single projection
            for i in range(batch):
                assert torch.equal(P.ct_project(g, xg[i].contiguous()), outs[-1][i])
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert rel_l2(to_np(outs[0][0]), O.project(xs[0], V, B)) <= TOL


def test_projector_and_prox_shapes_leave_the_solve_unchanged():
    # every projector shape (form, items per block, steps per pass) and every
    # prox tile height gives the same solve bit for bit: the tiles and unit
    # ranges only decide which thread forms which sum, not how
    P = need_gpu()
    import torch
    N, V, B = 96, 60, 137
    x_true = synth.ellipse_phantom(N, 8, 4) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x_true, V, B), 1e4, 104)
    g = P.Geometry(N, V, B)
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=8, tv_iters=10, beta=0.01, sigma=0.5)
    ref = None
    for items, rows, form, tv in [(0, 0, 0, 0), (6, 2, 1, 4), (12, 4, 1, 64), (8, 2, 2, 8), (12, 4, 2, 16)]:
        g.set_tuning(items_per_block=items, proj_rows=rows, proj_form=form, tv_rows=tv)
        xg, _ = P.ct_pdtv_solve(g, to_gpu(f32(b)), to_gpu(f32(w)), prm)
        if ref is None:
            ref = xg.clone()
        else:
            assert torch.equal(xg, ref), (items, rows, form, tv)


@pytest.mark.parametrize("rows", [4, 16, 64])
def test_tv_rows_solve_parity(rows):
    # the low-dose 64^2 / 90 / 95 solve (20 iterations, n_tv = 10) under
    # three TV tile shapes, against the oracle run with the same tau, sigma, taps
    P = need_gpu()
    N, V, B = 64, 90, 95
    x_true = synth.ellipse_phantom(N, 10, 0) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x_true, V, B), 1e4, 100)
    b, w = f32(b), f32(w)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    g = P.Geometry(N, V, B)
    g.set_tuning(tv_rows=rows)
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=20, tv_iters=10, precond=1, beta=0.01, tau=tau, sigma=0.5)
    xg, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    st, _ = O.pdtv(b, w, taps, 0, 0.01, tau, 0.5, 10, 20, N)
    assert rel_l2(to_np(xg), st.x) <= 1e-3


def test_autotune_picks_valid_shapes_and_keeps_parity():
    P = need_gpu()
    N, V, B = 128, 60, 185
    g = P.Geometry(N, V, B)
    t = g.autotune(batch=2)
    assert 4 <= t["items_per_block"] <= (12 if t["proj_rows"] == 4 else 16)
    assert t["proj_rows"] in (2, 4)
    assert 1 <= t["orbit_slices"] <= 8
    assert t["tv_rows"] in (4, 8, 16, 32, 64)
    assert t["proj_form"] in (1, 2)
    x = f32(synth.ellipse_phantom(N, 8, 5))
    assert rel_l2(to_np(P.ct_project(g, to_gpu(x))), O.project(x, V, B)) <= TOL
    y = f32(synth.random_sinogram(V, B, 6))
    assert rel_l2(to_np(P.ct_backproject(g, to_gpu(y))), O.backproject(y, N)) <= TOL


def test_autotune_without_shared_paths():
    # custom angles and odd N: neither the view-pair projector nor the orbit
    # backprojector applies; only the TV shape is tuned
    P = need_gpu()
    g = P.Geometry(37, 13, 53, angles=np.linspace(0.0, 3.0, 13))
    t = g.autotune()
    assert t["items_per_block"] == 0 and t["proj_rows"] == 0 and t["orbit_slices"] == 0 and t["proj_form"] == 0
    assert t["tv_rows"] in (4, 8, 16, 32, 64)


@pytest.mark.parametrize("bad", [dict(items_per_block=3), dict(items_per_block=17), dict(orbit_slices=9),
                                 dict(orbit_slices=-1), dict(tv_rows=2), dict(tv_rows=65), dict(proj_rows=3),
                                 dict(items_per_block=13, proj_rows=4), dict(proj_form=3), dict(proj_form=-1)])
def test_set_tuning_rejects_out_of_range(bad):
    P = need_gpu()
    g = P.Geometry(64, 90, 95)
    with pytest.raises(P.CTError):
        g.set_tuning(**bad)
    assert g.tuning == {"items_per_block": 0, "proj_rows": 0, "orbit_slices": 0, "tv_rows": 0, "proj_form": 0}


def test_orbit_slices_limit_large_view_count():
    # 8192 views: a slice holds at most 1024 base views, so 1 and 2 slices are refused
    P = need_gpu()
    g = P.Geometry(32, 8192, 46)
    with pytest.raises(P.CTError):
        g.set_tuning(orbit_slices=2)
    g.set_tuning(orbit_slices=4)
    assert g.tuning["orbit_slices"] == 4


def test_single_orbit_slice_writes_the_result():
    # with one base-view slice the orbit backprojector writes A^T y (and, in
    # the solve, z = x - tau A^T mubar) itself, with no reduction pass:
    # batched A^T and the low-dose solve against the oracle
    P = need_gpu()
    import torch
    N, V, B = 64, 90, 95
    g = P.Geometry(N, V, B)
    g.set_tuning(orbit_slices=1)
    ys = np.stack([f32(synth.random_sinogram(V, B, 20 + s)) for s in range(3)])
    out = to_np(P.ct_backproject(g, to_gpu(ys)))
    for s in range(3):
        assert rel_l2(out[s], O.backproject(ys[s], N)) <= TOL
    x_true = synth.ellipse_phantom(N, 10, 1) * (2.0 / N)
    b, w = synth.poisson_data(O.project(x_true, V, B), 1e4, 101)
    b, w = f32(b), f32(w)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, V, kappa)
    taps = O.ramp_taps(0, V, B, tau, kappa)
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=20, tv_iters=10, precond=1, beta=0.01, tau=tau, sigma=0.5)
    n0 = P.ct_kernel_launches()
    x, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    torch.cuda.synchronize()
    st, _ = O.pdtv(b, w, taps, 0, 0.01, tau, 0.5, 10, 20, N)
    assert rel_l2(to_np(x), st.x) <= 1e-3
    g.set_tuning(orbit_slices=2)
    n1 = P.ct_kernel_launches()
    x2, _ = P.ct_pdtv_solve(g, to_gpu(b), to_gpu(w), prm)
    torch.cuda.synchronize()
    # two slices: their sums are added in a cluster of the slices' blocks,
    # so no reduction pass runs either
    assert P.ct_kernel_launches() - n1 == n1 - n0
    assert rel_l2(to_np(x2), st.x) <= 1e-3


def test_measured_balance_ranges_give_the_same_projection():
    # at 512^2 / 720 views the tuner picks the work-balanced projector and
    # balances its unit ranges from measured block times; every unit must
    # still be formed exactly once, so the projection with the tuned table
    # equals, bit for bit, the one with equal unit counts (another shape,
    # for which the table does not apply) and matches the oracle
    P = need_gpu()
    import torch
    N, V, B = 512, 720, 736
    g = P.Geometry(N, V, B)
    t = g.autotune()
    if t["proj_form"] != 2:
        pytest.skip("the tuner picked the band-pair form on this device")
    x = f32(synth.ellipse_phantom(N, 20, 7) * (2.0 / N))
    xg = to_gpu(x)
    tuned = P.ct_project_bands(g, xg).clone()
    g.set_tuning(items_per_block=8, proj_rows=2, proj_form=2, orbit_slices=t["orbit_slices"], tv_rows=t["tv_rows"])
    equal = P.ct_project_bands(g, xg)
    assert torch.equal(tuned, equal)
    g.set_tuning(items_per_block=t["items_per_block"], proj_rows=t["proj_rows"], proj_form=2,
                 orbit_slices=t["orbit_slices"], tv_rows=t["tv_rows"])
    again = P.ct_project(g, xg)
    assert rel_l2(to_np(again), O.project(x, V, B)) <= TOL
