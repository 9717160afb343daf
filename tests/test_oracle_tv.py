"""Pins of the oracle's TV pieces (Eq. 2) and of the prox of Eq. 17:
div = -grad^T, TV of a step image, the closed form on a two-level image, the
duality-gap optimality certificate, and the bound-constrained special cases."""
import numpy as np
import pytest

import oracle as O
import synth


def test_div_is_minus_grad_adjoint():
    N = 7
    x = synth.random_image(N, 1)
    px, py = synth.random_image(N, 2), synth.random_image(N, 3)
    gx, gy = O.grad(x)
    lhs = float((gx * px).sum() + (gy * py).sum())
    rhs = -float((x * O.div(px, py)).sum())
    assert abs(lhs - rhs) < 1e-12


def test_grad_directions_and_boundary():
    x = np.arange(16.0).reshape(4, 4)          # x[r][c] = 4r + c
    gx, gy = O.grad(x)
    assert (gx[:, :3] == 1).all() and (gx[:, 3] == 0).all()
    assert (gy[:3, :] == 4).all() and (gy[3, :] == 0).all()


def test_tv_of_step_image():
    N = 9
    x = np.zeros((N, N))
    x[:, 5:] = 1.0
    assert O.tv(x) == pytest.approx(N)         # one unit jump per row
    x2 = np.zeros((N, N))
    x2[4:, 5:] = 2.0                           # corner: 4+5 edges, one diagonal pixel
    gx, gy = O.grad(x2)
    assert O.tv(x2) == pytest.approx(np.sqrt(gx ** 2 + gy ** 2).sum())
    assert O.tv(x2) == pytest.approx(2.0 * (4 + 5))


@pytest.mark.parametrize("a,b,lam", [(2.0, 1.2, 0.1), (1.0, 3.0, 0.25), (2.0, 1.9, 0.1)])
def test_prox_two_level_closed_form(a, b, lam):
    # 2x2 image with identical rows (a, b): each row is the 1-D problem
    # min 1/2((x0-a)^2+(x1-b)^2) + lam |x1-x0| whose solution moves both
    # values lam toward each other, or meets at the mean if |a-b| <= 2 lam.
    z = np.array([[a, b], [a, b]])
    x, _, _ = O.tv_prox(z, lam, 4000)
    if abs(a - b) > 2 * lam:
        s = np.sign(a - b)
        expect = [a - lam * s, b + lam * s]
    else:
        expect = [(a + b) / 2] * 2
    np.testing.assert_allclose(x, [expect, expect], atol=1e-9)


def test_prox_duality_gap_certificate():
    # For any |p_j| <= 1, x(p) = max(0, z + lam div p) has primal-dual gap
    # lam (TV(x) - <p, grad x>) >= 0; it is 0 only at the prox.
    rng = np.random.default_rng(0)
    z = rng.standard_normal((8, 8))
    lam = 0.3
    x, px, py = O.tv_prox(z, lam, 20000)
    assert np.sqrt(px ** 2 + py ** 2).max() <= 1 + 1e-12
    gx, gy = O.grad(x)
    gap = lam * (O.tv(x) - float((px * gx + py * gy).sum()))
    assert -1e-12 <= gap < 1e-9
    assert x.min() >= 0.0
    # the objective at x beats perturbations
    f = lambda y: lam * O.tv(y) + 0.5 * ((y - z) ** 2).sum()
    for s in range(5):
        d = 1e-3 * rng.standard_normal(z.shape)
        assert f(x) <= f(np.maximum(x + d, 0)) + 1e-12


def test_prox_special_cases():
    z = np.full((5, 5), -0.3)
    x, _, _ = O.tv_prox(z, 0.2, 10)
    assert (x == 0).all()
    z = np.full((5, 5), 0.7)
    x, _, _ = O.tv_prox(z, 0.2, 10)
    assert (x == 0.7).all()
    z = synth.random_image(6, 4)
    x, _, _ = O.tv_prox(z, 0.0, 10)            # lam = 0: projection onto x >= 0
    np.testing.assert_array_equal(x, np.maximum(z, 0))


# ---- the fast gradient projection (FGP) form of the same prox ----

@pytest.mark.parametrize("a,b,lam", [(2.0, 1.2, 0.1), (1.0, 3.0, 0.25), (2.0, 1.9, 0.1)])
def test_fgp_two_level_closed_form(a, b, lam):
    z = np.array([[a, b], [a, b]])
    x, _, _ = O.tv_prox(z, lam, 2000, fgp=True)
    if abs(a - b) > 2 * lam:
        s = np.sign(a - b)
        expect = [a - lam * s, b + lam * s]
    else:
        expect = [(a + b) / 2] * 2
    np.testing.assert_allclose(x, [expect, expect], atol=1e-9)


def test_fgp_duality_gap_certificate_and_same_prox():
    rng = np.random.default_rng(0)
    z = rng.standard_normal((8, 8))
    lam = 0.3
    x, px, py = O.tv_prox(z, lam, 4000, fgp=True)
    assert np.sqrt(px ** 2 + py ** 2).max() <= 1 + 1e-12
    gx, gy = O.grad(x)
    gap = lam * (O.tv(x) - float((px * gx + py * gy).sum()))
    assert -1e-12 <= gap < 1e-9
    xg, _, _ = O.tv_prox(z, lam, 20000)
    np.testing.assert_allclose(x, xg, atol=1e-7)


def test_fgp_first_step_is_a_gradient_projection_step():
    # t_1 = 1: the first extrapolation weight is 0, so one FGP step from any
    # warm start is one step of the plain projected gradient
    z = synth.random_image(9, 5)
    p0x, p0y = 0.3 * synth.random_image(9, 6), 0.3 * synth.random_image(9, 7)
    a = O.tv_prox(z, 0.2, 1, p0x, p0y, fgp=True)
    b = O.tv_prox(z, 0.2, 1, p0x, p0y)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_fgp_special_cases():
    z = np.full((5, 5), -0.3)
    assert (O.tv_prox(z, 0.2, 10, fgp=True)[0] == 0).all()
    z = np.full((5, 5), 0.7)
    assert (O.tv_prox(z, 0.2, 10, fgp=True)[0] == 0.7).all()
    z = synth.random_image(6, 4)
    np.testing.assert_array_equal(O.tv_prox(z, 0.0, 10, fgp=True)[0], np.maximum(z, 0))


def test_fgp_approaches_the_prox_faster():
    # the dual objective converges as O(1/k^2) with momentum against O(1/k)
    z = synth.ellipse_phantom(24, 5, 2) + 0.3 * synth.random_image(24, 8)
    lam = 0.4
    xs, _, _ = O.tv_prox(z, lam, 40000)
    for k in (10, 30):
        d_gp = np.linalg.norm(O.tv_prox(z, lam, k)[0] - xs)
        d_fgp = np.linalg.norm(O.tv_prox(z, lam, k, fgp=True)[0] - xs)
        assert d_fgp < 0.7 * d_gp
