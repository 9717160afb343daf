"""Pins of the oracle's Joseph projector A and backprojector A^T against
geometry: hand sums, a constant image, analytic chord lengths of a disk and
a tilted ellipse, the 90-degree rotation symmetry, the adjoint identity and
the explicit matrix.  (A is the system matrix of Eq. 1; A^T enters Eq. 19.)"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def test_zero_degree_view_is_column_sums():
    # theta = 0 steps along rows with u = d - (B-1)/2 + (N-1)/2: integer when
    # B - N is even, so each row contributes x[r][c] exactly.
    x = synth.random_image(6, 1)
    s = O.project(x, 4, 8)
    np.testing.assert_allclose(s[0, 1:7], x.sum(axis=0), rtol=0, atol=1e-13)
    assert s[0, 0] == 0.0 and s[0, 7] == 0.0


def test_zero_degree_half_pixel_lerp():
    # B - N odd: every sample sits half-way between two columns.
    x = synth.random_image(5, 2)
    s = O.project(x, 2, 6)
    cols = x.sum(axis=0)
    expect = np.concatenate([[0.5 * cols[0]], 0.5 * (cols[:-1] + cols[1:]), [0.5 * cols[-1]]])
    np.testing.assert_allclose(s[0], expect, rtol=0, atol=1e-13)


def test_ninety_degree_view_is_row_sums():
    x = synth.random_image(6, 3)
    s = O.project(x, 4, 8)          # view 2 = 90 degrees, column stepping
    np.testing.assert_allclose(s[2, 1:7], x.sum(axis=1), rtol=0, atol=1e-12)


def test_constant_image_gives_n_over_cos():
    # A ray that crosses every row inside the image collects N samples of 1,
    # each weighted by the path length 1/|cos| per row.
    N, V, B = 32, 16, 45
    s = O.project(np.ones((N, N)), V, B)
    for v in range(V):
        th = v * math.pi / V
        rows = (4 * v <= V) or (4 * v >= 3 * V)
        if not rows:
            continue
        c, sn = math.cos(th), math.sin(th)
        for d in range(B):
            sd = d - (B - 1) / 2
            # column coordinate of the ray at the first and last row centre
            us = [(sd - (r - (N - 1) / 2) * sn) / c + (N - 1) / 2 for r in (0, N - 1)]
            if min(us) >= 0 and max(us) <= N - 1:
                assert abs(s[v, d] - N / abs(c)) < 1e-12


@pytest.mark.parametrize("shape", ["disk", "ellipse"])
def test_analytic_chords(shape):
    # Joseph of the rasterised shape follows the analytic chord within about
    # one pixel (boundary pixels), for chords well inside the shape.
    N, V, B = 256, 12, 256
    if shape == "disk":
        e = synth.Ellipse(0.0, 0.0, 100.0, 100.0, 0.0, 1.0)
    else:
        e = synth.Ellipse(12.5, -7.25, 110.0, 60.0, 0.4, 1.0)
    p = O.project(synth.rasterise(N, [e]), V, B)
    s = np.arange(B) - (B - 1) / 2
    for v in range(V):
        th = v * math.pi / V
        rho2 = (e.a * math.cos(th - e.phi)) ** 2 + (e.b * math.sin(th - e.phi)) ** 2
        sp = s - (e.cx * math.cos(th) + e.cy * math.sin(th))
        inside = sp ** 2 < 0.81 * rho2
        chord = 2 * e.a * e.b * np.sqrt(np.maximum(rho2 - sp ** 2, 0)) / rho2
        assert np.abs(p[v, inside] - chord[inside]).max() < 1.5


def test_rotation_by_ninety_degrees_shifts_views():
    # x'(r, c) = x(N-1-c, r) is x rotated by +90 degrees; its view v + V/2
    # equals view v of x (rows <-> columns), away from the 45-degree tie.
    N, V, B = 16, 12, 23
    x = synth.random_image(N, 3)
    xr = np.array([[x[N - 1 - c, r] for c in range(N)] for r in range(N)])
    s1, s2 = O.project(x, V, B), O.project(xr, V, B)
    for v in range(V // 2):
        np.testing.assert_allclose(s2[v + V // 2], s1[v], rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,V,B", [(8, 7, 11), (9, 16, 13), (16, 5, 24)])
def test_adjoint_identity(N, V, B):
    x = synth.random_image(N, 11)
    y = synth.random_sinogram(V, B, 12)
    lhs = float(np.vdot(O.project(x, V, B), y))
    rhs = float(np.vdot(x, O.backproject(y, N)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_explicit_matrix_transpose():
    N, V, B = 8, 6, 11
    A = np.zeros((V * B, N * N))
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        A[:, j] = O.project(e.reshape(N, N), V, B).ravel()
    AT = np.zeros((N * N, V * B))
    for i in range(V * B):
        e = np.zeros(V * B)
        e[i] = 1.0
        AT[:, i] = O.backproject(e.reshape(V, B), N).ravel()
    np.testing.assert_allclose(AT, A.T, rtol=0, atol=1e-14)
    # each ray has at most 2 non-zeros per row/column step; each (pixel,
    # view) pair has at most 2 rays
    for v in range(V):
        blk = A[v * B:(v + 1) * B]
        assert ((blk != 0).sum(axis=0) <= 2).all()


def test_custom_angles_match_default():
    N, V, B = 10, 9, 15
    x = synth.random_image(N, 4)
    ang = np.arange(V) * math.pi / V
    s1 = O.project(x, V, B)
    s2 = O.project(x, V, B, angles=ang)
    np.testing.assert_allclose(s1, s2, rtol=0, atol=1e-12)
