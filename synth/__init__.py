"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This module only draws numbers: random-ellipse phantoms rasterised at pixel
centres, Poisson transmission counts from given line integrals, and random
test vectors.  It holds none of the reconstruction arithmetic (no projector,
filter, TV or iteration); whoever needs line integrals computes them with
their own projector and passes them in.

Conventions (used throughout the project): an N x N image is stored row-major,
pixel (r, c) has centre (x, y) = (c - (N-1)/2, r - (N-1)/2) in pixel units.
The phantoms stand in for the spot phantom and chest slice of the paper's
simulation study (Sec. 4), which are not available: piecewise-constant
ellipses, parallel beam, transmission Poisson noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Ellipse",
    "random_ellipses",
    "rasterise",
    "ellipse_phantom",
    "poisson_data",
    "random_image",
    "random_sinogram",
    "CONFIGS",
    "bins_for",
]


@dataclass(frozen=True)
class Ellipse:
    cx: float      # centre x (pixel units, origin at the image centre)
    cy: float      # centre y
    a: float       # semi-axis along the tilted x' axis
    b: float       # semi-axis along the tilted y' axis
    phi: float     # tilt (radians)
    value: float   # intensity written inside the ellipse


def random_ellipses(n: int, count: int, seed: int) -> list[Ellipse]:
    """Draw `count` ellipses for an n x n image from numpy's default_rng(seed).

    Per ellipse, in this order: centre radius 0.6 R sqrt(U) and angle 2 pi U
    (R = n/2), two semi-axes U[0.05 R, 0.3 R], tilt U[0, pi), intensity
    U[0.1, 1].  Every ellipse lies within 0.9 R of the centre, so it stays
    inside the field of view of every parallel-beam view.
    """
    rng = np.random.default_rng(seed)
    R = n / 2.0
    out = []
    for _ in range(count):
        rad = 0.6 * R * math.sqrt(rng.uniform())
        ang = 2.0 * math.pi * rng.uniform()
        a = rng.uniform(0.05 * R, 0.3 * R)
        b = rng.uniform(0.05 * R, 0.3 * R)
        phi = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.1, 1.0)
        out.append(Ellipse(rad * math.cos(ang), rad * math.sin(ang), a, b, phi, val))
    return out


def rasterise(n: int, ellipses: list[Ellipse]) -> np.ndarray:
    """Point-sample the ellipses at pixel centres in painter's order (a later
    ellipse overwrites an earlier one); background 0.  Returns float64 (n, n)."""
    c0 = (n - 1) / 2.0
    ys, xs = np.meshgrid(np.arange(n) - c0, np.arange(n) - c0, indexing="ij")
    img = np.zeros((n, n), dtype=np.float64)
    for e in ellipses:
        cp, sp = math.cos(e.phi), math.sin(e.phi)
        dx, dy = xs - e.cx, ys - e.cy
        u = (dx * cp + dy * sp) / e.a
        v = (-dx * sp + dy * cp) / e.b
        img[u * u + v * v <= 1.0] = e.value
    return img


def ellipse_phantom(n: int, count: int, seed: int) -> np.ndarray:
    """Random-ellipse phantom (float64, values in {0} U [0.1, 1])."""
    return rasterise(n, random_ellipses(n, count, seed))


def poisson_data(line_integrals: np.ndarray, i0: float, seed: int):
    """Transmission Poisson data from expected line integrals p (any shape).

    n ~ Poisson(I0 exp(-p)), n <- max(n, 1), b = -ln(n / I0), w = n.
    w is the inverse noise variance of b to first order, the statistical
    weight W = diag(w) of the weighted least-squares cost (Eq. 1).
    Returns (b, w) as float64 arrays of p's shape.
    """
    rng = np.random.default_rng(seed)
    lam = i0 * np.exp(-np.asarray(line_integrals, dtype=np.float64))
    counts = np.maximum(rng.poisson(lam), 1).astype(np.float64)
    return -np.log(counts / i0), counts


def random_image(n: int, seed: int, positive: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 1.0, (n, n)) if positive else rng.standard_normal((n, n))
    return x.astype(np.float64)


def random_sinogram(n_views: int, n_bins: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_views, n_bins)).astype(np.float64)


def bins_for(n: int) -> int:
    """Detector bins that cover the image diagonal: ceil(1.44 n)."""
    return int(math.ceil(1.44 * n))


def mixed_slices(count: int, seed: int, sizes=(256, 384, 512), views=(32, 90, 360, 720)):
    """Slice shapes of a mixed batch: image side and view count drawn from
    the given sets by default_rng(seed), bins = ceil(1.44 N), low-dose when
    the sinogram has more samples than the image (V B > N^2), else few-view.
    Returns a list of (n, n_views, n_bins, mode, seed_i)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        v = int(rng.choice(views))
        b = bins_for(n)
        mode = 0 if v * b > n * n else 1
        out.append((n, v, b, mode, seed * 1000 + i))
    return out


# The workloads, by what they are.  'scale' is the attenuation scale that
# turns unit-range phantom intensities into line integrals of a few units
# (x_phys = scale * v); few-view data are noiseless b = A v.
CONFIGS = {
    "lowdose_64": dict(n=64, views=90, bins=95, ellipses=10, mode="lowdose",
                       i0=1e4, beta=0.01, iters=20, scale=2.0 / 64),
    "fewview_512": dict(n=512, views=32, bins=736, ellipses=20, mode="fewview",
                        i0=None, beta=0.0, iters=100, scale=1.0),
    "lowdose_512": dict(n=512, views=720, bins=736, ellipses=20, mode="lowdose",
                        i0=5e3, beta=0.005, iters=30, scale=2.0 / 512),
    "unrolled_256": dict(n=256, views=180, bins=368, ellipses=10, mode="lowdose",
                         i0=1e4, beta=0.01, iters=10, scale=2.0 / 256, batch=16),
}
