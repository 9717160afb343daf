"""FP64 CPU oracle for the ramp-preconditioned primal-dual TV reconstruction
(Kudo et al., arXiv 1609.06041).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
package never imports this module, and this module never imports the
product.  The arithmetic lives in ``ct_oracle.c`` (plain C, double
precision; OpenMP over views / image rows where gcc has it, with every
output element formed in the same order as on one thread); this file
compiles it with gcc on first use and wraps each routine for numpy arrays.

Parity status per routine (what pins it is in tests/test_oracle_*.py):
  project / backproject  -- pinned: hand sums at 0 and 90 degrees, constant
                            image, analytic disk/ellipse chords, 90-degree
                            rotation symmetry, adjoint identity, explicit matrix.
  ramp_taps / filter     -- pinned: DFT of a full period equals H (numpy FFT),
                            numpy.convolve, symmetry, Cholesky, FBP identity.
  grad / div / tv        -- pinned: adjoint identity, step-image TV.
  tv_prox                -- pinned: closed form on a two-level image,
                            duality-gap certificate, x >= 0 special case.
  cost / residual        -- pinned: the 1/2 of Eq. 1 by the quadratic at the
                            weighted least-squares minimiser (explicit A), the
                            TV term by a step image, W = I against residual.
  pdtv                   -- pinned: Step 1 equals the first form of Eq. 18 /
                            Eq. 29 at k = 0..5, first iterate = FBP + TV prox, beta = 0
                            limit = weighted least squares (numpy solve),
                            injective few-view limit = x_true, limit equal to
                            the independent Chambolle-Pock reference.
  power_norm             -- pinned: numpy 2-norm of the explicit matrix.
  cp_reference           -- pinned: beta = 0 limit = weighted least squares.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ct_oracle.c")
_LIB = os.path.join(_HERE, "libct_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ct_oracle.c into libct_oracle.so (gcc, -O2, portable flags,
    OpenMP when the compiler has it; results do not depend on it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_set_threads": [_i],
                "orc_get_threads": [],
                "orc_project": [_i, _i, _i, _p, _p, _p],
                "orc_backproject": [_i, _i, _i, _p, _p, _p],
                "orc_fft_len": [_i],
                "orc_ramp_taps": [_i, _i, _i, _d, _d, _i, _p],
                "orc_filter": [_i, _i, _p, _i, _p, _p],
                "orc_grad": [_i, _p, _p, _p],
                "orc_div": [_i, _p, _p, _p],
                "orc_tv": [_i, _p],
                "orc_tv_prox": [_i, _p, _d, _i, _p, _p, _p],
                "orc_tv_prox_fgp": [_i, _p, _d, _i, _p, _p, _p],
                "orc_cost": [_i, _i, _i, _p, _p, _p, _d, _p],
                "orc_residual": [_i, _i, _i, _p, _p, _p],
                "orc_apply_d": [_i, _i, _p, _p, _i, _p, _p, _p],
                "orc_pdtv": [_i, _i, _i, _p, _p, _p, _p, _p, _p, _i, _i, _d, _d, _d, _i, _i, _d,
                             _i, _i, _p, _p, _p, _p, _p, _p, _p],
                "orc_eps_prox": [_i, _i, _p, _i, _d, _p, _p],
                "orc_power_norm": [_i, _i, _i, _i, _p, _p, _p, _p, _i, _p, _i],
                "orc_cp_reference": [_i, _i, _i, _p, _p, _p, _i, _d, _d, _d, _d, _i, _p],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.orc_fft_len.restype = _i
            lib.orc_get_threads.restype = _i
            lib.orc_tv.restype = _d
            lib.orc_cost.restype = _d
            lib.orc_residual.restype = _d
            lib.orc_power_norm.restype = _d
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Threads of the projector, backprojector and filter (<= 0: every
    core).  Results are the same for any count."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _angles(angles):
    return None if angles is None else _f64(angles)


def project(x, n_views, n_bins, angles=None):
    """Joseph forward projection A x (Eq. 1's system matrix). x: (N, N)."""
    x = _f64(x)
    N = x.shape[-1]
    out = np.empty((n_views, n_bins))
    ang = _angles(angles)
    _load().orc_project(N, n_views, n_bins, _ptr(ang), _ptr(x), _ptr(out))
    return out


def backproject(sino, n, angles=None):
    """A^T y as the explicit scatter of each ray into the pixels A reads."""
    sino = _f64(sino)
    V, B = sino.shape
    out = np.empty((n, n))
    ang = _angles(angles)
    _load().orc_backproject(n, V, B, _ptr(ang), _ptr(sino), _ptr(out))
    return out


def fft_len(n_bins):
    return int(_load().orc_fft_len(n_bins))


def ramp_taps(mode, n_views, n_bins, tau, kappa=0.0, half=None, period=None):
    """Taps of D (Eq. 24 mode 0, Eq. 32 mode 1; modes 2 and 3 the low and
    high bands of the shift-variant split, which add up to mode 0); returns
    2*half-1 values, centre at index half-1.  Defaults: half = n_bins,
    period = fft_len."""
    half = n_bins if half is None else half
    P = fft_len(n_bins) if period is None else period
    out = np.empty(2 * half - 1)
    _load().orc_ramp_taps(int(mode), n_views, P, float(tau), float(kappa), half, _ptr(out))
    return out


def filt(sino, taps):
    """Per-view linear convolution with symmetric-centred taps."""
    sino = _f64(sino)
    taps = _f64(taps)
    V, B = sino.shape
    half = (taps.size + 1) // 2
    out = np.empty_like(sino)
    _load().orc_filter(V, B, _ptr(taps), half, _ptr(sino), _ptr(out))
    return out


def shift_variant_scale(w):
    """s_i = sqrt(kappa w_i), kappa = mean(1/w) (Eq. 24 text): the diagonal
    that scales the high band of the shift-variant preconditioner."""
    w = _f64(w)
    kappa = float(np.mean(1.0 / w))
    return np.sqrt(kappa * w)


def apply_d(sino, taps, taps_hi=None, s=None):
    """The iteration's preconditioner: filt(sino, taps), or with taps_hi the
    shift-variant D = T_lo + S T_hi S (taps = low band, S = diag(s))."""
    sino = _f64(sino)
    V, B = sino.shape
    taps = _f64(taps)
    half = (taps.size + 1) // 2
    out = np.empty_like(sino)
    th = None if taps_hi is None else _f64(taps_hi)
    sv = None if taps_hi is None else _f64(s)
    _load().orc_apply_d(V, B, _ptr(taps), _ptr(th), half, _ptr(sv), _ptr(sino), _ptr(out))
    return out


def grad(x):
    x = _f64(x)
    N = x.shape[-1]
    gx, gy = np.empty_like(x), np.empty_like(x)
    _load().orc_grad(N, _ptr(x), _ptr(gx), _ptr(gy))
    return gx, gy


def div(px, py):
    px, py = _f64(px), _f64(py)
    N = px.shape[-1]
    out = np.empty_like(px)
    _load().orc_div(N, _ptr(px), _ptr(py), _ptr(out))
    return out


def tv(x):
    x = _f64(x)
    return float(_load().orc_tv(x.shape[-1], _ptr(x)))


def tv_prox(z, lam, n_tv, px=None, py=None, fgp=False):
    """prox of lam*TV + i(x>=0) by n_tv projected-gradient dual steps (fgp:
    the fast gradient projection with momentum).  Returns (x, px, py); px,
    py are the warm-started dual fields."""
    z = _f64(z)
    N = z.shape[-1]
    px = np.zeros_like(z) if px is None else _f64(px).copy()
    py = np.zeros_like(z) if py is None else _f64(py).copy()
    x = np.empty_like(z)
    fn = _load().orc_tv_prox_fgp if fgp else _load().orc_tv_prox
    fn(N, _ptr(z), float(lam), int(n_tv), _ptr(px), _ptr(py), _ptr(x))
    return x, px, py


def cost(x, b, w, beta, angles=None):
    x, b = _f64(x), _f64(b)
    w = None if w is None else _f64(w)
    V, B = b.shape
    return float(_load().orc_cost(x.shape[-1], V, B, _ptr(_angles(angles)), _ptr(b),
                                  _ptr(w), float(beta), _ptr(x)))


def residual(x, b, angles=None):
    x, b = _f64(x), _f64(b)
    V, B = b.shape
    return float(_load().orc_residual(x.shape[-1], V, B, _ptr(_angles(angles)),
                                      _ptr(b), _ptr(x)))


class PDState:
    """Iterate of Algorithm 1/2: x^k, mu^k, mu^{k-1}, TV dual field, k."""

    def __init__(self, n, n_views, n_bins):
        self.x = np.zeros((n, n))
        self.mu = np.zeros((n_views, n_bins))
        self.mu_prev = np.zeros((n_views, n_bins))
        self.px = np.zeros((n, n))
        self.py = np.zeros((n, n))
        self.k = 0


def pdtv(b, w, taps, mode, beta, tau, sigma, n_tv, iters, n, angles=None,
         state=None, trace=False, taps_hi=None, s=None, fgp=False, eps=0.0, mubar=None):
    """Run `iters` iterations of Algorithm 1 (mode 0) / 2 (mode 1) from
    `state` (fresh zero state if None).  With taps_hi (and s) the
    preconditioner is the shift-variant D = T_lo + S T_hi S (apply_d); with
    fgp the prox runs the fast gradient projection; with eps > 0 (mode 1)
    the epsilon-constrained form, whose dual steps take eps_prox.  mubar (a
    V x B float64 array, optional) receives the mu_bar of the last
    iteration's Step 1.  Returns (state, trace or None)."""
    b = _f64(b)
    V, B = b.shape
    w = None if w is None else _f64(w)
    taps = _f64(taps)
    half = (taps.size + 1) // 2
    th = None if taps_hi is None else _f64(taps_hi)
    sv = None if taps_hi is None else _f64(s)
    st = PDState(n, V, B) if state is None else state
    tr = np.empty(iters) if trace else None
    _load().orc_pdtv(n, V, B, _ptr(_angles(angles)), _ptr(b), _ptr(w), _ptr(taps), _ptr(th), _ptr(sv), half,
                     int(mode), float(beta), float(tau), float(sigma), int(n_tv), int(bool(fgp)), float(eps),
                     int(st.k), int(iters), _ptr(st.x), _ptr(st.mu), _ptr(st.mu_prev),
                     _ptr(st.px), _ptr(st.py), _ptr(tr), _ptr(mubar))
    st.k += iters
    return st, tr


def power_norm(which, n, n_views, n_bins, taps=None, w=None, iters=50, angles=None, taps_hi=None, s=None):
    """which=0: ||A^T D A||; which=1: ||W^-1/2 D W^-1/2|| (D as in apply_d)."""
    taps = np.ones(1) if taps is None else _f64(taps)
    half = (taps.size + 1) // 2
    w = None if w is None else _f64(w)
    th = None if taps_hi is None else _f64(taps_hi)
    sv = None if taps_hi is None else _f64(s)
    return float(_load().orc_power_norm(int(which), n, n_views, n_bins, _ptr(_angles(angles)),
                                        _ptr(taps), _ptr(th), _ptr(sv), half, _ptr(w), int(iters)))


def cp_reference(b, w, mode, beta, s, t, iters, n, angles=None, eps=0.0):
    """Chambolle-Pock on K = [A; grad] (independent limit reference); mode 1
    with eps > 0: TV subject to ||Ax - b|| <= eps, x >= 0."""
    b = _f64(b)
    V, B = b.shape
    w = None if w is None else _f64(w)
    x = np.empty((n, n))
    _load().orc_cp_reference(n, V, B, _ptr(_angles(angles)), _ptr(b), _ptr(w), int(mode),
                             float(beta), float(eps), float(s), float(t), int(iters), _ptr(x))
    return x


def eps_prox(q, taps, se):
    """The epsilon-constrained form's dual step (Sec. 5 names the form
    without its steps; with the eps-ball's support function in h the dual
    step becomes a proximal map): argmin_nu
    se |nu| + 1/2 (nu - q)^T D^-1 (nu - q), D the per-view Toeplitz matrix of
    the taps, by bisection on c in (I + c D) nu = q, c = se / |nu|."""
    q = _f64(q)
    V, B = q.shape
    taps = _f64(taps)
    half = (taps.size + 1) // 2
    out = np.empty((V, B))
    _load().orc_eps_prox(V, B, _ptr(taps), half, float(se), _ptr(q), _ptr(out))
    return out


def fewview_ell(n, n_views, n_bins, angles=None):
    """l = (2/3) (N^2 / B) mean_v |a_v|, |a_v| = 1 / max(|cos t_v|, |sin t_v|):
    the mean over rays of diag(A A^T) for Joseph's weights (one pixel's
    weights in a view add up to 1, so a view's rays carry N^2 of weight in
    total, |a_v| per step, and the squared interpolation weights of a step
    average 2/3 of |a_v|^2).  It sets kappa = tau l of the few-view smoothed
    ramp (precond 3)."""
    t = np.arange(n_views) * np.pi / n_views if angles is None else _f64(angles)
    a = 1.0 / np.maximum(np.abs(np.cos(t)), np.abs(np.sin(t)))
    return (2.0 / 3.0) * (n * n / n_bins) * float(np.mean(a))


def default_tau(mode, n_views, kappa):
    """tau defaults: low-dose pi*kappa/(2m) puts the knee of H (Eq. 24) at the
    Nyquist frequency; few-view 0.01 (image-intensity units)."""
    return np.pi * kappa / (2.0 * n_views) if mode == 0 else 0.01


def step_sizes(mode, n, n_views, n_bins, taps, w, tau, rho=0.95, iters=50, angles=None, taps_hi=None, s=None):
    """sigma from the step rule of the Alg. 1 / Alg. 2 boxes with safety rho:
    low-dose sigma = rho*min(2/||W^-1/2 D W^-1/2||, 1/(tau ||A^T D A||)),
    few-view sigma = rho/(tau ||A^T D A||).  Returns (sigma, nADA, nWDW)."""
    nada = power_norm(0, n, n_views, n_bins, taps=taps, iters=iters, angles=angles, taps_hi=taps_hi, s=s)
    if mode == 0:
        nwdw = power_norm(1, n, n_views, n_bins, taps=taps, w=w, iters=iters, angles=angles,
                          taps_hi=taps_hi, s=s)
        sigma = rho * min(2.0 / nwdw, 1.0 / (tau * nada))
    else:
        nwdw = 0.0
        sigma = rho / (tau * nada)
    return sigma, nada, nwdw
