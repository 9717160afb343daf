"""Thin Python binding of libctpd.so (include/ctpd.h), one function per C
entry point with the same name.  Arguments are torch CUDA tensors (and, for
ct_pdtv_solve's b, w and x_out, page-locked CPU tensors, which the library
copies through the solve's workspace); this module only checks shapes and
passes raw pointers and the current CUDA stream.  All arithmetic runs in the library's CUDA kernels; there is no
CPU or PyTorch fallback: a missing library raises at import time.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctpd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA extension first "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double

CT_OK, CT_ERR_ARG, CT_ERR_CUDA, CT_ERR_OOM, CT_ERR_TIMEOUT, CT_ERR_NONFINITE = range(6)
CT_LOWDOSE, CT_FEWVIEW = 0, 1
CT_TAPS_LOW_BAND, CT_TAPS_HIGH_BAND = 2, 3   # ct_ramp_taps: bands of the shift-variant D
CT_BATCH_AUTO, CT_BATCH_POOL = 0, 1           # ct_batched_options: persistent launch when possible / stream pool


class ct_pdtv_params(ctypes.Structure):
    _fields_ = [("mode", _i), ("iters", _i), ("tv_iters", _i), ("precond", _i),
                ("norm_iters", _i), ("resume", _i), ("beta", _d), ("tau", _d),
                ("sigma", _d), ("rho", _d), ("tv_accel", _i), ("eps", _d)]


class ct_pdtv_report(ctypes.Structure):
    _fields_ = [("tau", _d), ("sigma", _d), ("kappa", _d), ("lambda_", _d),
                ("norm_ADA", _d), ("norm_WDW", _d), ("k", _i), ("trace", ctypes.POINTER(_d))]

    def as_dict(self):
        return {"tau": self.tau, "sigma": self.sigma, "kappa": self.kappa,
                "lambda": self.lambda_, "norm_ADA": self.norm_ADA,
                "norm_WDW": self.norm_WDW, "k": self.k}


EXPORTS = {
    "ct_version": ([], ctypes.c_char_p),
    "ct_last_error": ([], ctypes.c_char_p),
    "ct_kernel_launches": ([], ctypes.c_ulonglong),
    "ct_probe_fp32_fma": ([_i, ctypes.POINTER(_d), _vp], _i),
    "ct_batched_options": ([_i, _d], _i),
    "ct_geometry_create": ([_i, _i, _i, _vp, ctypes.POINTER(_vp)], _i),
    "ct_geometry_destroy": ([_vp], None),
    "ct_geometry_autotune": ([_vp, _i, _vp], _i),
    "ct_geometry_set_tuning": ([_vp, _i, _i, _i, _i, _i], _i),
    "ct_geometry_get_tuning": ([_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "ct_project": ([_vp, _vp, _vp, _i, _vp], _i),
    "ct_project_bands_count": ([_vp], _i),
    "ct_project_bands": ([_vp, _vp, _vp, _i, _vp], _i),
    "ct_backproject": ([_vp, _vp, _vp, _i, _vp], _i),
    "ct_ramp_taps": ([_vp, _i, _d, _d, _vp, _vp], _i),
    "ct_ramp_filter": ([_vp, _vp, _i, _vp, _vp, _i, _vp], _i),
    "ct_ramp_filter_split": ([_vp, _vp, _vp, _i, _vp, _vp, _vp, _i, _vp], _i),
    "ct_ramp_filter_noalloc": ([_vp, _vp, _i, _vp, _vp, _i, _vp], _i),
    "ct_sym_toeplitz_eig": ([_vp, _i, _vp, _vp], _i),
    "ct_pdtv_workspace_bytes": ([_vp, ctypes.POINTER(ct_pdtv_params)], ctypes.c_size_t),
    "ct_pdtv_solve": ([_vp, _vp, _vp, ctypes.POINTER(ct_pdtv_params), _vp, _vp,
                       ctypes.POINTER(ct_pdtv_report), _vp], _i),
    "ct_pdtv_status": ([_vp, _vp], _i),
    "ct_unrolled_workspace_bytes": ([_vp, _i, _i, _i, _i], ctypes.c_size_t),
    "ct_unrolled_forward": ([_vp, _vp, _vp, _i, _vp, _i, _d, _d, _d, _i, _i, _i, _vp, _vp, _vp], _i),
    "ct_unrolled_backward": ([_vp, _vp, _vp, _i, _vp, _i, _d, _d, _d, _i, _i, _i, _vp, _vp, _vp, _vp], _i),
    "ct_pdtv_solve_batched": ([_i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               ctypes.POINTER(ct_pdtv_params), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               ctypes.POINTER(ct_pdtv_report), _vp], _i),
}
for _name, (_args, _res) in EXPORTS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


class CTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _check(status):
    if status != CT_OK:
        raise CTError(status, _lib.ct_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, name, shape_tail=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected (..., {shape_tail})")
    return ctypes.c_void_p(t.data_ptr())


def _buf(t, name, shape_tail=None):
    """A CUDA tensor, or a page-locked CPU tensor (the solve copies it through its workspace)."""
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not t.is_pinned():
            raise ValueError(f"{name}: a CPU tensor must be page-locked (pin_memory())")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous float32")
        if shape_tail is not None and tuple(t.shape[-len(shape_tail):]) != tuple(shape_tail):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected (..., {shape_tail})")
        return ctypes.c_void_p(t.data_ptr())
    return _dev(t, name, shape_tail)


def _batch(t, ndim_tail):
    b = 1
    for s in t.shape[:-ndim_tail]:
        b *= s
    return b


def ct_version() -> str:
    return _lib.ct_version().decode()


def ct_last_error() -> str:
    return _lib.ct_last_error().decode()


def ct_kernel_launches() -> int:
    return int(_lib.ct_kernel_launches())


def ct_batched_options(form: int = CT_BATCH_AUTO, wait_seconds: float = -1.0) -> None:
    """How ct_pdtv_solve_batched schedules the slices (this process):
    CT_BATCH_AUTO (persistent launch when every slice qualifies) or
    CT_BATCH_POOL; wait_seconds < 0 restores the 5 s wait limit."""
    _check(_lib.ct_batched_options(int(form), float(wait_seconds)))


def ct_probe_fp32_fma(packed: bool = False) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    v = _d(0.0)
    _check(_lib.ct_probe_fp32_fma(int(bool(packed)), ctypes.byref(v), _stream()))
    return float(v.value)


class Geometry:
    """2-D parallel-beam geometry handle (ct_geometry_create / _destroy)."""

    def __init__(self, n: int, n_views: int, n_bins: int, angles=None):
        self.n, self.n_views, self.n_bins = int(n), int(n_views), int(n_bins)
        self._h = ctypes.c_void_p()
        arr = None
        if angles is not None:
            import numpy as np
            a = np.ascontiguousarray(angles, dtype=np.float64)
            if a.shape != (self.n_views,):
                raise ValueError("angles must have n_views entries")
            arr = a
        self._angles = arr
        ptr = None if arr is None else arr.ctypes.data_as(ctypes.c_void_p)
        _check(_lib.ct_geometry_create(self.n, self.n_views, self.n_bins, ptr, ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.ct_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def autotune(self, batch: int = 1) -> dict:
        """ct_geometry_autotune on the current stream; returns the chosen shapes.  With the
        work-balanced projector form it also balances that form's unit ranges for one image from
        measured block times (a table the geometry keeps; results are unchanged)."""
        _check(_lib.ct_geometry_autotune(self.handle, int(batch), _stream()))
        return self.tuning

    @property
    def tuning(self) -> dict:
        """Launch shapes held by the geometry (0: built-in rule)."""
        a, r, b, c, f = _i(), _i(), _i(), _i(), _i()
        _check(_lib.ct_geometry_get_tuning(self.handle, ctypes.byref(a), ctypes.byref(r), ctypes.byref(b),
                                           ctypes.byref(c), ctypes.byref(f)))
        return {"items_per_block": a.value, "proj_rows": r.value, "orbit_slices": b.value, "tv_rows": c.value,
                "proj_form": f.value}

    def set_tuning(self, items_per_block: int = 0, orbit_slices: int = 0, tv_rows: int = 0,
                   proj_rows: int = 0, proj_form: int = 0) -> None:
        _check(_lib.ct_geometry_set_tuning(self.handle, int(items_per_block), int(proj_rows), int(orbit_slices),
                                           int(tv_rows), int(proj_form)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_geometry_create(n, n_views, n_bins, angles=None) -> Geometry:
    return Geometry(n, n_views, n_bins, angles)


def ct_geometry_destroy(g: Geometry) -> None:
    g.close()


def ct_geometry_autotune(g: Geometry, batch: int = 1) -> dict:
    return g.autotune(batch)


def ct_geometry_set_tuning(g: Geometry, items_per_block: int = 0, orbit_slices: int = 0, tv_rows: int = 0,
                           proj_rows: int = 0, proj_form: int = 0) -> None:
    g.set_tuning(items_per_block, orbit_slices, tv_rows, proj_rows, proj_form)


def ct_geometry_get_tuning(g: Geometry) -> dict:
    return g.tuning


def ct_project(g: Geometry, img: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """sino = A img (batched over leading dims)."""
    pi = _dev(img, "img", (g.n, g.n))
    if out is None:
        out = torch.empty(*img.shape[:-2], g.n_views, g.n_bins, device=img.device, dtype=torch.float32)
    po = _dev(out, "out", (g.n_views, g.n_bins))
    _check(_lib.ct_project(g.handle, pi, po, _batch(img, 2), _stream()))
    return out


def ct_project_bands_count(g: Geometry) -> int:
    return int(_lib.ct_project_bands_count(g.handle))


def ct_project_bands(g: Geometry, img: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Band partial sums of A img: (..., n_bands, V, B), sino = |a_v| sum over the band axis."""
    pi = _dev(img, "img", (g.n, g.n))
    nb = ct_project_bands_count(g)
    if out is None:
        out = torch.empty(*img.shape[:-2], nb, g.n_views, g.n_bins, device=img.device, dtype=torch.float32)
    po = _dev(out, "out", (nb, g.n_views, g.n_bins))
    _check(_lib.ct_project_bands(g.handle, pi, po, _batch(img, 2), _stream()))
    return out


def ct_backproject(g: Geometry, sino: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """img = A^T sino (batched over leading dims)."""
    ps = _dev(sino, "sino", (g.n_views, g.n_bins))
    if out is None:
        out = torch.empty(*sino.shape[:-2], g.n, g.n, device=sino.device, dtype=torch.float32)
    po = _dev(out, "out", (g.n, g.n))
    _check(_lib.ct_backproject(g.handle, ps, po, _batch(sino, 2), _stream()))
    return out


def ct_ramp_taps(g: Geometry, mode: int, tau: float, kappa: float = 0.0, out=None) -> torch.Tensor:
    """Taps of D (Eq. 24 / Eq. 32; modes CT_TAPS_LOW_BAND / CT_TAPS_HIGH_BAND the
    bands of the shift-variant D), 2B-1 values centred at B-1."""
    if out is None:
        out = torch.empty(2 * g.n_bins - 1, device="cuda", dtype=torch.float32)
    _check(_lib.ct_ramp_taps(g.handle, int(mode), float(tau), float(kappa), _dev(out, "taps"), _stream()))
    return out


def ct_ramp_filter(g: Geometry, taps: torch.Tensor, sino: torch.Tensor, out=None) -> torch.Tensor:
    """Per-view linear convolution with centred taps (the D of Eqs. 18-20)."""
    if taps.numel() % 2 != 1:
        raise ValueError("taps must have an odd length 2*half-1")
    half = (taps.numel() + 1) // 2
    pt = _dev(taps, "taps")
    ps = _dev(sino, "sino", (g.n_views, g.n_bins))
    if out is None:
        out = torch.empty_like(sino)
    po = _dev(out, "out", (g.n_views, g.n_bins))
    _check(_lib.ct_ramp_filter(g.handle, pt, half, ps, po, _batch(sino, 2), _stream()))
    return out


def ct_ramp_filter_split(g: Geometry, taps_lo: torch.Tensor, taps_hi: torch.Tensor, s: torch.Tensor,
                         sino: torch.Tensor, out=None) -> torch.Tensor:
    """The shift-variant preconditioner: out = T_lo sino + s * T_hi (s * sino)."""
    if taps_lo.numel() % 2 != 1 or taps_hi.numel() != taps_lo.numel():
        raise ValueError("taps_lo, taps_hi must have the same odd length 2*half-1")
    half = (taps_lo.numel() + 1) // 2
    pl, ph = _dev(taps_lo, "taps_lo"), _dev(taps_hi, "taps_hi")
    pv = _dev(s, "s", (g.n_views, g.n_bins))
    ps = _dev(sino, "sino", (g.n_views, g.n_bins))
    if out is None:
        out = torch.empty_like(sino)
    po = _dev(out, "out", (g.n_views, g.n_bins))
    _check(_lib.ct_ramp_filter_split(g.handle, pl, ph, half, pv, ps, po, _batch(sino, 2), _stream()))
    return out


def ct_ramp_filter_noalloc(g: Geometry, taps: torch.Tensor, sino: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
    """ct_ramp_filter without device allocation: the caller passes `out`,
    the library uses a fixed device array for its scratch (n_bins <= 4096)."""
    if taps.numel() % 2 != 1:
        raise ValueError("taps must have an odd length 2*half-1")
    half = (taps.numel() + 1) // 2
    pt = _dev(taps, "taps")
    ps = _dev(sino, "sino", (g.n_views, g.n_bins))
    po = _dev(out, "out", (g.n_views, g.n_bins))
    _check(_lib.ct_ramp_filter_noalloc(g.handle, pt, half, ps, po, _batch(sino, 2), _stream()))
    return out


def ct_sym_toeplitz_eig(t):
    """Eigendecomposition of the symmetric Toeplitz matrix T[i][j] = t[|i-j|]
    (host, FP64): returns (q, lambda), q's columns the unit eigenvectors."""
    import numpy as np
    t = np.ascontiguousarray(t, dtype=np.float64)
    n = t.size
    q = np.empty((n, n))
    lam = np.empty(n)
    _check(_lib.ct_sym_toeplitz_eig(t.ctypes.data_as(_vp), n, q.ctypes.data_as(_vp), lam.ctypes.data_as(_vp)))
    return q, lam


@dataclass
class PDTVParams:
    mode: int = CT_LOWDOSE
    iters: int = 20
    tv_iters: int = 10
    precond: int = 1
    norm_iters: int = 0          # 0: the library default (12 Lanczos steps)
    resume: int = 0
    beta: float = 0.0
    tau: float = 0.0
    sigma: float = 0.0
    rho: float = 0.95
    tv_accel: int = 0
    eps: float = 0.0             # CT_FEWVIEW: > 0 solves min TV s.t. ||Ax - b|| <= eps

    def to_c(self):
        return ct_pdtv_params(int(self.mode), int(self.iters), int(self.tv_iters), int(self.precond),
                              int(self.norm_iters), int(self.resume), float(self.beta),
                              float(self.tau), float(self.sigma), float(self.rho), int(self.tv_accel),
                              float(self.eps))


def ct_pdtv_workspace_bytes(g: Geometry, params: PDTVParams) -> int:
    p = params.to_c()
    return int(_lib.ct_pdtv_workspace_bytes(g.handle, ctypes.byref(p)))


def ct_pdtv_solve(g: Geometry, b: torch.Tensor, w: torch.Tensor | None, params: PDTVParams,
                  x_out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                  report: bool = True, trace: bool = False):
    """Algorithm 1 / 1' / 2.  Returns (x, report dict or None).
    b, w, x_out: CUDA tensors or page-locked CPU tensors (a CPU x is ready
    once the stream has finished the call; at return when report is True).
    `workspace` (uint8 CUDA tensor of ct_pdtv_workspace_bytes) holds the
    iteration state for params.resume.  trace (needs report): the report's
    "trace" lists the cost of Eq. 1 (low-dose) or ||Ax - b|| (few-view)
    after each iteration."""
    pb = _buf(b, "b", (g.n_views, g.n_bins))
    pw = None if w is None else _buf(w, "w", (g.n_views, g.n_bins))
    if x_out is None:
        x_out = torch.empty(g.n, g.n, device=b.device, dtype=torch.float32, pin_memory=not b.is_cuda)
    px = _buf(x_out, "x_out", (g.n, g.n))
    pws = None
    if workspace is not None:
        if not workspace.is_cuda or workspace.numel() * workspace.element_size() < ct_pdtv_workspace_bytes(g, params):
            raise ValueError("workspace too small")
        pws = ctypes.c_void_p(workspace.data_ptr())
    p = params.to_c()
    rep = ct_pdtv_report() if report or trace else None
    tr = (_d * max(int(params.iters), 1))() if trace else None
    if tr is not None:
        rep.trace = ctypes.cast(tr, ctypes.POINTER(_d))
    _check(_lib.ct_pdtv_solve(g.handle, pb, pw, ctypes.byref(p), px, pws,
                              ctypes.byref(rep) if rep is not None else None, _stream()))
    out = rep.as_dict() if rep is not None else None
    if tr is not None:
        out["trace"] = [tr[i] for i in range(int(params.iters))]
    return x_out, out


def ct_pdtv_status(workspace: torch.Tensor) -> None:
    """Raise CTError if the last solve with this workspace found a weight
    w_i <= 0 or NaN / infinity in b, w or the image (synchronises)."""
    _check(_lib.ct_pdtv_status(ctypes.c_void_p(workspace.data_ptr()), _stream()))


def workspace_for(g: Geometry, params: PDTVParams, device="cuda") -> torch.Tensor:
    n = ct_pdtv_workspace_bytes(g, params)
    return torch.empty(n, dtype=torch.uint8, device=device)


class BatchedSolve:
    """ct_pdtv_solve_batched over a fixed list of slices.  The slices'
    workspaces and outputs are allocated once here, so run() enqueues only
    device work (and can be captured in a CUDA graph)."""

    def __init__(self, slices, autotune=False):
        # slices: list of (Geometry, b, w or None, PDTVParams).  autotune:
        # run ct_geometry_autotune once per distinct geometry first, then
        # time the batched call's two forms (persistent launch, stream
        # pool) once each and keep the faster for run() (not capturable; do
        # it here, before any graph capture of run()).
        self.slices = list(slices)
        n = len(self.slices)
        if autotune:
            seen = set()
            for g, _, _, _ in self.slices:
                if id(g) not in seen:
                    seen.add(id(g))
                    g.autotune()
        self.x = [torch.empty(g.n, g.n, device=b.device, dtype=torch.float32) for g, b, w, p in self.slices]
        self.ws = [workspace_for(g, p, b.device) for g, b, w, p in self.slices]
        for g, b, w, p in self.slices:
            _dev(b, "b", (g.n_views, g.n_bins))
            if w is not None:
                _dev(w, "w", (g.n_views, g.n_bins))
        V = ctypes.c_void_p * n
        self._g = V(*[g.handle for g, _, _, _ in self.slices])
        self._b = V(*[b.data_ptr() for _, b, _, _ in self.slices])
        self._w = V(*[(w.data_ptr() if w is not None else None) for _, _, w, _ in self.slices])
        self._p = (ct_pdtv_params * n)(*[p.to_c() for _, _, _, p in self.slices])
        self._x = V(*[t.data_ptr() for t in self.x])
        self._ws = V(*[t.data_ptr() for t in self.ws])
        self.n = n
        self.form = None          # None: the process-wide choice (ct_batched_options)
        self.form_ms = {}
        if autotune:
            self._pick_form()

    def _enqueue(self, rep=None):
        _check(_lib.ct_pdtv_solve_batched(self.n, self._g, self._b, self._w, self._p, self._x, self._ws,
                                          rep, _stream()))

    def _pick_form(self):
        """Time each form once after one warm-up call (CUDA events) and keep the faster."""
        try:
            for form in (CT_BATCH_AUTO, CT_BATCH_POOL):
                ct_batched_options(form)
                self._enqueue()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                self._enqueue()
                e1.record()
                torch.cuda.synchronize()
                self.form_ms[form] = e0.elapsed_time(e1)
        finally:
            ct_batched_options(CT_BATCH_AUTO)
        self.form = min(self.form_ms, key=self.form_ms.get)

    def run(self, reports=False):
        rep = (ct_pdtv_report * self.n)() if reports else None
        if self.form is None:
            self._enqueue(rep)
        else:
            try:
                ct_batched_options(self.form)
                self._enqueue(rep)
            finally:
                ct_batched_options(CT_BATCH_AUTO)
        return self.x, ([r.as_dict() for r in rep] if reports else None)


def ct_pdtv_solve_batched(slices, reports=True):
    """Solve a list of (Geometry, b, w or None, PDTVParams) slices in one call."""
    bs = BatchedSolve(slices)
    return bs.run(reports=reports)


def ct_unrolled_workspace_bytes(g: Geometry, batch: int, half_len: int, iters: int, tv_iters: int) -> int:
    return int(_lib.ct_unrolled_workspace_bytes(g.handle, int(batch), int(half_len), int(iters), int(tv_iters)))


def ct_unrolled_forward(g: Geometry, b: torch.Tensor, w: torch.Tensor | None, taps: torch.Tensor,
                        tau: float, sigma: float, beta: float, mode: int, iters: int, tv_iters: int,
                        workspace: torch.Tensor, x_out: torch.Tensor | None = None) -> torch.Tensor:
    """x_K of the unrolled iteration (batch over b's leading dims); the
    per-iteration checkpoints stay in `workspace` for ct_unrolled_backward."""
    pb = _dev(b, "b", (g.n_views, g.n_bins))
    batch = _batch(b, 2)
    pw = None if w is None else _dev(w, "w", (g.n_views, g.n_bins))
    half = (taps.numel() + 1) // 2
    if x_out is None:
        x_out = torch.empty(*b.shape[:-2], g.n, g.n, device=b.device, dtype=torch.float32)
    _check(_lib.ct_unrolled_forward(g.handle, pb, pw, batch, _dev(taps, "taps"), half, float(tau), float(sigma),
                                    float(beta), int(mode), int(iters), int(tv_iters),
                                    _dev(x_out, "x_out", (g.n, g.n)), ctypes.c_void_p(workspace.data_ptr()),
                                    _stream()))
    return x_out


def ct_unrolled_backward(g: Geometry, b: torch.Tensor, w: torch.Tensor | None, taps: torch.Tensor,
                         tau: float, sigma: float, beta: float, mode: int, iters: int, tv_iters: int,
                         grad_x: torch.Tensor, workspace: torch.Tensor) -> torch.Tensor:
    """(dL/dtaps, dL/dbeta) as one float tensor of 2*half_len values."""
    half = (taps.numel() + 1) // 2
    grad = torch.empty(2 * half, device=b.device, dtype=torch.float32)
    _check(_lib.ct_unrolled_backward(g.handle, _dev(b, "b", (g.n_views, g.n_bins)),
                                     None if w is None else _dev(w, "w", (g.n_views, g.n_bins)), _batch(b, 2),
                                     _dev(taps, "taps"), half, float(tau), float(sigma), float(beta), int(mode),
                                     int(iters), int(tv_iters), _dev(grad_x.contiguous(), "grad_x", (g.n, g.n)),
                                     _dev(grad, "grad"), ctypes.c_void_p(workspace.data_ptr()), _stream()))
    return grad
