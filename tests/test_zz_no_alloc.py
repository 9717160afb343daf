"""The allocation-free ramp filter (ct_ramp_filter_noalloc), called through
the C ABI, gives the allocating filter's result.  Some callers cannot
allocate device memory while they run (memory reserved once at start-up, or
a context where an allocation may block or fail); this entry point keeps its
scratch in a fixed device array instead.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth
from gpu_util import need_gpu, rel_l2, to_gpu, to_np, f32

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_noalloc_filter_matches_allocating_filter_twice():
    P = need_gpu()
    import torch
    # two different problems back to back: the shared scratch array must
    # carry nothing from one call into the next
    cases = [(90, 95, 95, 0.05, 0.3, 0), (13, 530, 200, 0.01, 0.0, 1)]
    for V, B, half, tau, kappa, mode in cases:
        g = P.Geometry(16, V, B)
        t = to_gpu(f32(O.ramp_taps(mode, V, B, tau, kappa, half=half)))
        y = to_gpu(f32(synth.random_sinogram(V, B, V)))
        ref = P.ct_ramp_filter(g, t, y)
        out = torch.empty_like(y)
        got = P.ct_ramp_filter_noalloc(g, t, y, out)
        torch.cuda.synchronize()
        assert rel_l2(to_np(got), to_np(ref)) <= TOL
        assert rel_l2(to_np(got), O.filt(to_np(y), to_np(t))) <= TOL


class PoolWatch:
    """High-water mark of the device's default stream-ordered memory pool
    (the pool cudaMallocAsync draws from), read through the driver API:
    reset it, run the code, synchronise, and see whether it rose."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8   # CUmemPool_attribute

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ctypes.c_int(ordinal)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
        return v.value

    def reset(self):
        v = ctypes.c_uint64(0)   # 0 resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, ctypes.c_int(self.USED_MEM_HIGH), ctypes.byref(v)) == 0
        return self._get(self.USED_MEM_CURRENT)

    def high(self):
        return self._get(self.USED_MEM_HIGH)


def test_noalloc_filter_allocates_nothing():
    # the allocating filter raises the pool's high-water mark (so the probe
    # sees allocations); the allocation-free one, called twice, does not
    P = need_gpu()
    import torch
    V, B = 90, 95
    g = P.Geometry(16, V, B)
    t = to_gpu(f32(O.ramp_taps(0, V, B, 0.05, 0.3)))
    y = to_gpu(f32(synth.random_sinogram(V, B, 3)))
    out = torch.empty_like(y)
    P.ct_ramp_filter_noalloc(g, t, y, out)   # first call: looks up the scratch address
    torch.cuda.synchronize()
    watch = PoolWatch(torch.cuda.current_device())
    base = watch.reset()
    P.ct_ramp_filter(g, t, y)
    torch.cuda.synchronize()
    assert watch.high() > base
    base = watch.reset()
    for _ in range(2):
        P.ct_ramp_filter_noalloc(g, t, y, out)
    torch.cuda.synchronize()
    assert watch.high() == base


def test_noalloc_filter_rejects_another_device():
    P = need_gpu()
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU: no other device to call from")
    g = P.Geometry(16, 4, 20)
    t = torch.zeros(39, device="cuda:0")
    y = torch.zeros(4, 20, device="cuda:0")
    with torch.cuda.device(1):
        with pytest.raises(P.CTError) as e:
            P.ct_ramp_filter_noalloc(g, t, y, torch.empty_like(y))
    assert e.value.status == 1 and "device" in str(e.value)


def test_noalloc_filter_rejects_large_detectors():
    P = need_gpu()
    import torch
    g = P.Geometry(16, 2, 4200)            # needs a 16384-point transform
    t = torch.zeros(2 * 4200 - 1, device="cuda")
    y = torch.zeros(2, 4200, device="cuda")
    with pytest.raises(P.CTError) as e:
        P.ct_ramp_filter_noalloc(g, t, y, torch.empty_like(y))
    assert e.value.status == 1 and "4096" in str(e.value)
