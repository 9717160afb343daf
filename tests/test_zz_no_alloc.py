"""The allocation-free ramp filter (ct_ramp_filter_noalloc), called through
the C ABI, gives the allocating filter's result.  Some callers cannot
allocate device memory while they run (memory reserved once at start-up, or
a context where an allocation may block or fail); this entry point keeps its
scratch in a fixed device array instead.  This file is collected last."""
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


def test_noalloc_filter_rejects_large_detectors():
    P = need_gpu()
    import torch
    g = P.Geometry(16, 2, 4200)            # needs a 16384-point transform
    t = torch.zeros(2 * 4200 - 1, device="cuda")
    y = torch.zeros(2, 4200, device="cuda")
    with pytest.raises(P.CTError) as e:
        P.ct_ramp_filter_noalloc(g, t, y, torch.empty_like(y))
    assert e.value.status == 1 and "4096" in str(e.value)
