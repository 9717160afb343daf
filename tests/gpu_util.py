"""Helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from conftest import build_library
    build_library()
    import paper_1609_06041_gb300 as P
    return P


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    """The float32 values the GPU sees, as float64 for the oracle."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
