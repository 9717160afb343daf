import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built libctpd.so")


def build_library():
    """Build libctpd.so (by path, before the package that loads it is imported)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_1609_06041_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("ctpd_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
