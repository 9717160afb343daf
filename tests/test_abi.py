"""The C ABI library loads without a GPU and exports every entry point the
public header declares; the binding declares exactly those names."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ct_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from conftest import build_library
    return build_library()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ct_\w+)", out))
    declared = declared_functions()
    assert declared, "no declarations found"
    assert declared <= exported, f"missing: {sorted(declared - exported)}"


def test_binding_loads_and_names_match(lib_path):
    from paper_1609_06041_gb300 import ctpd
    assert set(ctpd.EXPORTS) == declared_functions()
    assert ctpd.ct_version().startswith("ctpd")
    assert ctpd.ct_last_error() == ""


def test_geometry_rejects_bad_sizes_without_gpu(lib_path):
    from paper_1609_06041_gb300 import ctpd
    with pytest.raises(ctpd.CTError) as e:
        ctpd.Geometry(0, 10, 10)
    assert e.value.status == ctpd.CT_ERR_ARG
    with pytest.raises(ctpd.CTError):
        ctpd.Geometry(16, 10, 9000)
