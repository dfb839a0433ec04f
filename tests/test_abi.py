"""The C-ABI library loads and exports every entry point include/fp.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import paper_1711_08475_gb300 as fp
from paper_1711_08475_gb300 import native
from paper_1711_08475_gb300 import build as fpbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "fp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*FP_API\s+(?:const\s+)?[a-z_0-9]+\s*\**\s*(fp_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_header_symbols():
    path = fpbuild.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    names = header_functions()
    assert len(names) >= 16, names
    for n in names:
        assert hasattr(L, n), f"{n} missing from libfpmatch.so"
    # the binding declares exactly the header's functions
    assert sorted(native.SIGNATURES) == names


def test_host_only_calls():
    fp.load()
    assert "sm_103a" in fp.fp_version()
    L = native.load()
    assert L.fp_strerror(-2).decode().startswith("unsupported")
    assert fp.fp_launch_count() >= 0
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert L.fp_build(None, None, 0, 0, 32, None, None, ctypes.byref(h)) == native.FP_E_INVAL
    assert L.fp_query(None, None, None, 0, 1, 0, None, ctypes.byref(h)) == native.FP_E_INVAL


def test_no_cpu_fallback_in_product_package():
    pkg = os.path.join(ROOT, "paper_1711_08475_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert "import oracle" not in src and "from oracle" not in src, name
