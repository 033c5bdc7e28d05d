"""The C ABI library builds, loads and exports every symbol include/sho.h declares (CPU only: only
host-side entry points are called here; nothing touches a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            with open(os.path.join(ROOT, "include", f)) as fh:
                txt = fh.read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sho_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1905_00480_gb300 import build
    build.build()
    from paper_1905_00480_gb300 import _native
    return _native.lib()


def test_header_declares_entry_points():
    names = _declared_symbols()
    for required in ("sho_project", "sho_add", "sho_forces", "sho_create", "sho_destroy", "sho_sync",
                     "sho_nstates", "sho_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported by libsho.so"


def test_binding_signatures_cover_header(lib):
    from paper_1905_00480_gb300 import _native
    assert set(_declared_symbols()) <= set(_native.SIGNATURES), "binding misses a declared symbol"


def test_host_only_entry_points(lib):
    assert lib.sho_version() == 1
    assert [lib.sho_nstates(n) for n in range(6)] == [1, 4, 10, 20, 35, 56]
    assert lib.sho_nstates(-1) == 0
    import math
    assert abs(lib.sho_max_spacing(0.8, 5) - math.pi * 0.8 / math.sqrt(11)) < 1e-15
    for st in range(-12, 1):
        assert lib.sho_strerror(st)


def test_null_handle_is_rejected_before_any_device_work(lib):
    from paper_1905_00480_gb300 import _native as N
    g = N.sho_grid()
    g.n[0] = g.n[1] = g.n[2] = 16
    g.h = 0.25
    st = lib.sho_project(None, ctypes.byref(g), None, 0, 4, 1, None, None, 3, 16, 0, None, 0, None)
    assert st == -1
    assert lib.sho_destroy(None) == -1
    assert lib.sho_sync(None) == -1


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.sho_create(ctypes.byref(h), 0)
    assert st in (-7, -1)
