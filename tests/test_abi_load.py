"""The C-ABI library builds, loads and exports every entry point the header declares.

Runs without a GPU: only argument validation is exercised (it happens before
any CUDA call), never a kernel.
"""
import ctypes
import os
import re

import pytest

import paper_1610_09146_gb300 as fd
from paper_1610_09146_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    fd.build()
    return native.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("fd_create", "fd_step", "fd_get_state", "fd_set_state", "fd_diagnostics", "fd_destroy",
                     "fd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(native.exported_symbols()) | {"fd_create"}


def test_binding_constants_match_the_header():
    text = open(os.path.join(ROOT, "include", "fdgb300.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (FD_[A-Z0-9_]+) \(?(-?\d+)\)?", text)}
    assert len(defines) >= 20
    for name, value in defines.items():
        assert getattr(native, name) == value, name
    # the profile class names follow the FD_KERNEL_* numbering
    classes = sorted((v, k) for k, v in defines.items() if k.startswith("FD_KERNEL_") and k != "FD_KERNEL_CLASSES")
    assert [k[len("FD_KERNEL_"):].lower() for _, k in classes] == list(native.KERNEL_CLASS_NAMES)
    assert len(classes) == defines["FD_KERNEL_CLASSES"]


@pytest.mark.parametrize("args,code", [
    ((4, 16, 16, 1600, 0.1, 0.71, 1.4, 1e-3, 0, 0), fd.FD_EINVAL),          # axis < 5
    ((16, 16, 16, 0.0, 0.1, 0.71, 1.4, 1e-3, 0, 0), fd.FD_EINVAL),          # Re <= 0
    ((16, 16, 16, 1600, 0.1, 0.71, 1.0, 1e-3, 0, 0), fd.FD_EINVAL),         # gamma <= 1
    ((16, 16, 16, 1600, 0.1, 0.71, 1.4, -1.0, 0, 0), fd.FD_EINVAL),         # dt <= 0
    ((16, 16, 16, 1600, float("nan"), 0.71, 1.4, 1e-3, 0, 0), fd.FD_EINVAL),
    ((16, 16, 16, 1600, 0.1, 0.71, 1.4, 1e-3, 7, 0), fd.FD_EINVAL),         # unknown algorithm
    ((16, 16, 16, 1600, 0.1, 0.71, 1.4, 1e-3, 0, 9), fd.FD_EINVAL),         # unknown dtype
    ((2048, 2048, 1024, 1600, 0.1, 0.71, 1.4, 1e-3, 0, 0), fd.FD_EINVAL),   # >= 2^31 points
    ((600, 600, 600, 1600, 0.1, 0.71, 1.4, 1e-3, 0, 0), fd.FD_EINVAL),      # above 214748364 points
])
def test_create_rejects_bad_arguments(lib, args, code):
    h = ctypes.c_void_p()
    rc = lib.fd_create(ctypes.byref(h), *args, None, None)
    assert rc == code
    assert h.value is None
    assert fd.fd_last_error(None) != ""


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.fd_step(None, 1) == fd.FD_EINVAL
    assert lib.fd_diagnostics(None, None, None) == fd.FD_EINVAL
    assert lib.fd_destroy(None) == fd.FD_OK
    assert lib.fd_device_bytes(None) == 0
    assert "NULL" in fd.fd_last_error(None) or fd.fd_last_error(None) != ""
