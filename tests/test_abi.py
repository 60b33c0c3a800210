"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/mcproj.h declares; the binding's signatures cover them all."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mcp_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2604_13323_gb300 import build
    return ctypes.CDLL(build.build())


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 14, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2604_13323_gb300 import mcproj
    assert sorted(mcproj.EXPORTED) == declared_functions()


def test_create_without_device_fails_cleanly(lib):
    """No GPU here: mcp_create reports an error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.mcp_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.mcp_create(0, ctypes.byref(h)) != 0
    assert not h.value


def test_every_entry_point_rejects_a_null_context(lib):
    """Bad arguments never abort: with no context every call returns
    MCP_ERR_ARG (1) before touching memory or the GPU; destroy, the error
    message and the launch count accept NULL; the allocation count takes no
    context."""
    from paper_2604_13323_gb300 import mcproj
    L = mcproj.load_library()
    skip = {"mcp_create", "mcp_destroy", "mcp_last_error", "mcp_launch_count", "mcp_alloc_count"}
    for name in mcproj.EXPORTED:
        if name in skip:
            continue
        fn = getattr(L, name)
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_float, ctypes.c_double):
                args.append(0.0)
            elif t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64):
                args.append(0)
            else:
                args.append(None)
        assert fn(*args) == 1, name
    assert L.mcp_create(0, None) == 1
    L.mcp_destroy(None)
    assert L.mcp_last_error(None)
    assert L.mcp_launch_count(None) == 0
    assert L.mcp_alloc_count() == 0   # nothing allocated without a device
