"""The C-ABI library builds, loads and exports every entry point that
include/nfft_gb300.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nfft_gb300.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(nfft_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2208_00049_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["nfft_plan_create", "nfft_set_nodes", "nfft_forward", "nfft_adjoint",
                     "nfft_grad", "nfft_plan_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    handle = ctypes.CDLL(built_lib)
    for name in _declared_functions():
        assert hasattr(handle, name), name


def test_binding_covers_every_declared_symbol(built_lib):
    from paper_2208_00049_gb300 import binding
    assert sorted(binding.SIGNATURES) == _declared_functions()
    lib = binding.lib()
    for name in binding.SIGNATURES:
        assert getattr(lib, name).argtypes is not None or name == "nfft_strerror"


def test_status_strings_and_argument_validation(built_lib):
    """Host-side checks fail with status codes before touching a device."""
    from paper_2208_00049_gb300 import binding as B
    assert B.strerror(B.NFFT_OK) == "success"
    assert "invalid" in B.strerror(B.NFFT_ERR_INVALID_ARG)
    assert B.strerror(12345) == "unknown status code"
    bad = [
        dict(D=0, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0),
        dict(D=4, N=(16, 16, 16, 16), M=4, sigma=2.0, m=4, dtype=0, flags=0),
        dict(D=1, N=(1,), M=4, sigma=2.0, m=4, dtype=0, flags=0),
        dict(D=1, N=(16,), M=4, sigma=1.0, m=4, dtype=0, flags=0),
        dict(D=1, N=(16,), M=4, sigma=2.0, m=0, dtype=0, flags=0),
        dict(D=1, N=(40,), M=4, sigma=2.0, m=11, dtype=0, flags=0),
        dict(D=1, N=(4,), M=4, sigma=2.0, m=4, dtype=0, flags=0),   # 2m >= N~
        dict(D=1, N=(16,), M=-1, sigma=2.0, m=4, dtype=0, flags=0),
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=7, flags=0),
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0x100),
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0x60),   # two window modes
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0x48),   # LINEAR with the wide window
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0x81),   # POLYNOMIAL with closed support
        dict(D=1, N=(16,), M=4, sigma=2.0, m=4, dtype=0, flags=0x24),   # window mode with FULL_MATRIX
    ]
    for a in bad:
        s, h = B.nfft_plan_create(a["D"], a["N"], a["M"], a["sigma"], a["m"], a["dtype"], a["flags"], None)
        assert s == B.NFFT_ERR_INVALID_ARG and h is None, a
    # m = 9, 10 are built for 1D and 2D only
    s, h = B.nfft_plan_create(3, (24, 24, 24), 4, 2.0, 9, 0, 0, None)
    assert s == B.NFFT_ERR_UNSUPPORTED and h is None
    # null plan handles are rejected, destroy(NULL) is a no-op
    assert B.nfft_forward(None, None, None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_set_nodes(None, None, 1) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_plan_set_graph(None, 1) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_plan_set_async(None, 1) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_plan_sync(None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_plan_destroy(None) == B.NFFT_OK
    assert B.nfft_plan_grid(None) is None


def test_spread_noalloc_rejects_before_touching_a_device(built_lib):
    """The allocation-free spreading call checks its arguments on the host:
    invalid sizes, sizes beyond its static scratch, and buffers that are not
    device memory are rejected with a status code (no kernel is launched)."""
    import numpy as np
    from paper_2208_00049_gb300 import binding as B
    dummy = 256  # never dereferenced: the size checks come first
    assert B.nfft_spread_noalloc(0, (32,), 2.0, 4, 8, dummy, dummy, dummy, None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_spread_noalloc(1, (32,), 1.0, 4, 8, dummy, dummy, dummy, None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 0, 8, dummy, dummy, dummy, None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 4, 8, 0, dummy, dummy, None) == B.NFFT_ERR_INVALID_ARG
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 4, B.NFFT_NOALLOC_MAX_NODES + 1, dummy, dummy, dummy,
                                 None) == B.NFFT_ERR_UNSUPPORTED
    # host buffers of valid sizes: not device memory
    k = np.zeros((8, 1))
    w = np.zeros(8, np.complex64)
    g = np.zeros(64, np.complex64)
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 4, 8, k.ctypes.data, w.ctypes.data, g.ctypes.data,
                                 None) == B.NFFT_ERR_INVALID_ARG
