"""Shared helpers for the GPU parity tests (imported only by -m gpu tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import __graft_entry__
    __graft_entry__.build()


def rel_l2(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.linalg.norm((got - want).ravel()) / max(np.linalg.norm(want.ravel()), 1e-300))


def rel_max(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def assert_close(got, want, tol, what=""):
    """Element-wise parity: both the relative L2 error and the largest
    element error (relative to the largest element) within tol."""
    e2 = rel_l2(got, want)
    ei = rel_max(got, want)
    assert e2 <= tol and ei <= 10 * tol, "%s: rel L2 %.3e, rel max %.3e, tol %.1e" % (what, e2, ei, tol)
    return e2


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def cdtype(name):
    return torch.complex64 if name == "c64" else torch.complex128


TOL = {"c64": 1e-5, "c128": 1e-12}
