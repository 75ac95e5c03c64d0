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


def assert_close(got, want, tol, what="", tol_max=None):
    """Element-wise parity: the relative L2 error within tol and the largest
    element error (relative to the largest element) within tol_max
    (default 10 tol)."""
    e2 = rel_l2(got, want)
    ei = rel_max(got, want)
    tm = 10 * tol if tol_max is None else tol_max
    assert e2 <= tol and ei <= tm, "%s: rel L2 %.3e, rel max %.3e, tol %.1e / %.1e" % (what, e2, ei, tol, tm)
    return e2


def to_dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def cdtype(name):
    return torch.complex64 if name == "c64" else torch.complex128


TOL = {"c64": 1e-5, "c128": 1e-12}
UNIT_ROUNDOFF = {"c64": 2.0 ** -24, "c128": 2.0 ** -53}


def kappa(N, sigma, m, norm="rms"):
    """Amplification of rounding errors by the resampling correction:
    prod_d rms(beta_d) / min(beta_d) over I_{N_d} (beta_d = 1/(N~_d phi_d));
    with norm="max" the element-wise version prod_d max(beta_d)/min(beta_d)."""
    from oracle import nfft as onfft
    from oracle import window
    p = onfft.Params(N, sigma, m)
    k = 1.0
    for n, nt, b in zip(p.N, p.Nt, p.b):
        beta = window.deconv_factor(window.index_set(n), nt, m, b)
        top = np.sqrt(np.mean(beta ** 2)) if norm == "rms" else beta.max()
        k *= float(top / beta.min())
    return k


def tol_for(N, sigma, m, dt):
    """Parity tolerance: the stated target (1e-5 complex64, 1e-12 complex128)
    unless the method's own conditioning in that precision is worse: the
    rounding of the deconvolved grid and of the FFT is amplified by kappa, so
    the bound is max(target, u * kappa), u the unit roundoff."""
    return max(TOL[dt], UNIT_ROUNDOFF[dt] * kappa(N, sigma, m))


def tol_max_for(N, sigma, m, dt):
    """Element-wise counterpart of tol_for: max(10 target, u * kappa_max)."""
    return max(10 * TOL[dt], UNIT_ROUNDOFF[dt] * kappa(N, sigma, m, norm="max"))
