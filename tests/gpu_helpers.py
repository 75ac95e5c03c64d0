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


def fp32_floor(N, sigma, m, k, f, w):
    """Single-precision floor of the method: the oracle's steps (Algorithms 1
    and 2) run with complex64 arrays, FP32 window weights (scaled to 1 at
    u = 0, as the library stores them) and single-precision sums and FFTs,
    compared with the FP64 oracle.  Returns the relative L2 errors (forward
    on the nodes k, adjoint from the nodes k with inputs w).  The kernels
    use another summation order, so their error is a small multiple of this,
    not equal to it."""
    import itertools
    from oracle import nfft as onfft
    p = onfft.Params(N, sigma, m)
    c64, f32 = np.complex64, np.float32
    peaks = [float(onfft.psi(0.0, m, b)) for b in p.b]
    peak = float(np.prod(peaks))
    ls, us = onfft.footprint(p, k)
    wts = [(p.window(u, b) / pk).astype(f32) for u, b, pk in zip(us, p.b, peaks)]
    taps = list(itertools.product(range(p.taps()), repeat=p.D))

    def tap_index(tap):
        return tuple(np.mod(ls[d][:, tap[d]], p.Nt[d]) for d in range(p.D))

    def tap_weight(tap):
        wt = np.ones(k.shape[0], f32)
        for d in range(p.D):
            wt = wt * wts[d][:, tap[d]]
        return wt

    # forward
    exact = onfft.resample(p, k, onfft.fft_forward(onfft.correction_pad(p, f)))
    gh = np.fft.fftn((onfft.correction_pad(p, f) * peak).astype(c64))
    assert gh.dtype == c64, "numpy FFT must run in single precision for this model"
    out = np.zeros(k.shape[0], c64)
    for tap in taps:
        out += gh[tap_index(tap)] * tap_weight(tap)
    e_f = rel_l2(out.astype(np.complex128), exact)
    # adjoint
    exact_a = onfft.crop_correction(p, onfft.fft_adjoint(onfft.resample_adjoint(p, k, w)))
    acc = np.zeros(int(np.prod(p.Nt)), c64)
    w32 = np.asarray(w).astype(c64)
    for tap in taps:
        np.add.at(acc, np.ravel_multi_index(tap_index(tap), p.Nt), w32 * tap_weight(tap))
    g = np.fft.ifftn(acc.reshape(p.Nt), norm="forward")
    y = onfft.crop_correction(p, g.astype(np.complex128)).astype(c64) * f32(peak)
    return e_f, rel_l2(y.astype(np.complex128), exact_a)


def oracle_spread_box(N, sigma, m, k, w, lo, size):
    """The oracle's adjoint resampling step (Algorithm 2, Eq. SumOverNodeAdjoint)
    on the grid box [lo_d, lo_d + size) (periodic): only the nodes whose
    footprint meets the box contribute there, so the oracle runs on those
    alone.  Returns the box (size^D complex) and its index arrays."""
    from oracle import nfft as onfft
    p = onfft.Params(N, sigma, m)
    sel = np.ones(k.shape[0], bool)
    for d in range(p.D):
        c = np.mod(np.floor(p.Nt[d] * k[:, d]).astype(np.int64), p.Nt[d])
        d0 = np.mod(c - m + 1 - lo[d], p.Nt[d])    # footprint = d0 .. d0 + 2m - 1 (mod N~) from lo
        sel &= (d0 < size) | (d0 + 2 * m - 1 >= p.Nt[d])
    g = onfft.resample_adjoint(p, k[sel], w[sel])
    idx = np.ix_(*[np.mod(np.arange(lo[d], lo[d] + size), p.Nt[d]) for d in range(p.D)])
    return g[idx], idx, int(sel.sum())

