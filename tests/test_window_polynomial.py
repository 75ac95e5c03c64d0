"""The POLYNOMIAL window representation used by the specialised complex64
kernels (Sec. 3.7.4, item 5, as read here): on each of the 2m unit tap
intervals the window, scaled to 1 at u = 0, is a polynomial of degree 2m in
zeta = t - 1/2 (t the node's fraction), fitted by interpolation at the 2m + 1
Chebyshev points of [-1/2, 1/2] in FP64, stored in FP32 and evaluated by a
Horner chain of fused multiply-adds in FP32.  This re-derives that scheme on
the CPU and checks it against the oracle's direct window: the fit itself is
far below FP32 resolution, and the FP32 evaluation stays within 1e-7 of the
window's peak (the kernels' 1e-5 target leaves ample room)."""
import numpy as np
import pytest

from oracle import window as ow


def _fit(m, b, i):
    """Coefficients (increasing powers of zeta) for tap i of the 2m-point
    footprint: u = N~k - l = t + m - 1 - i, zeta = t - 1/2."""
    Z = 2 * m + 1
    zeta = 0.5 * np.cos(np.pi * (np.arange(Z) + 0.5) / Z)
    u = zeta + 0.5 + (m - 1) - i
    val = ow.psi(u, m, b) / ow.psi(np.array([0.0]), m, b)[0]
    return np.linalg.solve(np.vander(zeta, Z, increasing=True), val)


def _horner_fp32_fma(c, zeta):
    """FP32 coefficients, FP32 Horner with one rounding per step (a float32
    product is exact in float64, so rounding p * z + c once to float32 is a
    fused multiply-add)."""
    c32 = c.astype(np.float32)
    z = zeta.astype(np.float32).astype(np.float64)
    p = np.full(zeta.shape, c32[-1], dtype=np.float32)
    for cz in c32[-2::-1]:
        p = (p.astype(np.float64) * z + np.float64(cz)).astype(np.float32)
    return p.astype(np.float64)


@pytest.mark.parametrize("m,sigma,fit_tol", [(4, 2.0, 1e-8), (4, 1.25, 1e-8), (6, 2.0, 1e-12),
                                             (6, 1.25, 1e-12), (8, 2.0, 1e-12)])
def test_polynomial_window_against_direct_window(m, sigma, fit_tol):
    b = np.pi * (2.0 - 1.0 / sigma)
    zeta = np.linspace(-0.5, 0.5, 2001)[:-1]          # t in [0, 1)
    worst_fit = worst_fp32 = 0.0
    for i in range(2 * m):
        c = _fit(m, b, i)
        u = zeta + 0.5 + (m - 1) - i
        ref = ow.psi(u, m, b) / ow.psi(np.array([0.0]), m, b)[0]
        worst_fit = max(worst_fit, np.max(np.abs(np.polynomial.polynomial.polyval(zeta, c) - ref)))
        worst_fp32 = max(worst_fp32, np.max(np.abs(_horner_fp32_fma(c, zeta) - ref)))
    assert worst_fit <= fit_tol
    assert worst_fp32 <= 1e-7


def test_polynomial_taps_cover_the_footprint():
    """The 2m tap intervals tile u in [-m, m) exactly once: tap i covers
    u in [m - 1 - i, m - i); the last tap at t = 0 is the support's edge
    u = -m, where the window is b / pi (reproduced to the fit's accuracy,
    which is relative to the window's peak psi(0))."""
    m, b = 4, np.pi * 1.5
    lo = np.array([m - 1 - i for i in range(2 * m)], dtype=float)
    assert np.array_equal(np.sort(lo), np.arange(-m, m, dtype=float))
    c = _fit(m, b, 2 * m - 1)
    peak = ow.psi(np.array([0.0]), m, b)[0]
    edge = np.polynomial.polynomial.polyval(-0.5, c) * peak
    assert abs(edge - b / np.pi) <= 1e-8 * peak


def _fit_deg(m, b, i, deg):
    """As _fit, at another degree (deg + 1 Chebyshev points)."""
    Z = deg + 1
    zeta = 0.5 * np.cos(np.pi * (np.arange(Z) + 0.5) / Z)
    u = zeta + 0.5 + (m - 1) - i
    val = ow.psi(u, m, b) / ow.psi(np.array([0.0]), m, b)[0]
    return np.linalg.solve(np.vander(zeta, Z, increasing=True), val)


@pytest.mark.parametrize("sigma", [1.5, 2.0])
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7, 8])
def test_complex128_default_polynomial_reaches_fp64_rounding(m, sigma):
    """Complex128 plans without a window flag and with oversampling of at
    least 1.5 (or m >= 7) read the window from a polynomial of degree
    max(2m, 16) per tap interval, fitted in FP64 the same way: its error
    against the direct window stays within 2e-14 of the peak, the level of
    the direct form's own FP64 evaluation, for every m the complex128
    kernels take."""
    b = np.pi * (2.0 - 1.0 / sigma)
    deg = max(2 * m, 16)
    zeta = np.linspace(-0.5, 0.5, 2001)[:-1]
    worst = 0.0
    for i in range(2 * m):
        c = _fit_deg(m, b, i, deg)
        u = zeta + 0.5 + (m - 1) - i
        ref = ow.psi(u, m, b) / ow.psi(np.array([0.0]), m, b)[0]
        worst = max(worst, np.max(np.abs(np.polynomial.polynomial.polyval(zeta, c) - ref)))
    assert worst <= 2e-14


def test_complex128_default_polynomial_leaves_the_transform_at_rounding():
    """The oracle's NFFT with the window replaced by the degree-16 table
    reading (2D, 48 x 40, m = 4, sigma = 2; 1D, N = 257, m = 3) against the
    oracle with the direct window: the transforms differ at the FP64
    rounding level (<= 1e-13 relative L2), three orders below the
    complex128 target of 1e-12."""
    from oracle import nfft as onfft
    from paper_2208_00049_gb300 import inputs

    for N, M, sigma, m in (((48, 40), 600, 2.0, 4), ((257,), 513, 2.0, 3)):
        case = inputs.small_case(N, M, seed=17, sigma=sigma, m=m)
        p = onfft.Params(N, sigma, m)
        deg = max(2 * m, 16)
        tables = {bb: [_fit_deg(m, bb, i, deg) for i in range(2 * m)] for bb in set(p.b)}
        peak = {bb: ow.psi(np.array([0.0]), m, bb)[0] for bb in set(p.b)}

        def poly_window(self, u, bb):
            u = np.asarray(u, dtype=float)
            fl = np.floor(u)
            tap = (m - 1 - fl).astype(int)
            zeta = (u - fl) - 0.5
            out = np.zeros_like(u)
            for i, c in enumerate(tables[bb]):
                sel = tap == i
                out[sel] = np.polynomial.polynomial.polyval(zeta[sel], c) * peak[bb]
            return out

        ref_f = onfft.forward(case["k"], case["f"], sigma, m)
        ref_a = onfft.adjoint(case["k"], case["w"], N, sigma, m)
        orig = onfft.Params.window
        onfft.Params.window = poly_window
        try:
            got_f = onfft.forward(case["k"], case["f"], sigma, m)
            got_a = onfft.adjoint(case["k"], case["w"], N, sigma, m)
        finally:
            onfft.Params.window = orig
        assert np.linalg.norm(got_f - ref_f) <= 1e-13 * np.linalg.norm(ref_f)
        assert np.linalg.norm(got_a - ref_a) <= 1e-13 * np.linalg.norm(ref_a)
