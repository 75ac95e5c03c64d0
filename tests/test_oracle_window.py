"""Pins for oracle/window.py (no GPU).

Each test checks the oracle against something other than its own formula:
quadrature of the Fourier integral, a power series, finite differences, the
value printed in the paper.
"""
import math
import os

import numpy as np
import pytest

from oracle import window

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _i0_series(x):
    # I0(x) = sum_k (x^2/4)^k / (k!)^2 summed in Python floats.
    t, s, k = 1.0, 1.0, 0
    while t > 1e-18 * s:
        k += 1
        t *= (x * x / 4.0) / (k * k)
        s += t
    return s


@pytest.mark.parametrize("x", [0.0, 0.5, 3.0, 11.0, 18.849555921538759, 37.7])
def test_i0_against_power_series(x):
    assert np.i0(x) == pytest.approx(_i0_series(x), rel=1e-14)


@pytest.mark.parametrize("m,sigma,N", [(4, 2.0, 64), (6, 1.25, 128), (8, 2.0, 256), (2, 2.0, 16)])
def test_window_pair_by_quadrature(m, sigma, N):
    """The pair is exact in this direction: phi, compactly supported in
    frequency (|2 pi xi / N~| <= b), transforms to the window,
        psi(u) = (1/(2 pi)) int_{-b}^{b} I0(m sqrt(b^2 - w^2)) cos(w u) dw,
    (Sec. 2.2, Eq. FTWindow, with xi = N~ w / (2 pi)); the integrand is
    entire, so Gauss-Legendre converges to rounding.  This pins b, the
    normalisation and the edge value b/pi together."""
    Nt = window.oversampled_size(N, sigma)
    b = window.kb_shape(N, Nt)
    x, wq = np.polynomial.legendre.leggauss(300)
    om = b * x
    spec = np.i0(m * np.sqrt(b * b - om * om))
    peak = float(window.psi(0.0, m, b))
    for u in [0.0, 0.37, 1.0, m / 2.0, m - 0.5, m - 1e-3, float(m)]:
        quad = b * np.sum(wq * spec * np.cos(om * u)) / (2 * np.pi)
        # the cosine sum cancels near the edge: bound the error by the peak
        assert abs(quad - float(window.psi(u, m, b, closed=True))) < 1e-13 * peak
    # and phi(n) samples that spectrum: (1/N~) I0(...) at w = 2 pi n / N~
    for n in [0, 1, N // 4, N // 2 - 1, -N // 2]:
        om_n = 2 * np.pi * n / Nt
        assert window.phi(n, Nt, m, b) == pytest.approx(_i0_series(m * math.sqrt(b * b - om_n ** 2)) / Nt, rel=1e-13)


def test_truncated_window_transform_is_close_to_phi():
    """Truncating the window to [-m, m) changes its transform only by the
    truncation error, which shrinks with m (Eq. approxTrunc)."""
    x, wq = np.polynomial.legendre.leggauss(400)
    for m, tol in [(4, 1e-8), (6, 1e-12), (8, 1e-13)]:
        Nt = 128
        b = window.kb_shape(64, Nt)
        u = m * x
        vals = window.psi(u, m, b, closed=True)
        for n in [0, 9, 31]:
            quad = m * np.sum(wq * vals * np.cos(2 * np.pi * n * u / Nt)) / Nt
            assert abs(quad / window.phi(n, Nt, m, b) - 1) < tol


def test_window_support_and_edges():
    m, b = 4, window.kb_shape(64, 128)
    assert window.psi(m, m, b) == 0.0            # half-open [-m, m)
    assert window.psi(-m, m, b) == pytest.approx(b / np.pi, rel=1e-15)
    assert window.psi(m, m, b, closed=True) == pytest.approx(b / np.pi, rel=1e-15)
    assert window.psi(m + 1e-9, m, b, closed=True) == 0.0
    # continuity at the edge: the s -> 0 limit is b/pi
    assert window.psi(m - 1e-10, m, b) == pytest.approx(b / np.pi, rel=1e-6)
    u = np.linspace(-3.9, 3.9, 101)
    assert np.allclose(window.psi(u, m, b), window.psi(-u, m, b), rtol=1e-15)
    # peak at u = 0: sinh(b m)/(pi m)
    assert window.psi(0.0, m, b) == pytest.approx(math.sinh(b * m) / (math.pi * m), rel=1e-14)


@pytest.mark.parametrize("m", [2, 4, 8])
def test_dpsi_by_finite_differences(m):
    b = window.kb_shape(100, 200)
    h = 1e-6
    # interior points, points near the edge (small z series) and u = 0
    u = np.concatenate([np.linspace(-m + 0.3, m - 0.3, 37), [m - 1e-3, -m + 1e-3, m - 1e-5, 0.0]])
    fd = (window.psi(u + h, m, b, closed=True) - window.psi(u - h, m, b, closed=True)) / (2 * h)
    an = window.dpsi(u, m, b, closed=True)
    scale = np.max(np.abs(window.psi(np.linspace(-m, m, 9), m, b, closed=True)))
    assert np.max(np.abs(fd - an)) < 1e-6 * scale


def test_dpsi_edge_limit():
    """Near the support edge the derivative tends to -u b^3/(3 pi)."""
    m, b = 4, window.kb_shape(64, 128)
    u = m - 1e-12
    assert window.dpsi(u, m, b) == pytest.approx(-u * b ** 3 / (3 * np.pi), rel=1e-6)


def test_lut_size_matches_paper_value():
    path = os.path.join(os.path.dirname(__file__), "golden", "lut_size_m8.txt")
    line = [ln for ln in open(path) if ln.startswith("m=")][0]
    fields = dict(kv.split("=") for kv in line.split())
    assert window.lut_size(int(fields["m"])) == int(fields["S"])
    # the rule caps the exponent index at 8
    assert window.lut_size(10) == 10 * 2 ** 24 + 2


def test_oversampled_sizes():
    assert window.oversampled_size(256, 2.0) == 512
    assert window.oversampled_size(128, 1.25) == 160
    assert window.oversampled_size(16, 2.0) == 32
    assert window.oversampled_size(15, 2.0) == 30
    assert window.oversampled_size(13, 1.25) == 18   # 16.25 -> even ceiling


def test_index_set_even_and_odd():
    assert list(window.index_set(4)) == [-2, -1, 0, 1]
    assert list(window.index_set(5)) == [-2, -1, 0, 1, 2]


def test_deconv_factor_is_reciprocal_of_scaled_phi():
    """beta^tensor of Sec. 3.5 in unscaled form: 1/(N~ phi(n)) = 1/I0(...)."""
    Nt, m = 128, 4
    b = window.kb_shape(64, Nt)
    n = np.arange(-32, 32)
    expect = np.array([1.0 / _i0_series(m * math.sqrt(b * b - (2 * math.pi * v / Nt) ** 2)) for v in n])
    assert np.allclose(window.deconv_factor(n, Nt, m, b), expect, rtol=1e-13)


def test_untruncated_window_continuation():
    """psi_full equals psi inside the support, is continuous through |u| = m
    (both branches tend to b/pi) and is the sin form beyond."""
    m, b = 4, window.kb_shape(64, 128)
    u = np.linspace(-3.9, 3.9, 41)
    assert np.allclose(window.psi_full(u, m, b), window.psi(u, m, b), rtol=1e-15)
    for eps in (1e-8, 1e-10):   # deviation ~ b^2 2m eps / 6
        assert window.psi_full(m - eps, m, b) == pytest.approx(b / np.pi, rel=1e-6)
        assert window.psi_full(m + eps, m, b) == pytest.approx(b / np.pi, rel=1e-6)
    x = 4.6
    sp = math.sqrt(x * x - m * m)
    assert window.psi_full(x, m, b) == pytest.approx(math.sin(b * sp) / (math.pi * sp), rel=1e-14)


def test_dpsi_full_by_finite_differences():
    m, b = 3, window.kb_shape(50, 100)
    h = 1e-6
    u = np.concatenate([np.linspace(-m - 0.95, m + 0.95, 53), [m + 1e-3, -m - 1e-3, m - 1e-3]])
    fd = (window.psi_full(u + h, m, b) - window.psi_full(u - h, m, b)) / (2 * h)
    an = window.dpsi_full(u, m, b)
    assert np.max(np.abs(fd - an)) < 1e-6 * np.max(np.abs(window.psi_full(np.linspace(-m, m, 9), m, b)))


@pytest.mark.parametrize("m,sigma", [(2, 2.0), (4, 2.0), (6, 1.25), (8, 2.0)])
def test_untruncated_window_is_one_entire_function(m, sigma):
    """psi_full continues sinh(b s)/(pi s) past |u| = m.  Since
    sinh(b s)/s = sum_k b^(2k+1) (s^2)^k/(2k+1)! is a power series in
    s^2 = m^2 - u^2 alone, that one series must give psi_full on both sides of
    the edge (no inside/outside branch): a wrong continuation beyond the
    support, or a wrong branch choice, fails here."""
    b = window.kb_shape(64, window.oversampled_size(64, sigma))
    u = np.concatenate([np.linspace(-m - 1.5, -m + 1.5, 61), np.linspace(m - 1.5, m + 1.5, 61)])
    s2 = m * m - u * u
    series = np.zeros_like(u)
    term = np.full_like(u, b)           # b^(2k+1) (s^2)^k / (2k+1)!, k = 0
    for kk in range(60):
        series += term
        term = term * b * b * s2 / ((2 * kk + 2) * (2 * kk + 3))
    want = series / np.pi
    got = window.psi_full(u, m, b)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))



@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_linear_table_lookup(m):
    """LINEAR (Sec. 3.7.4): exact at the table's sample points u = m s/(S-2),
    linear between them, the edge entry S-2 holds b/pi (read by the tap at
    u = -m through |u|), entry S-1 is 0, and the interpolation error stays
    within the linear-interpolation bound h^2/8 max|psi''| (h = m/(S-2))."""
    b = window.kb_shape(32, 64)
    S = window.lut_size(m)
    h = m / (S - 2.0)
    s = np.array([0, 1, 7, (S - 2) // 3, S - 3, S - 2])
    assert np.allclose(window.psi_linear(s * h, m, b), window.psi(s * h, m, b), rtol=0, atol=1e-15)
    assert window.lut_entry(S - 2, m, b) == pytest.approx(b / np.pi, rel=1e-15)
    assert window.lut_entry(S - 1, m, b) == 0.0
    assert window.psi_linear(-float(m), m, b) == pytest.approx(b / np.pi, rel=1e-15)
    mid = (s[:-1] + 0.5) * h
    avg = 0.5 * (window.psi(s[:-1] * h, m, b, closed=True) + window.psi((s[:-1] + 1) * h, m, b, closed=True))
    assert np.allclose(window.psi_linear(mid, m, b), avg, rtol=0, atol=1e-15)
    assert np.allclose(window.psi_linear(-mid, m, b), avg, rtol=0, atol=1e-15)
    u = np.linspace(-m, m, 200001)[:-1]
    fd2 = np.abs(np.diff(window.psi(u, m, b), 2)) / (u[1] - u[0]) ** 2
    bound = h * h / 8 * fd2.max() * 1.01 + 1e-15
    assert np.max(np.abs(window.psi_linear(u, m, b) - window.psi(u, m, b))) <= bound


def test_linear_window_nfft_error_matches_direct():
    """Sec. 3.7.4: the table sizes keep the window's interpolation error below
    the NFFT's own error: with the LINEAR window the NFFT is as accurate
    against the exact NDFT as with the evaluated window (m = 2..6), and the
    NFFT operator stays adjoint to its adjoint."""
    from oracle import ndft, nfft
    rng = np.random.default_rng(30)
    k = rng.random((200, 2)) - 0.5
    f = rng.standard_normal((24, 20)) + 1j * rng.standard_normal((24, 20))
    w = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    ex = ndft.ndft(k, f)
    for m in range(2, 7):
        e_dir = np.linalg.norm(nfft.forward(k, f, 2.0, m) - ex) / np.linalg.norm(ex)
        e_lin = np.linalg.norm(nfft.forward(k, f, 2.0, m, window="linear") - ex) / np.linalg.norm(ex)
        assert e_lin <= 1.05 * e_dir
    lhs = np.vdot(w, nfft.forward(k, f, 2.0, 4, window="linear"))
    rhs = np.vdot(nfft.adjoint(k, w, (24, 20), 2.0, 4, window="linear"), f)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(w)
