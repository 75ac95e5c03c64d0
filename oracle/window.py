"""Kaiser-Bessel window pair used by the oracle (TEST INFRASTRUCTURE ONLY).

Sources (arXiv 2208.00049, NFFT.jl):
  * Sec. 2.2 "Direct NFFT": the D-variate window is a tensor product of a
    1-D base window scaled by N~_d/m (window equation), and its inverse
    Fourier transform phi factorises the same way.
  * Sec. 2.2, Eq. approxTrunc: the window is truncated to the half-open
    support [-m/N~_d, m/N~_d) in k, i.e. u = N~_d k in [-m, m) in grid units.
  * Sec. 3.5: the deconvolution uses beta_d(n_d) = 1/(m phi_Base(m n_d/N~_d)),
    which equals 1/(N~_d phi_d(n_d)) in the unscaled notation used here.
  * Sec. 4 (Materials and Methods): the window is Kaiser-Bessel; the paper
    prints no formula, so the oracle takes the standard Kaiser-Bessel pair of
    the NFFT literature with shape b = pi (2 - 1/sigma) (reading recorded in
    the design notes) written in grid units:

        psi(u)  = sinh(b s) / (pi s),   s = sqrt(m^2 - u^2),   |u| < m
        psi(+-m) = b / pi              (limit s -> 0)
        phi(n)  = (1/N~) I0(m sqrt(b^2 - (2 pi n / N~)^2))

    phi(n) = integral psi(N~ k) exp(2 pi i n k) dk is pinned numerically by
    the tests (Gauss-Legendre quadrature), not assumed.
  * Sec. 3.7.4 (LINEAR precomputation): table size S = m 2^{c_min(m,8)} + 2
    with C = (3, 7, 9, 14, 17, 20, 23, 24); the paper prints S = 134217730
    for m = 8; entries psi_s = psi_Base(s/(S-2)) read with linear
    interpolation (Eq. linInterp).

Plain numpy, FP64.  Library primitives used: numpy.sinh, numpy.cosh,
numpy.sqrt, numpy.i0.
"""
import numpy as np

# Sec. 3.7.4: NFFT3's experimentally determined exponents c_m, m = 1..8.
LUT_EXPONENTS = (3, 7, 9, 14, 17, 20, 23, 24)


def oversampled_size(N, sigma):
    """N~ = sigma N rounded up to an even integer (Sec. 2.2 says N~ = sigma N;
    rounding up to even is the reading taken for non-integer sigma N)."""
    return int(2 * np.ceil(sigma * N / 2.0 - 1e-12))


def kb_shape(N, Ntilde):
    """Kaiser-Bessel shape b = pi (2 - 1/sigma_eff), sigma_eff = N~/N."""
    return np.pi * (2.0 - float(N) / float(Ntilde))


def psi(u, m, b, closed=False):
    """Truncated 1-D window in grid units u = N~ k - l.

    Support is [-m, m) (Eq. approxTrunc); with ``closed=True`` it is the
    closed interval [-m, m] of the (2m+1)-point variant discussed in
    Sec. 3.7.5.  Returns 0 outside the support.
    """
    u = np.asarray(u, dtype=np.float64)
    if closed:
        inside = (u >= -m) & (u <= m)
    else:
        inside = (u >= -m) & (u < m)
    s = np.sqrt(np.where(inside, np.maximum(m * m - u * u, 0.0), 1.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        val = np.sinh(b * s) / (np.pi * s)
    val = np.where(s == 0.0, b / np.pi, val)
    return np.where(inside, val, 0.0)


def psi_full(u, m, b):
    """The untruncated window in grid units (the phi-hat of Sec. 2.2 before
    Eq. approxTrunc): sinh(b s)/(pi s) with s = sqrt(m^2 - u^2) for |u| < m,
    b/pi at |u| = m, and sin(b s')/(pi s') with s' = sqrt(u^2 - m^2) beyond
    (the same analytic function continued past the support).  Used by the
    (2m+2)-point variant that Sec. 3.7.5 attributes to NFFT3."""
    u = np.asarray(u, dtype=np.float64)
    d = m * m - u * u
    s_in = np.sqrt(np.maximum(d, 0.0))
    s_out = np.sqrt(np.maximum(-d, 0.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        inner = np.sinh(b * s_in) / (np.pi * s_in)
        outer = np.sin(b * s_out) / (np.pi * s_out)
    val = np.where(d > 0, inner, outer)
    return np.where(d == 0.0, b / np.pi, val)


def dpsi_full(u, m, b):
    """d psi_full / du.  Inside: -u (z cosh z - sinh z)/(pi s^3) b^0 with
    z = b s; outside: u (z cos z - sin z)/(pi s'^3), z = b s'.  For small z
    both use the series b^3 h(z) with h = 1/3 + z^2/30 + ... inside and
    -1/3 + z^2/30 - ... outside (12 terms)."""
    u = np.asarray(u, dtype=np.float64)
    d = m * m - u * u
    inside = d >= 0
    s = np.sqrt(np.abs(d))
    z = b * s
    small = z < 0.5
    zs = np.where(small, z, 0.0)
    ser_in = np.zeros_like(zs)
    ser_out = np.zeros_like(zs)
    fact = 6.0
    for k in range(1, 13):
        if k > 1:
            fact *= (2 * k) * (2 * k + 1)
        term = (2.0 * k) / fact * zs ** (2 * k - 2)
        ser_in += term
        ser_out += term * (-1.0) ** k      # (z cos z - sin z)/z^3 = sum (-1)^k 2k z^(2k-2)/(2k+1)!
    zb = np.where(small, 1.0, z)
    dir_in = (zb * np.cosh(zb) - np.sinh(zb)) / zb ** 3
    dir_out = (zb * np.cos(zb) - np.sin(zb)) / zb ** 3
    h_in = np.where(small, ser_in, dir_in)
    h_out = np.where(small, ser_out, dir_out)
    return np.where(inside, -u * b ** 3 * h_in / np.pi, u * b ** 3 * h_out / np.pi)


def dpsi(u, m, b, closed=False):
    """Derivative d psi / d u inside the support (0 outside).

    d/du [sinh(b s)/(pi s)] with ds/du = -u/s gives
        -u (b s cosh(b s) - sinh(b s)) / (pi s^3).
    For small z = b s the bracket divided by s^3 is b^3 times
    h(z) = (z cosh z - sinh z)/z^3 = sum_{k>=1} 2k z^(2k-2)/(2k+1)!,
    which the oracle sums directly (12 terms) to avoid cancellation.
    """
    u = np.asarray(u, dtype=np.float64)
    if closed:
        inside = (u >= -m) & (u <= m)
    else:
        inside = (u >= -m) & (u < m)
    s = np.sqrt(np.where(inside, np.maximum(m * m - u * u, 0.0), 1.0))
    z = b * s
    small = z < 0.5
    zs = np.where(small, z, 0.0)
    series = np.zeros_like(zs)
    fact = 6.0  # (2k+1)! for k = 1
    for k in range(1, 13):
        if k > 1:
            fact *= (2 * k) * (2 * k + 1)
        series += (2.0 * k) / fact * zs ** (2 * k - 2)
    zb = np.where(small, 1.0, z)
    direct = (zb * np.cosh(zb) - np.sinh(zb)) / (zb ** 3)
    h = np.where(small, series, direct)
    val = -u * b ** 3 * h / np.pi
    return np.where(inside, val, 0.0)


def phi(n, Ntilde, m, b):
    """phi_d(n) = (1/N~) I0(m sqrt(b^2 - (2 pi n/N~)^2)) for |2 pi n/N~| <= b.

    Only the I0 branch is needed: for n in I_N, |2 pi n / N~| <= pi/sigma <= b.
    """
    n = np.asarray(n, dtype=np.float64)
    arg = b * b - (2.0 * np.pi * n / Ntilde) ** 2
    if np.any(arg < 0):
        raise ValueError("phi: frequency outside the I0 branch")
    return np.i0(m * np.sqrt(arg)) / Ntilde


def deconv_factor(n, Ntilde, m, b):
    """1 / (N~_d phi_d(n_d)) -- one factor of 1/(|I_N~| phi(n)) (Alg. 1 and
    Alg. 2 resampling correction; beta^tensor of Sec. 3.5)."""
    return 1.0 / (Ntilde * phi(n, Ntilde, m, b))


def lut_size(m):
    """LINEAR table size S = m 2^{c_min(m,8)} + 2 (Sec. 3.7.4); m > 8 keeps c_8."""
    if m < 1:
        raise ValueError("m >= 1")
    return m * 2 ** LUT_EXPONENTS[min(m, 8) - 1] + 2


def lut_entry(s, m, b):
    """Entry s of the LINEAR table of Sec. 3.7.4, psi_s = psi_Base(s/(S-2)):
    the window at u = m s / (S - 2) in grid units on its closed support
    [-m, m] (entry S - 2 is the edge value b/pi that the tap at u = -m reads
    through |u|), 0 beyond it (entry S - 1, outside the support)."""
    S = lut_size(m)
    s = np.asarray(s)
    return psi(m * s / (S - 2.0), m, b, closed=True)


def psi_linear(u, m, b, closed=False):
    """The window looked up in the LINEAR table with linear interpolation
    (Eq. linInterp, Sec. 3.7.4): kappa = |(S-2)/m u|, s = floor(kappa),
    alpha = kappa - s, value = psi_s + alpha (psi_{s+1} - psi_s), on the
    support of psi (0 outside it).  The table entries are evaluated where the
    lookup reads them (S reaches 1.3e8 at m = 8)."""
    u = np.asarray(u, dtype=np.float64)
    S = lut_size(m)
    kappa = np.abs(u) * ((S - 2.0) / m)
    s = np.floor(kappa)
    alpha = kappa - s
    lo = lut_entry(s, m, b)
    hi = lut_entry(s + 1, m, b)
    val = lo + alpha * (hi - lo)
    inside = (u >= -m) & ((u <= m) if closed else (u < m))
    return np.where(inside, val, 0.0)


def dpsi_linear(u, m, b, closed=False):
    """d psi_linear / du: the slope of the interpolant's segment,
    sign(u) (S-2)/m (psi_{s+1} - psi_s), 0 outside the support."""
    u = np.asarray(u, dtype=np.float64)
    S = lut_size(m)
    kappa = np.abs(u) * ((S - 2.0) / m)
    s = np.floor(kappa)
    slope = (lut_entry(s + 1, m, b) - lut_entry(s, m, b)) * ((S - 2.0) / m)
    inside = (u >= -m) & ((u <= m) if closed else (u < m))
    return np.where(inside, np.sign(u) * slope, 0.0)


def index_set(N):
    """I_N along one dimension: n = -floor(N/2), ..., ceil(N/2) - 1 (Sec. 2.1)."""
    return np.arange(N) - N // 2
