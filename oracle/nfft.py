"""Plain FP64 NFFT, step by step (TEST INFRASTRUCTURE ONLY).

arXiv 2208.00049, Sec. 2.2:
  Algorithm 1 (direct NFFT)
    1. resampling correction + zero pad: g_n = f_n / (|I_N~| phi(n)) for
       n in I_N, 0 on I_N~ \\ I_N;
    2. FFT on the oversampled grid: ghat_l = sum_n g_n exp(-2 pi i n.l/N~);
    3. resampling: fhat_j = sum_{l in I_{N~,m}(k_j)} ghat_l psi~(k_j - l/N~).
  Algorithm 2 (adjoint NFFT)
    1. adjoint resampling: ghat_l = sum_{j : l in I_{N~,m}(k_j)} fhat_j psi~(k_j - l/N~);
    2. adjoint FFT: g_n = sum_l ghat_l exp(+2 pi i n.l/N~);
    3. resampling correction + crop: y_n = g_n / (|I_N~| phi(n)), n in I_N.

Storage: a grid index l in I_N~ lives at position (l mod N~) of an
(N~_1, ..., N~_D) array, which is the natural order of numpy.fft (the
fftshift of Sec. 3.5 folded into the index map).  numpy.fft.fftn is the
unnormalised exp(-2 pi i) transform of the FFT step of Algorithm 1;
numpy.fft.ifftn with norm="forward" is the unnormalised exp(+2 pi i)
transform of the adjoint FFT step of Algorithm 2.

Footprint I_{N~,m}(k) (Sec. 2.2, definition after Eq. approxNFFT2): the grid
indices l with -m <= N~ k - l + p N~ < m for some integer p.  For the
unwrapped integer l' = l - p N~ that is N~k - m < l' <= N~k + m, i.e.
l' = floor(N~ k) - m + 1 + i for i = 0, ..., 2m - 1 (2m points per
dimension; Sec. 3.7.5).  The printed closed form omega is read as this set
(it is off by N~/2 as printed); the tests also check this enumeration against
the set definition by brute force.  With ``closed=True`` the support is
[-m, m] and the footprint has 2m + 1 points l' = floor(N~k) - m + i,
i = 0, ..., 2m (the (2m+1)^D variant).  With ``wide=True`` the footprint has
2m + 2 points l' = floor(N~k) - m + i, i = 0, ..., 2m + 1, weighted with the
untruncated window (the NFFT3 variant of Sec. 3.7.5).  With
``window="linear"`` the window values come from the LINEAR table of Sec. 3.7.4
(lookup with linear interpolation) instead of being evaluated.

N~ k is formed in FP64 and its floor taken in FP64.
"""
import itertools

import numpy as np

from .window import (deconv_factor, dpsi, dpsi_full, dpsi_linear, index_set, kb_shape,
                     oversampled_size, psi, psi_full, psi_linear)


class Params:
    """Sizes and window shape of one transform (plan-time quantities)."""

    def __init__(self, N, sigma=2.0, m=4, closed=False, wide=False, window="direct"):
        self.N = tuple(int(v) for v in N)
        self.D = len(self.N)
        self.sigma = float(sigma)
        self.m = int(m)
        self.closed = bool(closed)
        self.wide = bool(wide)
        if self.closed and self.wide:
            raise ValueError("closed and wide are exclusive")
        # "direct": the window evaluated; "linear": looked up in the LINEAR
        # table with linear interpolation (Sec. 3.7.4; needs |u| <= m, so not
        # with the (2m+2)-point footprint)
        if window not in ("direct", "linear") or (window == "linear" and self.wide):
            raise ValueError("window must be 'direct' or 'linear' (not with wide)")
        self.window_mode = window
        self.Nt = tuple(oversampled_size(n, sigma) for n in self.N)
        self.b = tuple(kb_shape(n, nt) for n, nt in zip(self.N, self.Nt))
        for n, nt in zip(self.N, self.Nt):
            if not (2 * self.m < nt):
                raise ValueError("need 2m < N~")

    def taps(self):
        if self.wide:
            return 2 * self.m + 2
        return 2 * self.m + 1 if self.closed else 2 * self.m

    def window(self, u, b):
        if self.window_mode == "linear":
            return psi_linear(u, self.m, b, self.closed)
        return psi_full(u, self.m, b) if self.wide else psi(u, self.m, b, self.closed)

    def dwindow(self, u, b):
        if self.window_mode == "linear":
            return dpsi_linear(u, self.m, b, self.closed)
        return dpsi_full(u, self.m, b) if self.wide else dpsi(u, self.m, b, self.closed)


def _correction(p):
    """Per-dimension vectors 1/(N~_d phi_d(n_d)) over I_{N_d} (Sec. 3.5)."""
    return [deconv_factor(index_set(n), nt, p.m, b)
            for n, nt, b in zip(p.N, p.Nt, p.b)]


def _outer(vecs):
    out = vecs[0]
    for v in vecs[1:]:
        out = np.multiply.outer(out, v)
    return out


def _positions(p):
    """Grid positions (n mod N~_d) of every n in I_{N_d}, per dimension."""
    return [np.mod(index_set(n), nt) for n, nt in zip(p.N, p.Nt)]


def correction_pad(p, f):
    """Algorithm 1, correction and zero-pad step: g on I_N~ with
    g_n = f_n/(|I_N~| phi(n)) on I_N, else 0."""
    f = np.asarray(f, dtype=np.complex128)
    if f.shape != p.N:
        raise ValueError("f has the wrong shape")
    g = np.zeros(p.Nt, dtype=np.complex128)
    g[np.ix_(*_positions(p))] = f * _outer(_correction(p))
    return g


def crop_correction(p, g):
    """Algorithm 2, crop and correction step: y_n = g_n/(|I_N~| phi(n)) for n in I_N."""
    return g[np.ix_(*_positions(p))] * _outer(_correction(p))


def footprint(p, k):
    """For each dimension: the unwrapped footprint indices l' (M, taps) and
    u = N~ k - l' (M, taps), with N~ k and its floor in FP64."""
    k = np.asarray(k, dtype=np.float64)
    ls, us = [], []
    first = -p.m if (p.closed or p.wide) else -p.m + 1
    offs = np.arange(p.taps()) + first
    for d in range(p.D):
        x = p.Nt[d] * k[:, d]
        c = np.floor(x)
        lprime = c[:, None] + offs[None, :]
        ls.append(lprime.astype(np.int64))
        us.append(x[:, None] - lprime)
    return ls, us


def resample(p, k, ghat):
    """Algorithm 1, resampling step (Eq. SumOverNode):
    fhat_j = sum_l ghat_l psi~(k_j - l/N~)."""
    ls, us = footprint(p, k)
    w = [p.window(u, b) for u, b in zip(us, p.b)]
    M = ls[0].shape[0]
    out = np.zeros(M, dtype=np.complex128)
    for tap in itertools.product(range(p.taps()), repeat=p.D):
        idx = tuple(np.mod(ls[d][:, tap[d]], p.Nt[d]) for d in range(p.D))
        wt = np.ones(M)
        for d in range(p.D):
            wt = wt * w[d][:, tap[d]]
        out += ghat[idx] * wt
    return out


def resample_adjoint(p, k, fhat):
    """Algorithm 2, adjoint resampling step (Eq. SumOverNodeAdjoint), evaluated node by node as
    Sec. 2.2.2 describes: every node adds fhat_j psi~ into its footprint."""
    fhat = np.asarray(fhat, dtype=np.complex128).ravel()
    ls, us = footprint(p, k)
    w = [p.window(u, b) for u, b in zip(us, p.b)]
    M = fhat.shape[0]
    acc = np.zeros(int(np.prod(p.Nt)), dtype=np.complex128)
    for tap in itertools.product(range(p.taps()), repeat=p.D):
        idx = tuple(np.mod(ls[d][:, tap[d]], p.Nt[d]) for d in range(p.D))
        flat = np.ravel_multi_index(idx, p.Nt)
        wt = np.ones(M)
        for d in range(p.D):
            wt = wt * w[d][:, tap[d]]
        np.add.at(acc, flat, fhat * wt)
    return acc.reshape(p.Nt)


def fft_forward(g):
    """Algorithm 1, FFT step: unnormalised exp(-2 pi i) DFT on the oversampled grid."""
    return np.fft.fftn(g)


def fft_adjoint(ghat):
    """Algorithm 2, inverse FFT step: unnormalised exp(+2 pi i) DFT on the oversampled grid."""
    return np.fft.ifftn(ghat, norm="forward")


def forward(k, f, sigma=2.0, m=4, closed=False, wide=False, window="direct"):
    """Direct NFFT, Algorithm 1: fhat ~= A f."""
    f = np.asarray(f, dtype=np.complex128)
    p = Params(f.shape, sigma, m, closed, wide, window)
    g = correction_pad(p, f)
    ghat = fft_forward(g)
    return resample(p, k, ghat)


def adjoint(k, fhat, N, sigma=2.0, m=4, closed=False, wide=False, window="direct"):
    """Adjoint NFFT, Algorithm 2: y ~= A^H fhat."""
    p = Params(N, sigma, m, closed, wide, window)
    ghat = resample_adjoint(p, k, fhat)
    g = fft_adjoint(ghat)
    return crop_correction(p, g)


def resample_node_derivative(p, k, ghat):
    """d/dk_{j,d} of the resampling step of Algorithm 1: sum_l ghat_l N~_d psi'(u_d) prod_{e != d} psi(u_e).

    Differentiates Eq. SumOverNode through u_d = N~_d k_{j,d} - l_d with the
    footprint held fixed (the window vanishes at the footprint's open end).
    Returns a complex (M, D) array.
    """
    ls, us = footprint(p, k)
    w = [p.window(u, b) for u, b in zip(us, p.b)]
    dw = [p.dwindow(u, b) for u, b in zip(us, p.b)]
    M = ls[0].shape[0]
    out = np.zeros((M, p.D), dtype=np.complex128)
    for tap in itertools.product(range(p.taps()), repeat=p.D):
        idx = tuple(np.mod(ls[d][:, tap[d]], p.Nt[d]) for d in range(p.D))
        val = ghat[idx]
        for d in range(p.D):
            wt = p.Nt[d] * dw[d][:, tap[d]]
            for e in range(p.D):
                if e != d:
                    wt = wt * w[e][:, tap[e]]
            out[:, d] += val * wt
    return out


def node_grad(k, f, cot, sigma=2.0, m=4, closed=False, wide=False, window="direct"):
    """Node gradient of a real loss through the NFFT fhat = A f:
    g[j, d] = Re(conj(cot_j) d fhat_j / d k_{j,d}) (PyTorch's convention for a
    real loss of complex outputs)."""
    f = np.asarray(f, dtype=np.complex128)
    p = Params(f.shape, sigma, m, closed, wide, window)
    ghat = fft_forward(correction_pad(p, f))
    dk = resample_node_derivative(p, k, ghat)
    return np.real(np.conj(np.asarray(cot, dtype=np.complex128))[:, None] * dk)
