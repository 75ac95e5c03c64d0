"""Pins for oracle/nfft.py (no GPU).

* brute force: the operator A = B F D assembled entry by entry from its
  definitions (Sec. 2.2.3) on tiny grids, including the footprint set
  I_{N~,m}(k) checked against its set definition;
* the paper's error behaviour: exponential decay in m, saturation by m = 8
  for sigma = 2 (Sec. 5.1), and the NFFT close to the exact NDFT;
* invariants: adjointness of the NFFT operator itself, the exact grid-shift
  identity, periodicity in k, conjugate symmetry for real input;
* the node derivative by finite differences and against the exact NDFT
  derivative.
"""
import itertools

import numpy as np
import pytest

from oracle import ndft, nfft, window


def _cn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _grid_index_list(Nt):
    return list(itertools.product(*[window.index_set(n) for n in Nt]))


def _dense_operator(p, k):
    """A = B F D built from the matrix definitions of Sec. 2.2.3 by loops."""
    In = list(itertools.product(*[window.index_set(n) for n in p.N]))
    It = _grid_index_list(p.Nt)
    size_t = len(It)
    # D: generalised diagonal, 1/(|I_N~| phi(n)) at row l = n
    Dm = np.zeros((size_t, len(In)))
    pos = {l: r for r, l in enumerate(It)}
    for c, n in enumerate(In):
        val = 1.0
        for d in range(p.D):
            val *= 1.0 / (p.Nt[d] * window.phi(n[d], p.Nt[d], p.m, p.b[d]))
        Dm[pos[n], c] = val
    # F: exp(-2 pi i n.(l / N~)) over I_N~ x I_N~
    Fm = np.zeros((size_t, size_t), complex)
    for r, l in enumerate(It):
        for c, n in enumerate(It):
            Fm[r, c] = np.exp(-2j * np.pi * sum(n[d] * l[d] / p.Nt[d] for d in range(p.D)))
    # B: periodised truncated window psi~(k_j - l/N~) = sum_p psi(N~ (k - l/N~ + p));
    # the (2m+2)-point variant takes the untruncated window on the grid points
    # with -(m+1) <= N~ k - l' < m + 1 (the 2m + 2 nearest, Sec. 3.7.5)
    Bm = np.zeros((k.shape[0], size_t))
    for j in range(k.shape[0]):
        for c, l in enumerate(It):
            val = 1.0
            for d in range(p.D):
                acc = 0.0
                for per in (-1, 0, 1):
                    # u = N~ k - l + p N~, the form of the set definition (exact
                    # when N~ k is an integer, i.e. for on-grid nodes)
                    u = p.Nt[d] * k[j, d] - l[d] + per * p.Nt[d]
                    if p.wide:
                        if -(p.m + 1) <= u < p.m + 1:
                            acc += float(window.psi_full(u, p.m, p.b[d]))
                    else:
                        acc += float(window.psi(u, p.m, p.b[d], p.closed))
                val *= acc
            Bm[j, c] = val
    return Bm, Fm, Dm


@pytest.mark.parametrize("N,m,closed,wide", [((6,), 2, False, False), ((4, 5), 1, False, False),
                                             ((6, 4), 2, True, False), ((6,), 2, False, True),
                                             ((5, 6), 1, False, True), ((7,), 3, False, True)])
def test_operator_against_dense_definition(N, m, closed, wide):
    rng = np.random.default_rng(10)
    p = nfft.Params(N, 2.0, m, closed, wide)
    k = rng.random((5, len(N))) - 0.5
    if closed or wide:
        k[0] = [int(np.floor(0.3 * nt)) / nt for nt in p.Nt]   # an on-grid node
    Bm, Fm, Dm = _dense_operator(p, k)
    f = _cn(rng, N)
    w = _cn(rng, 5)
    In = list(itertools.product(*[range(n) for n in N]))
    fv = np.array([f[i] for i in In])
    want = Bm @ (Fm @ (Dm @ fv))
    got = nfft.forward(k, f, 2.0, m, closed, wide)
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    want_a = Dm.T @ (Fm.conj().T @ (Bm.T @ w))
    got_a = nfft.adjoint(k, w, N, 2.0, m, closed, wide)
    got_av = np.array([got_a[i] for i in In])
    assert np.allclose(got_av, want_a, rtol=0, atol=1e-12 * np.abs(want_a).max())


def test_footprint_matches_set_definition():
    """I_{N~,m}(k) = {l in I_N~ : exists p, -m <= N~k - l + p N~ < m}."""
    rng = np.random.default_rng(11)
    for Nt, m in [(16, 2), (20, 4), (12, 3)]:
        p = nfft.Params((Nt // 2,), 2.0, m)
        assert p.Nt == (Nt,)
        k = np.concatenate([rng.random(40) - 0.5, np.arange(-Nt // 2, Nt // 2) / Nt])[:, None]
        ls, us = nfft.footprint(p, k)
        for j in range(k.shape[0]):
            enum = {int(np.mod(v, Nt)) for v in ls[0][j]}
            defn = set()
            for l in window.index_set(Nt):
                for per in (-1, 0, 1):
                    x = Nt * k[j, 0] - l + per * Nt
                    if -m <= x < m:
                        defn.add(int(np.mod(l, Nt)))
            assert enum == defn and len(enum) == 2 * m


@pytest.mark.parametrize("N", [(128,), (24, 20), (10, 12, 8)])
def test_close_to_ndft_and_decay_in_m(N):
    """Sec. 5.1: the error decays exponentially in m and saturates by m = 8
    (sigma = 2); at m = 4 it is far below 1e-5."""
    rng = np.random.default_rng(12)
    M = 300
    k = rng.random((M, len(N))) - 0.5
    f = _cn(rng, N)
    w = _cn(rng, M)
    ex = ndft.ndft(k, f)
    exa = ndft.ndft_adjoint(k, w, N)
    errs, errs_a = [], []
    for m in range(2, 9):
        if 2 * m >= 2 * min(N):
            break
        errs.append(np.linalg.norm(nfft.forward(k, f, 2.0, m) - ex) / np.linalg.norm(ex))
        errs_a.append(np.linalg.norm(nfft.adjoint(k, w, N, 2.0, m) - exa) / np.linalg.norm(exa))
    for e in (errs, errs_a):
        assert e[2] < 1e-6                           # m = 4
        for a, b in zip(e[:4], e[1:5]):              # m = 2..6: each step gains > 10x
            assert b < a / 10
        if len(e) == 7:
            assert e[-1] < 1e-13                     # m = 8: saturated near machine precision


def test_adjointness_of_nfft_operator():
    """<A f, w> = <f, A^H w> for the approximate operator B F D itself."""
    rng = np.random.default_rng(13)
    for N, m in [((64,), 4), ((20, 18), 3), ((8, 10, 6), 2)]:
        k = rng.random((150, len(N))) - 0.5
        f = _cn(rng, N)
        w = _cn(rng, 150)
        lhs = np.vdot(w, nfft.forward(k, f, 2.0, m))
        rhs = np.vdot(nfft.adjoint(k, w, N, 2.0, m), f)
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(f) * np.linalg.norm(w) * 10


def test_grid_shift_identity():
    """Shifting every node by one grid cell along d multiplies f by
    exp(-2 pi i n_d / N~_d) exactly (pins the wrap, the index map and the
    FFT sign)."""
    rng = np.random.default_rng(14)
    N = (16, 12)
    p = nfft.Params(N, 2.0, 3)
    k = rng.random((80, 2)) - 0.5
    f = _cn(rng, N)
    for d in range(2):
        e = np.zeros(2)
        e[d] = 1.0 / p.Nt[d]
        shape = [1, 1]
        shape[d] = N[d]
        ph = np.exp(-2j * np.pi * window.index_set(N[d]).reshape(shape) / p.Nt[d])
        a = nfft.forward(k + e, f, 2.0, 3)
        b = nfft.forward(k, f * ph, 2.0, 3)
        assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())


def test_periodicity_and_conjugate_symmetry():
    rng = np.random.default_rng(15)
    N = (20, 16)
    k = rng.random((60, 2)) - 0.5
    f = _cn(rng, N)
    a = nfft.forward(k, f, 2.0, 4)
    b = nfft.forward(k + np.array([1.0, -1.0]), f, 2.0, 4)
    assert np.allclose(a, b, rtol=0, atol=1e-11 * np.abs(a).max())
    fr = rng.standard_normal(N)
    plus = nfft.forward(k, fr, 2.0, 4)
    minus = nfft.forward(np.mod(-k + 0.5, 1.0) - 0.5, fr, 2.0, 4)
    assert np.allclose(minus, np.conj(plus), rtol=0, atol=1e-11 * np.abs(plus).max())


def test_closed_support_differs_only_on_grid():
    rng = np.random.default_rng(16)
    N = (16,)
    f = _cn(rng, N)
    k_off = rng.random((30, 1)) - 0.5
    assert np.allclose(nfft.forward(k_off, f, 2.0, 3, closed=True), nfft.forward(k_off, f, 2.0, 3), atol=1e-13)
    k_on = (np.arange(-4, 4) / 32.0)[:, None]
    d = nfft.forward(k_on, f, 2.0, 3, closed=True) - nfft.forward(k_on, f, 2.0, 3)
    assert np.min(np.abs(d)) > 0


def test_node_derivative_by_finite_differences():
    rng = np.random.default_rng(17)
    N = (16, 12)
    m = 4
    p = nfft.Params(N, 2.0, m)
    f = _cn(rng, N)
    k = rng.random((40, 2)) - 0.5
    ghat = nfft.fft_forward(nfft.correction_pad(p, f))
    dk = nfft.resample_node_derivative(p, k, ghat)
    h = 1e-7
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fd = (nfft.resample(p, k + e, ghat) - nfft.resample(p, k - e, ghat)) / (2 * h)
        assert np.allclose(dk[:, d], fd, rtol=0, atol=2e-6 * np.abs(fd).max())


def test_node_grad_close_to_exact_ndft_gradient():
    rng = np.random.default_rng(18)
    N = (20, 16)
    f = _cn(rng, N)
    k = rng.random((50, 2)) - 0.5
    cot = _cn(rng, 50)
    g = nfft.node_grad(k, f, cot, 2.0, 8)
    ge = ndft.ndft_node_grad(k, f, cot)
    assert np.linalg.norm(g - ge) <= 1e-10 * np.linalg.norm(ge)


@pytest.mark.parametrize("N,sigma,m", [((16, 16, 16), 1.25, 6), ((64, 64), 1.25, 6), ((20, 18, 16), 2.0, 4),
                                       ((12, 10, 14), 2.0, 8), ((33, 47), 1.5, 5)])
def test_fp32_rounding_bound(N, sigma, m):
    """The complex64 parity tolerance max(1e-5, u32 * kappa) bounds the error
    of the plain algorithm when its deconvolved grid (scaled to O(1) by the
    window peak, as single precision requires) and its FFT are rounded to
    single precision; kappa is the deconvolution's amplification."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from gpu_helpers import tol_for
    rng = np.random.default_rng(21)
    M = 3000
    k = rng.random((M, len(N))) - 0.5
    f = _cn(rng, N)
    p = nfft.Params(N, sigma, m)
    peak = np.prod([float(window.psi(0.0, m, b)) for b in p.b])
    g = nfft.correction_pad(p, f) * peak
    ref = nfft.resample(p, k, nfft.fft_forward(g))
    g32 = np.fft.fftn(g.astype(np.complex64))
    assert g32.dtype == np.complex64
    err = np.linalg.norm(nfft.resample(p, k, g32.astype(np.complex128)) - ref) / np.linalg.norm(ref)
    assert err <= tol_for(N, sigma, m, "c64") / 4


def test_wide_footprint_against_paper_claims():
    """Sec. 5.1 / Sec. 6: NFFT3's (2m+2)-point footprint with the untruncated
    window is more accurate than 2m points at the same m, but increasing m by
    one (2(m+1) points) gains much more."""
    rng = np.random.default_rng(22)
    N = (24, 20)
    M = 300
    k = rng.random((M, 2)) - 0.5
    f = _cn(rng, N)
    ex = ndft.ndft(k, f)
    err = lambda fh: np.linalg.norm(fh - ex) / np.linalg.norm(ex)
    for m in (2, 3, 4, 5):
        e2m = err(nfft.forward(k, f, 2.0, m))
        ewide = err(nfft.forward(k, f, 2.0, m, wide=True))
        enext = err(nfft.forward(k, f, 2.0, m + 1))
        assert ewide < e2m
        assert enext < ewide


def test_wide_footprint_invariants():
    rng = np.random.default_rng(23)
    N = (16, 12)
    k = rng.random((80, 2)) - 0.5
    f = _cn(rng, N)
    w = _cn(rng, 80)
    lhs = np.vdot(w, nfft.forward(k, f, 2.0, 3, wide=True))
    rhs = np.vdot(nfft.adjoint(k, w, N, 2.0, 3, wide=True), f)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(f) * np.linalg.norm(w)
    p = nfft.Params(N, 2.0, 3, wide=True)
    e = np.array([0.0, 1.0 / p.Nt[1]])
    ph = np.exp(-2j * np.pi * window.index_set(N[1]).reshape(1, -1) / p.Nt[1])
    a = nfft.forward(k + e, f, 2.0, 3, wide=True)
    b = nfft.forward(k, f * ph, 2.0, 3, wide=True)
    assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(b).max())
    # node derivative of the wide form by finite differences
    ghat = nfft.fft_forward(nfft.correction_pad(p, f))
    dk = nfft.resample_node_derivative(p, k, ghat)
    h = 1e-7
    for d in range(2):
        ee = np.zeros(2)
        ee[d] = h
        fd = (nfft.resample(p, k + ee, ghat) - nfft.resample(p, k - ee, ghat)) / (2 * h)
        assert np.allclose(dk[:, d], fd, rtol=0, atol=2e-6 * np.abs(fd).max())


@pytest.mark.parametrize("N", [(8,), (6, 10), (4, 6, 8)])
def test_fftshift_as_phase_when_oversampling_by_two(N):
    """The pruned FFT's reading of the index map (Sec. 3.5) for N~ = 2N: the
    oracle's correction + zero pad (f_n stored at n mod N~) followed by the
    forward FFT equals storing the corrected f at array index n + N/2 (a plain
    zero pad) and multiplying the DFT output at l by i^l per dimension; the
    adjoint FFT followed by crop + correction equals multiplying the grid by
    (-i)^l, the inverse DFT, and reading index n + N/2."""
    rng = np.random.default_rng(31)
    p = nfft.Params(N, 2.0, 2)
    assert p.Nt == tuple(2 * n for n in N)
    f = _cn(rng, N)
    g = nfft.correction_pad(p, f)
    want = nfft.fft_forward(g)
    # the same corrected values, stored at index n + N/2 (no wrap)
    corrected = g[np.ix_(*[np.mod(window.index_set(n), nt) for n, nt in zip(N, p.Nt)])]
    shifted = np.zeros(p.Nt, complex)
    shifted[tuple(slice(0, n) for n in N)] = corrected
    phase = np.ones(p.Nt, complex)
    for d, nt in enumerate(p.Nt):
        shape = [1] * len(N)
        shape[d] = nt
        phase = phase * (1j ** np.arange(nt)).reshape(shape)
    got = np.fft.fftn(shifted) * phase
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # adjoint: (-i)^l on the grid, unnormalised inverse DFT, read index n + N/2
    gh = _cn(rng, p.Nt)
    want_y = nfft.crop_correction(p, nfft.fft_adjoint(gh))
    y = np.fft.ifftn(gh * np.conj(phase), norm="forward")[tuple(slice(0, n) for n in N)]
    corr = nfft.crop_correction(p, np.ones(p.Nt, complex))  # the correction factors alone
    assert np.allclose(y * corr, want_y, rtol=0, atol=1e-12 * np.abs(want_y).max())
