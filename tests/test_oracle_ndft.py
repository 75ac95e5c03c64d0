"""Pins for oracle/ndft.py (no GPU): reductions to numpy's FFT, closed forms,
brute-force loops and finite differences."""
import cmath
import itertools

import numpy as np
import pytest

from oracle import ndft


def _rng(seed=0):
    return np.random.default_rng(seed)


def _cnormal(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("N", [(16,), (15,), (8, 6), (4, 5, 6)])
def test_equispaced_nodes_reduce_to_fft(N):
    """With nodes on the N-point grid, k_j = j/N (wrapped), the NDFT is the DFT
    of the fftshift-ordered signal: fhat = fft(ifftshift(f))."""
    rng = _rng(1)
    f = _cnormal(rng, N)
    axes = [np.arange(n) / n for n in N]
    mesh = np.meshgrid(*axes, indexing="ij")
    k = np.stack([a.ravel() for a in mesh], axis=1)
    k = np.mod(k + 0.5, 1.0) - 0.5
    got = ndft.ndft(k, f)
    want = np.fft.fftn(np.fft.ifftshift(f)).ravel()
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # adjoint on the same nodes = unnormalised inverse DFT, shifted back
    w = _cnormal(rng, k.shape[0])
    got_a = ndft.ndft_adjoint(k, w, N)
    want_a = np.fft.fftshift(np.fft.ifftn(w.reshape(N), norm="forward"))
    assert np.allclose(got_a, want_a, rtol=0, atol=1e-12 * np.abs(want_a).max())


def test_delta_closed_form():
    """f = delta at n0 gives fhat_j = exp(-2 pi i n0.k_j)."""
    rng = _rng(2)
    N = (8, 10)
    n0 = (-3, 4)
    f = np.zeros(N, complex)
    f[n0[0] + N[0] // 2, n0[1] + N[1] // 2] = 1.0
    k = rng.random((50, 2)) - 0.5
    want = np.exp(-2j * np.pi * (k @ np.array(n0, float)))
    assert np.allclose(ndft.ndft(k, f), want, atol=1e-14)


def test_single_node_adjoint_closed_form():
    """One node: y_n = fhat exp(+2 pi i n.k)."""
    N = (6, 7)
    k = np.array([[0.1234, -0.377]])
    c = 0.3 - 1.7j
    y = ndft.ndft_adjoint(k, np.array([c]), N)
    for i0, i1 in itertools.product(range(N[0]), range(N[1])):
        n = (i0 - N[0] // 2, i1 - N[1] // 2)
        assert y[i0, i1] == pytest.approx(c * cmath.exp(2j * cmath.pi * (n[0] * k[0, 0] + n[1] * k[0, 1])), abs=1e-14)


def test_brute_force_loops():
    """Both transforms against pure-Python double loops on a tiny 2D case."""
    rng = _rng(3)
    N = (5, 4)
    M = 7
    f = _cnormal(rng, N)
    w = _cnormal(rng, M)
    k = rng.random((M, 2)) - 0.5
    fh = ndft.ndft(k, f)
    y = ndft.ndft_adjoint(k, w, N)
    for j in range(M):
        acc = 0j
        for i0, i1 in itertools.product(range(N[0]), range(N[1])):
            n0, n1 = i0 - N[0] // 2, i1 - N[1] // 2
            acc += f[i0, i1] * cmath.exp(-2j * cmath.pi * (n0 * k[j, 0] + n1 * k[j, 1]))
        assert fh[j] == pytest.approx(acc, abs=1e-13)
    for i0, i1 in itertools.product(range(N[0]), range(N[1])):
        n0, n1 = i0 - N[0] // 2, i1 - N[1] // 2
        acc = sum(w[j] * cmath.exp(2j * cmath.pi * (n0 * k[j, 0] + n1 * k[j, 1])) for j in range(M))
        assert y[i0, i1] == pytest.approx(acc, abs=1e-13)


def test_node_derivative_by_finite_differences():
    rng = _rng(4)
    N = (12, 10)
    f = _cnormal(rng, N)
    k = rng.random((9, 2)) - 0.5
    dk = ndft.ndft_node_derivative(k, f)
    h = 1e-6
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fd = (ndft.ndft(k + e, f) - ndft.ndft(k - e, f)) / (2 * h)
        assert np.allclose(dk[:, d], fd, rtol=0, atol=1e-6 * np.abs(fd).max())


def test_node_grad_convention():
    """Re(conj(cot) dfhat/dk) is the derivative of the real loss Re<cot, fhat>."""
    rng = _rng(5)
    N = (16,)
    f = _cnormal(rng, N)
    cot = _cnormal(rng, 6)
    k = rng.random((6, 1)) - 0.5
    g = ndft.ndft_node_grad(k, f, cot)
    h = 1e-6
    for j in range(6):
        kp, km = k.copy(), k.copy()
        kp[j, 0] += h
        km[j, 0] -= h
        lp = np.real(np.vdot(cot, ndft.ndft(kp, f)))
        lm = np.real(np.vdot(cot, ndft.ndft(km, f)))
        assert g[j, 0] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-8)


def test_adjoint_at_selected_outputs():
    """ndft_adjoint_at equals the full adjoint at the selected outputs (odd and
    even N), and reduces to the single-node closed form y_n = fhat e^{2 pi i n.k}."""
    rng = np.random.default_rng(17)
    for N in [(7, 6), (5, 4, 3)]:
        M = 40
        k = rng.random((M, len(N))) - 0.5
        w = rng.standard_normal(M) + 1j * rng.standard_normal(M)
        full = ndft.ndft_adjoint(k, w, N)
        flat = rng.choice(int(np.prod(N)), 9, replace=False)
        idx = np.unravel_index(flat, N)
        assert np.allclose(ndft.ndft_adjoint_at(k, w, N, idx), full[idx], rtol=0, atol=1e-12)
    k1 = np.array([[0.3, -0.15]])
    idx = (np.array([0, 3]), np.array([5, 1]))
    n = np.stack([idx[0] - 4, idx[1] - 3], axis=1)
    want = 2.0 * np.exp(2j * np.pi * (n @ k1[0]))
    assert np.allclose(ndft.ndft_adjoint_at(k1, np.array([2.0]), (8, 7), idx), want, rtol=0, atol=1e-13)

