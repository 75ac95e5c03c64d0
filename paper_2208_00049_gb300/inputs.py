"""Seeded synthetic workloads shared by the tests, the bench and the oracle legs.

This module holds random-number draws and array shapes only -- none of the
transform's arithmetic -- so that the CUDA path and the CPU oracle can be fed
identical inputs without sharing code.  Every generator is numpy PCG64 with a
fixed seed (2208 + workload number).

Workloads (shapes of the paper's benchmarks, Sec. 4: random nodes with
M = |I_N|, sigma = 2, Kaiser-Bessel; plus the radial and batched sets):
  1  1D   N = 256,        M = 1024 uniform nodes, complex128, sigma 2, m 4
  2  2D   N = 256 x 256,  M = 65536 uniform nodes, complex64 m 4 / complex128 m 8
  3  3D   N = 128^3,      M = 2097152 uniform nodes, complex64, sigma 2 m 4
          (lean variant sigma 1.25, m 6)
  4  batched 2D: 64 problems, N_d drawn from {64,128,256,512},
          M = floor(N1 N2 U(0.5, 2)); plus 32 right-hand sides on one
          256 x 256 radial set (402 spokes x 512 samples)
  5  differentiation: 256 x 256, radial set with angle jitter N(0, 1e-3),
          f and y complex iid N(0, 1)
Nodes are always generated in FP64 in [-1/2, 1/2)^D.
"""
import numpy as np

SEED_BASE = 2208


def rng_for(workload, salt=0):
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(workload) + 1000 * int(salt)))


def uniform_nodes(rng, M, D):
    """M nodes iid uniform in [-1/2, 1/2)^D, FP64, shape (M, D)."""
    return rng.random((int(M), int(D))) - 0.5


def complex_normal(rng, shape, dtype=np.complex128):
    """Real and imaginary parts iid N(0, 1)."""
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(dtype)


def wrap_half(k):
    """Wrap coordinates into [-1/2, 1/2)."""
    return np.mod(k + 0.5, 1.0) - 0.5


def radial_nodes(n_spokes=402, n_samples=512, jitter=0.0, rng=None):
    """2D radial set: theta_s = pi s / n_spokes, r_i = (i - n_samples/2)/n_samples,
    k = r (cos theta, sin theta), wrapped into [-1/2, 1/2)^2.  With jitter > 0
    every spoke angle gets an iid N(0, jitter) perturbation."""
    theta = np.pi * np.arange(n_spokes) / n_spokes
    if jitter > 0.0:
        theta = theta + rng.normal(0.0, jitter, size=theta.shape)
    r = (np.arange(n_samples) - n_samples // 2) / float(n_samples)
    kx = np.cos(theta)[:, None] * r[None, :]
    ky = np.sin(theta)[:, None] * r[None, :]
    k = np.stack([kx.ravel(), ky.ravel()], axis=1)
    return wrap_half(k)


def workload(name, rng_salt=0):
    """Return a dict describing one named workload with its seeded inputs.

    Keys: N (tuple), M, sigma, m, dtype ('c64'|'c128'), k (M, D) float64,
    f (complex128 array of shape N) and w (complex128 (M,), an adjoint input).
    """
    spec = {
        "1d": dict(wl=1, N=(256,), M=1024, sigma=2.0, m=4, dtype="c128"),
        "2d_c64": dict(wl=2, N=(256, 256), M=65536, sigma=2.0, m=4, dtype="c64"),
        "2d_c128": dict(wl=2, N=(256, 256), M=65536, sigma=2.0, m=8, dtype="c128"),
        "3d": dict(wl=3, N=(128, 128, 128), M=2097152, sigma=2.0, m=4, dtype="c64"),
        "3d_lean": dict(wl=3, N=(128, 128, 128), M=2097152, sigma=1.25, m=6, dtype="c64"),
    }
    if name not in spec:
        raise KeyError(name)
    s = dict(spec[name])
    rng = rng_for(s["wl"], rng_salt)
    D = len(s["N"])
    s["k"] = uniform_nodes(rng, s["M"], D)
    s["f"] = complex_normal(rng, s["N"])
    s["w"] = complex_normal(rng, (s["M"],))
    s["name"] = name
    return s


def small_case(N, M, seed, sigma=2.0, m=4):
    """A small random case (for parity tests that span several tiles)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D = len(N)
    return dict(N=tuple(N), M=int(M), sigma=sigma, m=m,
                k=uniform_nodes(rng, M, D), f=complex_normal(rng, tuple(N)),
                w=complex_normal(rng, (int(M),)))


def batched_problems(n_problems=64, sizes=(64, 128, 256, 512), salt=0):
    """Workload 4a: independent 2D problems with uneven N and M."""
    rng = rng_for(4, salt)
    probs = []
    for _ in range(n_problems):
        N = (int(rng.choice(sizes)), int(rng.choice(sizes)))
        M = int(np.floor(N[0] * N[1] * rng.uniform(0.5, 2.0)))
        probs.append(dict(N=N, M=M, k=uniform_nodes(rng, M, 2),
                          f=complex_normal(rng, N), w=complex_normal(rng, (M,))))
    return probs


def radial_rhs(n_rhs=32, N=(256, 256), salt=0):
    """Workload 4b: n_rhs coefficient arrays sharing one radial node set."""
    rng = rng_for(4, 7 + salt)
    k = radial_nodes()
    f = np.stack([complex_normal(rng, N) for _ in range(n_rhs)])
    w = np.stack([complex_normal(rng, (k.shape[0],)) for _ in range(n_rhs)])
    return dict(N=tuple(N), k=k, f=f, w=w)


def differentiation(salt=0):
    """Workload 5: jittered radial set, f and target y (iid complex normal)."""
    rng = rng_for(5, salt)
    k = radial_nodes(jitter=1e-3, rng=rng)
    N = (256, 256)
    f = complex_normal(rng, N)
    y = complex_normal(rng, (k.shape[0],))
    return dict(N=N, M=k.shape[0], k=k, f=f, y=y, sigma=2.0, m=4)
