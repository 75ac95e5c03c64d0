"""The seeded synthetic input recipe (paper_2208_00049_gb300/inputs.py) that
the parity tests, the bench and the oracle legs share: shapes, ranges,
distributions and structure of each workload, and determinism."""
import numpy as np
import pytest

from paper_2208_00049_gb300 import inputs


@pytest.mark.parametrize("name,N,M,sigma,m,dtype", [
    ("1d", (256,), 1024, 2.0, 4, "c128"),
    ("2d_c64", (256, 256), 65536, 2.0, 4, "c64"),
    ("2d_c128", (256, 256), 65536, 2.0, 8, "c128"),
])
def test_single_problem_workloads(name, N, M, sigma, m, dtype):
    wl = inputs.workload(name)
    assert wl["N"] == N and wl["M"] == M and wl["sigma"] == sigma and wl["m"] == m
    assert wl["dtype"] == dtype
    k = wl["k"]
    assert k.shape == (M, len(N)) and k.dtype == np.float64
    assert k.min() >= -0.5 and k.max() < 0.5
    # uniform in [-1/2, 1/2): mean 0, variance 1/12 per coordinate (the
    # variance estimate's standard error is sqrt(1/180 / n))
    assert abs(k.mean()) < 5 / np.sqrt(12 * k.size)
    assert abs(k.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / k.size)
    assert wl["f"].shape == N and wl["w"].shape == (M,)
    for z in (wl["f"], wl["w"]):
        assert np.iscomplexobj(z)
        # real and imaginary parts iid N(0, 1), within five standard errors
        n = z.size
        assert abs(z.real.mean()) < 5 / np.sqrt(n) and abs(z.imag.mean()) < 5 / np.sqrt(n)
        assert abs(z.real.std() - 1) < 5 / np.sqrt(2 * n) and abs(z.imag.std() - 1) < 5 / np.sqrt(2 * n)
        assert abs(np.corrcoef(z.real.ravel(), z.imag.ravel())[0, 1]) < 5 / np.sqrt(n)


def test_3d_workloads_share_nodes_and_coefficients():
    a = inputs.workload("3d")
    b = inputs.workload("3d_lean")
    assert a["N"] == (128, 128, 128) and a["M"] == 2097152 and (a["sigma"], a["m"]) == (2.0, 4)
    assert (b["sigma"], b["m"]) == (1.25, 6)
    assert np.array_equal(a["k"], b["k"]) and np.array_equal(a["f"], b["f"])
    assert a["k"].min() >= -0.5 and a["k"].max() < 0.5


def test_workloads_are_deterministic_and_salted():
    a = inputs.workload("1d")
    b = inputs.workload("1d")
    c = inputs.workload("1d", rng_salt=1)
    assert np.array_equal(a["k"], b["k"]) and np.array_equal(a["f"], b["f"])
    assert not np.array_equal(a["k"], c["k"])
    with pytest.raises(KeyError):
        inputs.workload("4d")


def test_radial_set_structure():
    """402 spokes x 512 samples, theta_s = pi s / 402, r_i = (i - 256) / 512:
    the r = 0 sample of every spoke is the origin (on a grid point), the
    theta = 0 spoke lies on a grid line, everything is wrapped into
    [-1/2, 1/2)."""
    k = inputs.radial_nodes()
    assert k.shape == (402 * 512, 2)
    assert k.min() >= -0.5 and k.max() < 0.5
    spokes = k.reshape(402, 512, 2)
    assert np.all(spokes[:, 256] == 0.0)
    assert np.all(spokes[0, :, 1] == 0.0)
    # r = -1/2 on the theta = 0 spoke sits at k = -1/2 (kept, not wrapped to +1/2)
    assert spokes[0, 0, 0] == -0.5
    # the whole set is the recipe's formula, wrapped
    r = (np.arange(512) - 256) / 512.0
    theta = np.pi * np.arange(402) / 402
    want = inputs.wrap_half(np.stack([np.cos(theta)[:, None] * r, np.sin(theta)[:, None] * r], axis=-1))
    assert np.array_equal(spokes, want)


def test_differentiation_workload_jitter():
    wl = inputs.differentiation()
    assert wl["N"] == (256, 256) and wl["M"] == 402 * 512 and (wl["sigma"], wl["m"]) == (2.0, 4)
    k0 = inputs.radial_nodes()
    d = np.abs(inputs.wrap_half(wl["k"] - k0))
    # the angle jitter is N(0, 1e-3): displacement r |dtheta| <= 1/2 * 6e-3 at 6 sigma
    assert 0 < d.max() < 3e-3
    assert wl["f"].shape == (256, 256) and wl["y"].shape == (wl["M"],)


def test_batched_problems_recipe():
    probs = inputs.batched_problems(n_problems=64)
    assert len(probs) == 64
    sizes = {64, 128, 256, 512}
    seen = set()
    for p in probs:
        N1, N2 = p["N"]
        assert N1 in sizes and N2 in sizes
        seen.update(p["N"])
        assert 0.5 * N1 * N2 <= p["M"] < 2 * N1 * N2
        assert p["k"].shape == (p["M"], 2) and p["k"].min() >= -0.5 and p["k"].max() < 0.5
        assert p["f"].shape == (N1, N2) and p["w"].shape == (p["M"],)
    assert seen == sizes
    # uneven: both the sizes and the node counts vary across the batch
    assert len({p["N"] for p in probs}) > 8 and len({p["M"] for p in probs}) == 64


def test_radial_right_hand_sides():
    rhs = inputs.radial_rhs()
    assert rhs["N"] == (256, 256) and rhs["k"].shape == (402 * 512, 2)
    assert rhs["f"].shape == (32, 256, 256) and rhs["w"].shape == (32, 402 * 512)
    assert not np.array_equal(rhs["f"][0], rhs["f"][1])
