"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: relative L2 <= 1e-5 for complex64 and <= 1e-12 for complex128
(the stated targets), element-wise max within 10x that.  The oracle is the
plain FP64 NFFT of Algorithms 1/2 (same window, same footprint convention),
so the comparison isolates the arithmetic of the kernels; comparisons with
the exact NDFT check the method's accuracy as well.
"""
import numpy as np
import pytest

from oracle import ndft as ondft
from oracle import nfft as onfft
from oracle import window as owin
from paper_2208_00049_gb300 import inputs

from gpu_helpers import (TOL, assert_close, cdtype, fp32_floor, oracle_spread_box, rel_l2, rel_max, require_gpu,
                         to_dev, tol_for, tol_max_for)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _plan(N, M, sigma, m, dt, flags=0):
    from paper_2208_00049_gb300.nfft import Plan
    return Plan(N, M, sigma=sigma, m=m, dtype=cdtype(dt), flags=flags)


def _run(case, dt, flags=0, tile=None):
    N, M, sigma, m = case["N"], case["M"], case["sigma"], case["m"]
    plan = _plan(N, M, sigma, m, dt, flags)
    if tile is not None:
        plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    fh = plan.forward(to_dev(case["f"], cdtype(dt))).cpu().numpy()
    y = plan.adjoint(to_dev(case["w"], cdtype(dt))).cpu().numpy()
    plan.close()
    return fh, y


SMALL = [
    # (N, M, sigma, m): several tiles, ragged tails, odd sizes, non powers of 2
    ((300,), 700, 2.0, 4),
    ((257,), 513, 2.0, 3),
    ((48, 40), 2500, 2.0, 4),
    ((33, 47), 1777, 1.5, 5),
    ((64, 64), 4096, 2.0, 8),
    ((20, 18, 16), 5000, 2.0, 4),
    ((17, 23, 12), 3001, 2.0, 3),
    ((16, 16, 16), 4096, 1.25, 6),
    ((12, 10, 14), 1500, 2.0, 8),
    ((6, 8, 10), 500, 2.0, 2),
]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N,M,sigma,m", SMALL)
def test_small_cases_match_oracle(N, M, sigma, m, dt):
    case = inputs.small_case(N, M, seed=hash((N, M, m)) % 10000, sigma=sigma, m=m)
    fh, y = _run(case, dt)
    want_f = onfft.forward(case["k"], case["f"], sigma, m)
    want_a = onfft.adjoint(case["k"], case["w"], N, sigma, m)
    tol = tol_for(N, sigma, m, dt)
    tmax = tol_max_for(N, sigma, m, dt)
    assert_close(fh, want_f, tol, "forward", tol_max=tmax)
    assert_close(y, want_a, tol, "adjoint", tol_max=tmax)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_closed_support_matches_oracle(dt):
    """(2m+1)^D variant: nodes on grid lines get the u = +m tap."""
    N = (24, 20)
    case = inputs.small_case(N, 800, seed=3, m=3)
    p = onfft.Params(N, 2.0, 3)
    case["k"][:200, 0] = np.round(case["k"][:200, 0] * p.Nt[0]) / p.Nt[0]   # on a grid line
    case["k"][100:300, 1] = np.round(case["k"][100:300, 1] * p.Nt[1]) / p.Nt[1]
    from paper_2208_00049_gb300 import binding as B
    fh, y = _run(case, dt, flags=B.NFFT_FLAG_CLOSED_SUPPORT)
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 3, closed=True), TOL[dt], "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 3, closed=True), TOL[dt], "adjoint")


def test_workload1_1d_against_oracle_and_ndft():
    wl = inputs.workload("1d")
    for dt in ("c128", "c64"):
        fh, y = _run(wl, dt)
        assert_close(fh, onfft.forward(wl["k"], wl["f"], 2.0, 4), TOL[dt], "forward vs oracle")
        assert_close(y, onfft.adjoint(wl["k"], wl["w"], wl["N"], 2.0, 4), TOL[dt], "adjoint vs oracle")
        assert rel_l2(fh, ondft.ndft(wl["k"], wl["f"])) <= 1e-5
        assert rel_l2(y, ondft.ndft_adjoint(wl["k"], wl["w"], wl["N"])) <= 1e-5


@pytest.mark.parametrize("name", ["2d_c64", "2d_c128"])
def test_workload2_2d_full_size(name):
    wl = inputs.workload(name)
    dt, m = wl["dtype"], wl["m"]
    fh, y = _run(wl, dt)
    assert_close(fh, onfft.forward(wl["k"], wl["f"], 2.0, m), TOL[dt], "forward vs oracle")
    assert_close(y, onfft.adjoint(wl["k"], wl["w"], wl["N"], 2.0, m), TOL[dt], "adjoint vs oracle")
    # accuracy against the exact NDFT on 256 sampled nodes / 256 sampled outputs
    rng = np.random.default_rng(5)
    sel = rng.choice(wl["M"], 256, replace=False)
    ex = ondft.ndft(wl["k"][sel], wl["f"])
    assert rel_l2(fh[sel], ex) <= TOL[dt]
    flat = rng.choice(int(np.prod(wl["N"])), 256, replace=False)
    idx = np.unravel_index(flat, wl["N"])
    n = np.stack([idx[d] - wl["N"][d] // 2 for d in range(2)], axis=1).astype(float)
    ph = n @ wl["k"].T
    ph -= np.floor(ph)
    exa = np.exp(2j * np.pi * ph) @ wl["w"]
    assert rel_l2(y[idx], exa) <= TOL[dt]


@pytest.mark.parametrize("name", ["3d", "3d_lean"])
def test_workload3_3d_full_size_sampled(name):
    """Full 3D size in the launch configuration the bench times: forward on
    4096 sampled nodes against the plain oracle (which needs only those
    nodes' footprints) and 64 against the exact NDFT, adjoint on 64 sampled outputs against the exact NDFT,
    and the adjoint identity over all nodes."""
    wl = inputs.workload(name)
    sigma, m = wl["sigma"], wl["m"]
    rng = np.random.default_rng(6)
    sel = rng.choice(wl["M"], 4096, replace=False)
    tol = tol_a = tol_for(wl["N"], sigma, m, "c64")
    if tol > TOL["c64"]:
        # sigma = 1.25: the deconvolution amplifies single-precision rounding
        # (kappa ~ 1.7e5).  Forward: 3x the error of the oracle's own steps run
        # in single precision on the same nodes (the kernels measured at about
        # 2x of it).  The adjoint's floor depends on how many terms each grid
        # point sums (all M nodes), which the oracle cannot afford at this size:
        # its end-to-end bound stays u kappa here, and its steps are checked
        # one by one, tightly, in test_workload3_adjoint_steps.
        e_f, _ = fp32_floor(wl["N"], sigma, m, wl["k"][sel], wl["f"], wl["w"][sel])
        tol = max(TOL["c64"], 3 * e_f)
    fh, y = _run(wl, "c64")
    want = onfft.forward(wl["k"][sel], wl["f"], sigma, m)
    assert_close(fh[sel], want, tol, "forward (sampled) vs oracle")
    # exact NDFT on 64 of them
    ex = ondft.ndft(wl["k"][sel[:64]], wl["f"])
    assert rel_l2(fh[sel[:64]], ex) <= tol
    flat = rng.choice(int(np.prod(wl["N"])), 64, replace=False)
    idx = np.unravel_index(flat, wl["N"])
    n = np.stack([idx[d] - wl["N"][d] // 2 for d in range(3)], axis=1).astype(float)
    exa = np.empty(64, complex)
    for s in range(0, 64, 8):
        ph = n[s:s + 8] @ wl["k"].T
        ph -= np.floor(ph)
        exa[s:s + 8] = np.exp(2j * np.pi * ph) @ wl["w"]
    assert rel_l2(y[idx], exa) <= tol_a
    lhs = np.vdot(wl["w"], fh)
    rhs = np.vdot(y, wl["f"])
    # relative to the Cauchy-Schwarz scale (random vectors make <w, Af> itself small)
    assert abs(lhs - rhs) <= max(tol, tol_a) * np.linalg.norm(wl["w"]) * np.linalg.norm(fh)


@pytest.mark.parametrize("name", ["3d", "3d_lean"])
def test_workload3_adjoint_steps(name):
    """The full-size 3D adjoint in the bench's launch configuration, step by
    step: the adjoint resampling step element by element on two 16^3 boxes of
    the oversampled grid (one inside, one across the periodic corner; 8192
    grid values against the oracle's step run on the nodes that reach each
    box), then the inverse FFT + crop + correction steps on every output
    against the oracle's FP64 steps applied to the GPU's own grid, within 3x
    the error of numpy's complex64 inverse FFT on that grid at sigma = 2 and
    1.5x cuFFT's single-precision one at sigma = 1.25."""
    from paper_2208_00049_gb300.nfft import Plan
    wl = inputs.workload(name)
    N, sigma, m = wl["N"], wl["sigma"], wl["m"]
    plan = Plan(N, wl["M"], sigma=sigma, m=m, dtype=torch.complex64)
    plan.set_nodes(to_dev(wl["k"], torch.float64))
    plan.step_scatter(to_dev(wl["w"], torch.complex64))
    pruned = plan.paths()["pruned_fft"]
    grid_t = plan.grid_tensor().clone()
    grid = grid_t.cpu().numpy()
    y = torch.empty(N, dtype=torch.complex64, device="cuda")
    plan.step_fft_crop(y)
    y = y.cpu().numpy()
    plan.close()
    p = onfft.Params(N, sigma, m)
    peak = np.prod([float(onfft.psi(0.0, m, b)) for b in p.b])
    w32 = wl["w"].astype(np.complex64).astype(np.complex128)
    for lo in ((37, 101, 90), tuple(nt - 8 for nt in p.Nt)):
        want, idx, n = oracle_spread_box(N, sigma, m, wl["k"], w32, lo, 16)
        assert n > 1000
        assert_close(grid[idx] * peak, want, TOL["c64"], "scatter grid box at %s" % (lo,))
    want_y = onfft.crop_correction(p, onfft.fft_adjoint(grid.astype(np.complex128))) * peak
    if pruned and sigma == 2.0:
        # the library's own FFT at sigma = 2: within 3x numpy's complex64
        # inverse FFT (which is close to the rounding of the output alone)
        g32 = np.fft.ifftn(grid, norm="forward")
        assert g32.dtype == np.complex64
        f = 3
    else:
        # at sigma = 1.25 the correction amplifies the band edges by up to
        # 273 per dimension, and a single-precision FFT (cuFFT, or the
        # library's own 160-point form) loses about 1.6e-3 there while
        # numpy's complex64 FFT stays near 2e-5: the floor is cuFFT's inverse
        # FFT of the same grid, and the library's step may add little to it
        g32 = torch.fft.ifftn(grid_t, norm="forward").cpu().numpy()
        f = 1.5
    y_floor = onfft.crop_correction(p, g32.astype(np.complex128)) * peak
    assert_close(y, want_y, max(TOL["c64"], f * rel_l2(y_floor, want_y)), "inverse FFT + crop + correction",
                 tol_max=max(10 * TOL["c64"], f * rel_max(y_floor, want_y)))


def test_radial_set_on_grid_nodes():
    """Radial sets put the r = 0 sample of every spoke exactly on a grid
    point and two spokes on grid lines (t = 0 fractions)."""
    rad = inputs.radial_rhs(n_rhs=1)
    k = rad["k"]
    case = dict(N=rad["N"], M=k.shape[0], sigma=2.0, m=4, k=k, f=rad["f"][0], w=rad["w"][0])
    for dt in ("c64", "c128"):
        fh, y = _run(case, dt)
        assert_close(fh, onfft.forward(k, case["f"], 2.0, 4), TOL[dt], "forward")
        assert_close(y, onfft.adjoint(k, case["w"], case["N"], 2.0, 4), TOL[dt], "adjoint")


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_edge_cases(dt):
    # M = 0: empty forward, zero adjoint
    plan = _plan((16, 16), 0, 2.0, 4, dt)
    plan.set_nodes(torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    assert plan.forward(to_dev(np.ones((16, 16)), cdtype(dt))).numel() == 0
    y = plan.adjoint(torch.zeros(0, dtype=cdtype(dt), device="cuda"))
    assert torch.count_nonzero(y).item() == 0
    plan.close()
    # M = 1, nodes at the -1/2 corner and outside [-1/2, 1/2) (wrapped)
    for kval in ([-0.5, -0.5], [0.5, 0.25], [1.3, -0.7], [0.0, 0.0]):
        case = inputs.small_case((10, 12), 1, seed=1, m=2)
        case["k"] = np.array([kval])
        fh, y = _run(case, dt)
        kw = np.mod(case["k"] + 0.5, 1.0) - 0.5
        assert_close(fh, onfft.forward(kw, case["f"], 2.0, 2), TOL[dt] * 10, "M=1 forward")
        assert_close(y, onfft.adjoint(kw, case["w"], (10, 12), 2.0, 2), TOL[dt] * 10, "M=1 adjoint")
    # smallest grid: N = 2, m = 1
    case = inputs.small_case((2,), 5, seed=2, m=1)
    fh, y = _run(case, dt)
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 1), TOL[dt], "N=2")
    # one hot tile: every node in the same cell neighbourhood -> many work items
    case = inputs.small_case((64, 64), 5000, seed=3, m=4)
    case["k"] = 0.01 * case["k"]
    fh, y = _run(case, dt)
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), TOL[dt], "hot tile forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], (64, 64), 2.0, 4), TOL[dt], "hot tile adjoint")


@pytest.mark.parametrize("m", [4, 6])
def test_fast3d_edge_cases(m):
    """The 3D complex64 fast kernels (m = 4 and 6) with no nodes, one node at
    the corners of the unit cell, and nodes outside [-1/2, 1/2) (wrapped)."""
    N = (16, 14, 18)
    plan = _plan(N, 0, 2.0, m, "c64")
    plan.set_nodes(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert plan.paths()["fast_gather"] and plan.paths()["fast_scatter"]
    assert plan.forward(to_dev(np.ones(N), torch.complex64)).numel() == 0
    y = plan.adjoint(torch.zeros(0, dtype=torch.complex64, device="cuda"))
    assert torch.count_nonzero(y).item() == 0
    plan.close()
    for kval in ([-0.5, -0.5, -0.5], [0.5 - 1e-12, 0.25, -0.5], [1.3, -0.7, 2.0], [0.0, 0.0, 0.0]):
        case = inputs.small_case(N, 1, seed=5, m=m)
        case["k"] = np.array([kval])
        fh, y = _run(case, "c64")
        kw = np.mod(case["k"] + 0.5, 1.0) - 0.5
        assert_close(fh, onfft.forward(kw, case["f"], 2.0, m), 1e-4, "M=1 forward")
        assert_close(y, onfft.adjoint(kw, case["w"], N, 2.0, m), 1e-4, "M=1 adjoint")


@pytest.mark.parametrize("tile,sigma", [((9, 25), 2.0), ((8, 25), 2.0), ((3, 7), 2.0), ((9, 1), 2.0),
                                        ((1, 25), 2.0), ((9, 25), 1.5), ((8, 8), 1.25)])
def test_fast2d_m4_tile_shapes(tile, sigma):
    """2D, m = 4, complex64: the register-accumulating scatter and the
    warp-per-item gather (regions up to 16 x 32) on tiles dividing N~ or
    not, sigma 2, 1.5 and 1.25, with a hot tile (items split) and boundary
    nodes."""
    N = (40, 52)
    case = inputs.small_case(N, 6000, seed=43, sigma=sigma, m=4)
    case["k"][:2000] = 0.03 * case["k"][:2000]
    case["k"][2000:2200, 0] = -0.5
    from paper_2208_00049_gb300.nfft import Plan
    plan = Plan(N, case["M"], sigma=sigma, m=4, dtype=torch.complex64)
    plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    assert plan.paths()["fast_gather"] and plan.paths()["fast_scatter"]
    fh = plan.forward(to_dev(case["f"], torch.complex64)).cpu().numpy()
    y = plan.adjoint(to_dev(case["w"], torch.complex64)).cpu().numpy()
    plan.close()
    tol, tmax = tol_for(N, sigma, 4, "c64"), tol_max_for(N, sigma, 4, "c64")
    assert_close(fh, onfft.forward(case["k"], case["f"], sigma, 4), tol, "forward", tmax)
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, sigma, 4), tol, "adjoint", tmax)


def test_large_3d_against_ndft_samples():
    """A larger 3D plan (N = 256 x 256 x 128, N~ = 512 x 512 x 256, M = 4 194 304
    nodes, the default specialised kernels) against the exact NDFT on
    sampled outputs: 32 forward values and 32 adjoint values."""
    N = (256, 256, 128)
    rng = np.random.default_rng(2208 + 9)
    M = int(np.prod(N)) // 2
    k = inputs.uniform_nodes(rng, M, 3)
    f = inputs.complex_normal(rng, N, dtype=np.complex64)
    w = inputs.complex_normal(rng, (M,), dtype=np.complex64)
    plan = _plan(N, M, 2.0, 4, "c64")
    plan.set_nodes(to_dev(k, torch.float64))
    assert plan.paths()["fast_gather"] and plan.paths()["fast_scatter"]
    fh = plan.forward(to_dev(f, torch.complex64)).cpu().numpy()
    y = plan.adjoint(to_dev(w, torch.complex64)).cpu().numpy()
    plan.close()
    sel = rng.choice(M, 32, replace=False)
    assert_close(fh[sel], ondft.ndft(k[sel], f), 1e-5, "forward vs NDFT")
    idx = np.unravel_index(rng.choice(int(np.prod(N)), 32, replace=False), N)
    assert_close(y[idx], ondft.ndft_adjoint_at(k, w, N, idx), 1e-5, "adjoint vs NDFT")


@pytest.mark.parametrize("tile", [(4, 4, 4), (7, 5, 3), (8, 8, 16), (12, 32, 8)])
def test_tile_shapes_agree(tile):
    """Any tile shape (dividing N~ or not) gives the oracle's result."""
    N = (20, 16, 24)
    case = inputs.small_case(N, 4000, seed=9, m=4)
    fh, y = _run(case, "c128", tile=tile)
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), 1e-12, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 4), 1e-12, "adjoint")


def test_compensated_scatter():
    """The compensated shared-memory scatter against the plain one of the same
    kernel family (a 16 x 16 tile is outside the register-accumulating 2D
    kernels, which evaluate the window in POLYNOMIAL form; the shared-memory
    kernels evaluate it directly), and the default plan beside them."""
    from paper_2208_00049_gb300 import binding as B
    N = (48, 40)
    case = inputs.small_case(N, 20000, seed=11, m=4)
    want = onfft.adjoint(case["k"], case["w"], N, 2.0, 4)
    _, y0 = _run(case, "c64", tile=(16, 16))
    _, y1 = _run(case, "c64", flags=B.NFFT_FLAG_COMPENSATED, tile=(16, 16))
    _, y2 = _run(case, "c64")
    e0 = assert_close(y0, want, 1e-5, "plain")
    e1 = assert_close(y1, want, 1e-5, "compensated")
    assert_close(y2, want, 1e-5, "default plan")
    assert e1 <= 1.5 * e0 + 1e-7


@pytest.mark.parametrize("N,M", [((32, 32), 200000), ((16, 16, 16), 100000)])
def test_compensated_fast_scatter(N, M):
    """NFFT_FLAG_COMPENSATED on the register-accumulating complex64 scatters
    (2D and 3D, m = 4), with thousands of terms per grid point: the
    compensated grid is closer to the FP64 oracle's adjoint resampling step
    than the plain one, and both adjoint transforms are within the target.
    (Only the sums held in registers are compensated: the partial sums of
    neighbouring tiles still meet in FP32 global reductions, and the FP32
    products and window values set a floor, so the gain is bounded.)"""
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan
    case = inputs.small_case(N, M, seed=17, m=4)
    p = onfft.Params(N, 2.0, 4)
    peak = np.prod([float(onfft.psi(0.0, 4, b)) for b in p.b])
    w32 = case["w"].astype(np.complex64)
    want = onfft.resample_adjoint(p, case["k"], w32.astype(np.complex128))
    want_y = onfft.adjoint(case["k"], w32.astype(np.complex128), N, 2.0, 4)
    errs = {}
    for flags in (0, B.NFFT_FLAG_COMPENSATED):
        plan = Plan(N, M, sigma=2.0, m=4, dtype=torch.complex64, flags=flags)
        plan.set_nodes(to_dev(case["k"], torch.float64))
        assert plan.paths()["fast_scatter"]
        w = torch.from_numpy(w32).cuda()
        plan.step_scatter(w)
        errs[flags] = rel_l2(plan.grid_tensor().cpu().numpy() * peak, want)
        y = plan.adjoint(w).cpu().numpy()
        plan.close()
        assert_close(y, want_y, 1e-5, "adjoint flags=%d" % flags)
    assert errs[B.NFFT_FLAG_COMPENSATED] <= 0.85 * errs[0], errs


def test_steps_match_oracle_steps():
    """Each exported step against the oracle's step on the same input."""
    N, M, m = (30, 26), 3000, 4
    case = inputs.small_case(N, M, seed=13, m=m)
    p = onfft.Params(N, 2.0, m)
    plan = _plan(N, M, 2.0, m, "c128")
    plan.set_nodes(to_dev(case["k"], torch.float64))
    f = to_dev(case["f"], torch.complex128)
    plan.step_deconv_pad(f)
    grid = plan.grid_tensor().cpu().numpy()
    want_g = onfft.correction_pad(p, case["f"])
    # the library scales the deconvolution by the window peak prod_d psi_d(0)
    peak = np.prod([float(onfft.psi(0.0, m, b)) for b in p.b])
    assert_close(grid / peak, want_g, 1e-13, "deconv_pad")
    # gather from a given grid
    ghat = np.random.default_rng(1).standard_normal(p.Nt) + 0j
    plan.grid_tensor().copy_(torch.from_numpy(ghat))
    out = torch.empty(M, dtype=torch.complex128, device="cuda")
    plan.step_gather(out)
    assert_close(out.cpu().numpy() * peak, onfft.resample(p, case["k"], ghat), 1e-13, "gather")
    plan.step_scatter(to_dev(case["w"], torch.complex128))
    got = plan.grid_tensor().cpu().numpy() * peak
    assert_close(got, onfft.resample_adjoint(p, case["k"], case["w"]), 1e-13, "scatter")
    plan.close()


def test_host_pointers_match_device_path():
    N, M = (32, 24), 1500
    case = inputs.small_case(N, M, seed=17, m=4)
    plan = _plan(N, M, 2.0, 4, "c64")
    plan.set_nodes(torch.from_numpy(case["k"]))                 # pageable host nodes
    f_h = torch.from_numpy(case["f"]).to(torch.complex64).pin_memory()
    fh_host = plan.forward(f_h)                                  # pinned host in/out
    assert not fh_host.is_cuda
    fh_dev = plan.forward(f_h.cuda()).cpu()
    assert torch.equal(fh_host, fh_dev)
    w_h = torch.from_numpy(case["w"]).to(torch.complex64)        # pageable
    y_host = plan.adjoint(w_h)
    y_dev = plan.adjoint(w_h.cuda()).cpu()
    assert rel_l2(y_host.numpy(), y_dev.numpy()) <= 1e-6
    plan.close()


def test_gather_is_deterministic_and_fp32_nodes_accepted():
    N, M = (40, 40), 3000
    case = inputs.small_case(N, M, seed=19, m=4)
    plan = _plan(N, M, 2.0, 4, "c64")
    plan.set_nodes(to_dev(case["k"], torch.float64))
    f = to_dev(case["f"], torch.complex64)
    a = plan.forward(f).clone()
    b = plan.forward(f).clone()
    assert torch.equal(a, b)
    k32 = case["k"].astype(np.float32)
    plan.set_nodes(torch.from_numpy(k32).cuda())
    c = plan.forward(f).cpu().numpy()
    assert_close(c, onfft.forward(k32.astype(np.float64), case["f"], 2.0, 4), 1e-5, "fp32 nodes")
    plan.close()


@pytest.mark.parametrize("tile", [(8, 8, 8), (5, 7, 9), (16, 4, 3), (8, 8, 1), (3, 11, 2)])
def test_fast3d_m4_tile_shapes(tile):
    """3D, m = 4, complex64 (the warp-per-node kernels): any admissible tile
    shape, dividing N~ or not, gives the oracle's result."""
    N = (24, 20, 28)
    case = inputs.small_case(N, 6000, seed=23, m=4)
    fh, y = _run(case, "c64", tile=tile)
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), 1e-5, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 4), 1e-5, "adjoint")


@pytest.mark.parametrize("tile", [(9, 9, 8), (8, 8, 8), (4, 6, 2), (5, 7, 9)])
def test_region_copy_forms_agree(tile, monkeypatch):
    """3D, m = 4, complex64: the gather and the node gradient copy a region
    that lies inside the grid with one tensor-memory-accelerator box (even
    T2) and a wrapping region, or any region of an odd-T2 tile, with
    cp.async.  With the TMA switched off (NFFT_GB300_GATHER_TMA=0) every
    region goes through cp.async; the same bytes land in the same layout, so
    the results must be bit-identical; and both match the oracle."""
    from paper_2208_00049_gb300.nfft import Plan
    N, M = (40, 36, 44), 20000
    case = inputs.small_case(N, M, seed=53, m=4)
    cot = inputs.complex_normal(np.random.default_rng(7), (M,))
    plan = Plan(N, M, sigma=2.0, m=4, dtype=torch.complex64)
    plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    assert plan.paths()["fast_gather"]
    f, c = to_dev(case["f"], torch.complex64), to_dev(cot, torch.complex64)
    out = {}
    for form in ("1", "0"):
        monkeypatch.setenv("NFFT_GB300_GATHER_TMA", form)
        fh = plan.forward(f).cpu().numpy()
        gk = plan.grad(f, c).cpu().numpy()
        plan.sync()
        out[form] = (fh, gk)
    plan.close()
    assert np.array_equal(out["1"][0], out["0"][0]), "forward differs between the copy forms"
    assert np.array_equal(out["1"][1], out["0"][1]), "node gradient differs between the copy forms"
    assert_close(out["1"][0], onfft.forward(case["k"], case["f"], 2.0, 4), 1e-5, "forward")


@pytest.mark.parametrize("sigma", [2.0, 1.25])
@pytest.mark.parametrize("tile", [(5, 5, 5), (3, 4, 5), (5, 5, 1), (2, 5, 3)])
def test_fast_m6_tile_shapes(sigma, tile):
    """3D, m = 6, complex64: the K = 12 gather and the register-accumulating
    scatter (tiles of at most 5 cells per dimension) against the oracle,
    sigma = 2 and the lean sigma = 1.25."""
    from paper_2208_00049_gb300.nfft import Plan
    N = (20, 18, 24)
    case = inputs.small_case(N, 5000, seed=37, sigma=sigma, m=6)
    plan = Plan(N, case["M"], sigma=sigma, m=6, dtype=torch.complex64)
    plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    assert plan.paths()["fast_scatter"] and plan.paths()["fast_gather"]
    fh = plan.forward(to_dev(case["f"], torch.complex64)).cpu().numpy()
    y = plan.adjoint(to_dev(case["w"], torch.complex64)).cpu().numpy()
    plan.close()
    tol = tol_a = TOL["c64"]
    tmax = tol_max_for(N, sigma, 6, "c64")
    if sigma < 2.0:
        # 3x the error of the oracle's own steps run in single precision
        e_f, e_a = fp32_floor(N, sigma, 6, case["k"], case["f"], case["w"])
        tol, tol_a = max(tol, 3 * e_f), max(tol, 3 * e_a)
    assert_close(fh, onfft.forward(case["k"], case["f"], sigma, 6), tol, "forward", tmax)
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, sigma, 6), tol_a, "adjoint", tmax)


@pytest.mark.parametrize("m,tile,hot", [(6, (5, 5, 5), False), (6, (5, 5, 5), True), (6, (2, 5, 3), False),
                                        (4, (9, 9, 8), False), (4, (9, 9, 8), True), (4, (5, 7, 9), False),
                                        (4, (8, 8, 1), False)])
def test_gather_forms_match_oracle(m, tile, hot, monkeypatch):
    """3D complex64 gather in its two forms: the register-resident kernel
    (each thread holds two region lines in registers; the default at m = 6,
    selected by NFFT_GB300_GATHER=regs at m = 4) and the shared-tap kernels
    (NFFT_GB300_GATHER=smem).  Both against the oracle, on tiles that divide
    the grid or not, with hot tiles (work items split at the per-item cap)
    and nodes on the periodic boundary; the two forms differ only in the
    order of the sums, and each repeats its result bit for bit."""
    from paper_2208_00049_gb300.nfft import Plan
    N = (16, 16, 16) if hot else (20, 18, 24)
    case = inputs.small_case(N, 6000, seed=59 + m, m=m)
    if hot:
        case["k"][:4000] = 0.02 * case["k"][:4000]
        case["k"][4000:4400, 1] = -0.5
        case["k"][4400:4800, 2] = 0.5 - 1e-9
    plan = Plan(N, case["M"], sigma=2.0, m=m, dtype=torch.complex64)
    plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    assert plan.paths()["fast_gather"]
    f = to_dev(case["f"], torch.complex64)
    ref = onfft.forward(case["k"], case["f"], 2.0, m)
    out = {}
    for form in ("regs", "smem"):
        monkeypatch.setenv("NFFT_GB300_GATHER", form)
        a = plan.forward(f).clone()
        b = plan.forward(f).clone()
        plan.sync()
        assert torch.equal(a, b), form + " gather is not deterministic"
        out[form] = a.cpu().numpy()
        assert_close(out[form], ref, 1e-5, form + " forward")
    plan.close()
    assert rel_l2(out["regs"], out["smem"]) <= 1e-6


@pytest.mark.parametrize("N,M,sigma,m,tile,hot,flags", [
    ((64, 64), 4096, 2.0, 8, None, False, 0),
    ((64, 64), 4096, 2.0, 8, (7, 40), True, 0),
    ((48, 40), 2500, 2.0, 4, (16, 16), False, 0),
    ((33, 47), 1777, 1.5, 5, None, False, 0),
    ((40, 36), 3000, 2.0, 6, (3, 33), True, 0),
    ((40, 36), 3000, 2.0, 6, None, False, "linear"),
    ((20, 24), 800, 2.0, 1, None, False, 0),
    ((20, 18, 16), 5000, 2.0, 4, None, False, 0),
    ((20, 18, 16), 5000, 2.0, 4, (5, 7, 9), True, 0),
    ((17, 23, 12), 3001, 2.0, 3, (3, 11, 2), False, 0),
    ((16, 16, 16), 4096, 1.5, 2, None, True, 0),
    ((12, 10, 14), 1500, 2.0, 4, None, False, "linear"),
    ((10, 8, 12), 600, 2.0, 1, None, False, 0),
])
def test_f64_scatter_matches_oracle(N, M, sigma, m, tile, hot, flags, monkeypatch):
    """2D and 3D complex128 adjoint through the scatter without shared-memory
    atomics (threads own region points by residue class: in 2D columns mod 16
    and rows mod 8, in 3D (mod 4, mod 4, mod 8); the default for even K = 2m
    up to 16 in 2D and 8 in 3D) and through the generic shared-atomic scatter
    (NFFT_GB300_F64_SCATTER=generic): both against the oracle within the
    complex128 tolerance, on tiles wider and narrower than the residue
    classes, with hot tiles and boundary nodes, in the POLYNOMIAL (m >= 7),
    direct and LINEAR window forms."""
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan
    case = inputs.small_case(N, M, seed=71 + m, sigma=sigma, m=m)
    if hot:
        case["k"][: M // 2] = 0.02 * case["k"][: M // 2]
        case["k"][M // 2: M // 2 + 200, 0] = -0.5
        case["k"][M // 2 + 200: M // 2 + 400, len(N) - 1] = 0.5 - 1e-12
    fl = B.NFFT_FLAG_WINDOW_LINEAR if flags == "linear" else 0
    plan = Plan(N, M, sigma=sigma, m=m, dtype=torch.complex128, flags=fl)
    if tile is not None:
        plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    w = to_dev(case["w"], torch.complex128)
    out = {}
    for form in ("lanes", "generic"):
        if form == "generic":
            monkeypatch.setenv("NFFT_GB300_F64_SCATTER", "generic")
        out[form] = plan.adjoint(w).cpu().numpy()
        plan.sync()
    plan.close()
    if flags == "linear":  # the oracle reads the same table with linear interpolation
        want = onfft.adjoint(case["k"], case["w"], N, sigma, m, window="linear")
    else:
        want = onfft.adjoint(case["k"], case["w"], N, sigma, m)
    tol = tol_for(N, sigma, m, "c128")
    for form in out:
        assert_close(out[form], want, tol, form + " adjoint", tol_max_for(N, sigma, m, "c128"))
    assert rel_l2(out["lanes"], out["generic"]) <= 1e-13


def test_fast_m6_hot_tile():
    """m = 6: work items split at the per-item cap, nodes on the boundary."""
    from paper_2208_00049_gb300.nfft import Plan
    N = (16, 16, 16)
    case = inputs.small_case(N, 6000, seed=41, m=6)
    case["k"][:4000] = 0.02 * case["k"][:4000]
    case["k"][4000:4500, 1] = -0.5
    plan = Plan(N, case["M"], sigma=2.0, m=6, dtype=torch.complex64)
    plan.set_tile((5, 5, 5))
    plan.set_nodes(to_dev(case["k"], torch.float64))
    assert plan.paths()["fast_scatter"] and plan.paths()["fast_gather"]
    fh = plan.forward(to_dev(case["f"], torch.complex64)).cpu().numpy()
    y = plan.adjoint(to_dev(case["w"], torch.complex64)).cpu().numpy()
    plan.close()
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 6), 1e-5, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 6), 1e-5, "adjoint")


def test_fast3d_m4_hot_tile_and_boundaries():
    """Many nodes in one tile (work items split at the per-item cap) and nodes
    on the periodic boundary of the 3D grid."""
    N = (16, 16, 16)
    case = inputs.small_case(N, 7000, seed=29, m=4)
    case["k"][:5000] = 0.02 * case["k"][:5000]                  # hot tiles near the origin
    case["k"][5000:5500, 0] = -0.5                              # on the lower boundary
    case["k"][5500:6000, 2] = 0.5 - 1e-9                        # just below the upper boundary
    fh, y = _run(case, "c64")
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), 1e-5, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 4), 1e-5, "adjoint")


@pytest.mark.parametrize("N,M,dt", [((40, 36), 3000, "c64"), ((24, 20, 28), 6000, "c64"), ((300,), 900, "c128")])
def test_autotuned_plan_matches_oracle(N, M, dt):
    """The autotuner picks a tile by timing candidates; results stay exact."""
    from paper_2208_00049_gb300.nfft import Plan
    case = inputs.small_case(N, M, seed=59, m=4)
    plan = Plan(N, M, sigma=2.0, m=4, dtype=cdtype(dt))
    k = to_dev(case["k"], torch.float64)
    tile = plan.autotune(k)
    assert len(tile) == len(N) and plan.info()["tile"] == tuple(tile)
    fh = plan.forward(to_dev(case["f"], cdtype(dt))).cpu().numpy()
    y = plan.adjoint(to_dev(case["w"], cdtype(dt))).cpu().numpy()
    plan.close()
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), TOL[dt], "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, 4), TOL[dt], "adjoint")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N,M,m", [((300,), 700, 4), ((40, 36), 2500, 4), ((20, 18, 16), 3000, 4),
                                   ((12, 10, 14), 1500, 3), ((64, 48), 3000, 8)])
def test_full_matrix_form_matches_oracle(N, M, m, dt):
    """NFFT_FLAG_FULL_MATRIX (B and B^T as CSR applied with cuSPARSE)."""
    from paper_2208_00049_gb300 import binding as B
    case = inputs.small_case(N, M, seed=67, m=m)
    fh, y = _run(case, dt, flags=B.NFFT_FLAG_FULL_MATRIX)
    tol = TOL[dt]
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, m), tol, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, m), tol, "adjoint")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N,M,m", [((200,), 500, 3), ((40, 36), 2500, 4), ((16, 14, 18), 2000, 3), ((20, 18, 16), 3000, 4)])
def test_wide_window_matches_oracle(N, M, m, dt):
    """NFFT_FLAG_WIDE_WINDOW: (2m+2)^D taps of the untruncated window."""
    from paper_2208_00049_gb300 import binding as B
    case = inputs.small_case(N, M, seed=71, m=m)
    fh, y = _run(case, dt, flags=B.NFFT_FLAG_WIDE_WINDOW)
    tol = TOL[dt]
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, m, wide=True), tol, "forward")
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, m, wide=True), tol, "adjoint")


def test_accuracy_study_against_ndft():
    """Sec. 5.1 on the GPU path (complex128, 2D, M = |I_N|, sigma = 2): the
    error against the exact NDFT decays exponentially in m and saturates by
    m = 8; the (2m+2)-point variant beats 2m points and loses to m + 1."""
    from paper_2208_00049_gb300 import binding as B
    N = (40, 40)
    M = 1600
    case = inputs.small_case(N, M, seed=73)
    ex = ondft.ndft(case["k"], case["f"])
    exa = ondft.ndft_adjoint(case["k"], case["w"], N)
    errs, errs_a, wide = {}, {}, {}
    for m in range(2, 9):
        c = dict(case, m=m)
        fh, y = _run(c, "c128")
        errs[m] = rel_l2(fh, ex)
        errs_a[m] = rel_l2(y, exa)
        if m <= 6:
            fw, _ = _run(c, "c128", flags=B.NFFT_FLAG_WIDE_WINDOW)
            wide[m] = rel_l2(fw, ex)
    for e in (errs, errs_a):
        for m in range(2, 7):
            assert e[m + 1] < e[m] / 10
        assert e[8] < 1e-12
    for m in range(2, 6):
        assert wide[m] < errs[m]
        assert errs[m + 1] < wide[m]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N,M,m", [((300,), 700, 4), ((40, 36), 2500, 4), ((20, 18, 16), 3000, 4),
                                   ((24, 20), 2000, 6)])
def test_window_modes_match_oracle(N, M, m, dt):
    """The three window modes of Sec. 3.7.4 on the same (generic) kernels:
    DIRECT and LINEAR against the oracle with the same window reading (the
    LINEAR table read with linear interpolation on both sides), POLYNOMIAL
    against the evaluated window within its fit error (degree 2m: about
    1e-8 of the peak at m = 4, FP64-level from m = 6)."""
    from paper_2208_00049_gb300 import binding as B
    case = inputs.small_case(N, M, seed=83, m=m)
    for flag, win, tol in ((B.NFFT_FLAG_WINDOW_DIRECT, "direct", TOL[dt]),
                           (B.NFFT_FLAG_WINDOW_LINEAR, "linear", TOL[dt]),
                           (B.NFFT_FLAG_WINDOW_POLYNOMIAL, "direct", max(TOL[dt], 1e-7 if m < 6 else 1e-12))):
        fh, y = _run(case, dt, flags=flag)
        assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, m, window=win), tol, "forward %s" % win)
        assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, m, window=win), tol, "adjoint %s" % win)


def test_linear_window_node_gradient():
    """The node gradient with the LINEAR window: the derivative of the
    interpolant (its segment's slope), as in the oracle's reading."""
    from paper_2208_00049_gb300 import binding as B
    N, M = (24, 20), 1500
    case = inputs.small_case(N, M, seed=89, m=4)
    plan = _plan(N, M, 2.0, 4, "c128", flags=B.NFFT_FLAG_WINDOW_LINEAR)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    gk = plan.grad(to_dev(case["f"], torch.complex128), to_dev(case["w"], torch.complex128)).cpu().numpy()
    plan.close()
    want = onfft.node_grad(case["k"], case["f"], case["w"], 2.0, 4, window="linear")
    # The slope is the difference of two adjacent table entries divided by
    # the spacing m / (S - 2): last-bit differences between the two tables
    # (CUDA's and numpy's sinh) grow by (S - 2) / m, S = 4 * 2^14 + 2.
    S = owin.lut_size(4)
    tol = 4 * np.finfo(np.float64).eps * (S - 2) / 4
    assert_close(gk, want, tol, "node gradient (LINEAR)")


@pytest.mark.parametrize("N,M,m", [((40, 36), 2000, 9), ((44, 40), 2000, 10), ((300,), 600, 10)])
def test_high_m_against_oracle(N, M, m):
    """m = 9, 10 (the end of the paper's accuracy curves) in 1D and 2D,
    complex128, against the oracle; 3D reports NFFT_ERR_UNSUPPORTED there,
    and so does the node gradient at m = 10 (2m = 20 taps)."""
    from paper_2208_00049_gb300 import binding as B
    case = inputs.small_case(N, M, seed=97, m=m)
    fh, y = _run(case, "c128")
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, m), 1e-12, "forward m=%d" % m)
    assert_close(y, onfft.adjoint(case["k"], case["w"], N, 2.0, m), 1e-12, "adjoint m=%d" % m)
    s, h = B.nfft_plan_create(3, (24, 24, 24), 100, 2.0, 9, B.NFFT_C128, 0, None)
    assert s == B.NFFT_ERR_UNSUPPORTED and not h
    plan = _plan(N, M, 2.0, m, "c128")
    plan.set_nodes(to_dev(case["k"], torch.float64))
    fd, wd = to_dev(case["f"], torch.complex128), to_dev(case["w"], torch.complex128)
    if m == 9:
        gk = plan.grad(fd, wd).cpu().numpy()
        assert_close(gk, onfft.node_grad(case["k"], case["f"], case["w"], 2.0, m), 1e-12, "node gradient m=9")
    else:
        with pytest.raises(B.NFFTError):
            plan.grad(fd, wd)
    plan.close()


@pytest.mark.parametrize("N,M,dt", [((256,), 1024, "c128"), ((64, 48), 3000, "c64"), ((20, 18, 16), 3000, "c64"),
                                    ((128, 128, 128), 20000, "c64")])
def test_graph_replay_matches_direct_path(N, M, dt):
    """nfft_plan_set_graph: forward and adjoint replayed from captured graphs
    give the direct path's results, follow new input data in the same
    buffers, re-capture for new buffers, and survive nfft_set_nodes."""
    case = inputs.small_case(N, M, seed=101, m=4)
    plan = _plan(N, M, 2.0, 4, dt)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    f = to_dev(case["f"], cdtype(dt))
    w = to_dev(case["w"], cdtype(dt))
    want_f = plan.forward(f).cpu().numpy()
    want_a = plan.adjoint(w).cpu().numpy()
    plan.set_graph(True)
    fh = torch.empty(M, dtype=cdtype(dt), device="cuda")
    y = torch.empty(N, dtype=cdtype(dt), device="cuda")
    for _ in range(3):
        plan.forward(f, out=fh)
        plan.adjoint(w, out=y)
    assert_close(fh.cpu().numpy(), want_f, 1e-6 if dt == "c64" else 1e-14, "graph forward")
    assert_close(y.cpu().numpy(), want_a, 1e-6 if dt == "c64" else 1e-14, "graph adjoint")
    f.mul_(2)                                   # new data, same buffers: the replay reads it
    plan.forward(f, out=fh)
    assert_close(fh.cpu().numpy(), 2 * want_f, 1e-6 if dt == "c64" else 1e-14, "graph forward, new data")
    fh2 = torch.empty_like(fh)                  # new buffers: re-captured
    plan.forward(f, out=fh2)
    assert_close(fh2.cpu().numpy(), 2 * want_f, 1e-6 if dt == "c64" else 1e-14, "graph forward, new buffers")
    k2 = inputs.small_case(N, M, seed=103, m=4)["k"]
    plan.set_nodes(to_dev(k2, torch.float64))   # new nodes, same node buffers
    plan.forward(f, out=fh)
    assert_close(fh.cpu().numpy(), onfft.forward(k2, 2 * case["f"], 2.0, 4), TOL[dt], "graph after set_nodes")
    plan.close()


def test_graph_mode_full_matrix_takes_direct_path():
    """A FULL plan rebuilds its sparse matrices in nfft_set_nodes; in graph
    mode it keeps launching directly, so new nodes are always seen."""
    from paper_2208_00049_gb300 import binding as B
    N, M = (24, 20), 800
    case = inputs.small_case(N, M, seed=107, m=3)
    plan = _plan(N, M, 2.0, 3, "c128", flags=B.NFFT_FLAG_FULL_MATRIX)
    plan.set_graph(True)
    f = to_dev(case["f"], torch.complex128)
    fh = torch.empty(M, dtype=torch.complex128, device="cuda")
    for seed in (107, 109):
        k = inputs.small_case(N, M, seed=seed, m=3)["k"]
        plan.set_nodes(to_dev(k, torch.float64))
        plan.forward(f, out=fh)
        assert_close(fh.cpu().numpy(), onfft.forward(k, case["f"], 2.0, 3), TOL["c128"], "FULL, graph mode")
    plan.close()


@pytest.mark.parametrize("N,M,dt", [((20, 18, 16), 3000, "c64"), ((48, 40), 2500, "c128"), ((128, 128, 128), 20000, "c64")])
def test_async_host_transforms(N, M, dt):
    """nfft_plan_set_async: several host-buffer forward / adjoint calls in
    flight at once (alternating stage buffers, copies on their own streams)
    give the synchronous path's results once nfft_plan_sync returns; a call
    with a device buffer keeps the synchronous path."""
    cases = [inputs.small_case(N, M, seed=131 + i, m=4) for i in range(3)]
    plan = _plan(N, M, 2.0, 4, dt)
    plan.set_nodes(to_dev(cases[0]["k"], torch.float64))
    ct = cdtype(dt)
    want = []
    for c in cases:
        fh = plan.forward(torch.from_numpy(c["f"]).to(ct)).numpy().copy()
        y = plan.adjoint(torch.from_numpy(c["w"]).to(ct)).numpy().copy()
        want.append((fh, y))
    plan.set_async(True)
    f_h = [torch.from_numpy(c["f"]).to(ct).pin_memory() for c in cases]
    w_h = [torch.from_numpy(c["w"]).to(ct).pin_memory() for c in cases]
    fh_h = [torch.empty(M, dtype=ct).pin_memory() for _ in cases]
    y_h = [torch.empty(N, dtype=ct).pin_memory() for _ in cases]
    for rep in range(2):
        for i in range(3):
            plan.forward(f_h[i], out=fh_h[i])
            plan.adjoint(w_h[i], out=y_h[i])
        plan.sync()
        tol = 1e-6 if dt == "c64" else 1e-14
        for i in range(3):
            assert_close(fh_h[i].numpy(), want[i][0], tol, "async forward %d" % i)
            assert_close(y_h[i].numpy(), want[i][1], tol, "async adjoint %d" % i)
    # a device output keeps the synchronous path
    fd = torch.empty(M, dtype=ct, device="cuda")
    plan.forward(f_h[1], out=fd)
    assert_close(fd.cpu().numpy(), want[1][0], 1e-6 if dt == "c64" else 1e-14, "async mode, device output")
    plan.set_async(False)
    plan.forward(f_h[2], out=fh_h[2])
    assert_close(fh_h[2].numpy(), want[2][0], 1e-6 if dt == "c64" else 1e-14, "after async mode")
    plan.close()
