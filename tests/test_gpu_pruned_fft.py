"""GPU parity of the library's own FFT forms against the FP64 oracle: the
pruned 3D FFT (N~_d = 2 N_d = 256, complex64) and the direct sums of small 1D
complex128 plans.  The fused steps (Algorithm 1: correction + zero pad + FFT;
Algorithm 2: inverse FFT + crop + correction) element by element on the full
grid / output, the whole transforms and the node gradient through them, and
the selection rules."""
import numpy as np
import pytest

from oracle import nfft as onfft
from paper_2208_00049_gb300 import inputs

from gpu_helpers import assert_close, cdtype, rel_l2, require_gpu, to_dev, tol_for, tol_max_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N3 = (128, 128, 128)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _plan(N, M, dt="c64", flags=0, sigma=2.0, m=4):
    from paper_2208_00049_gb300.nfft import Plan
    return Plan(N, M, sigma=sigma, m=m, dtype=cdtype(dt), flags=flags)


def _peak(p):
    # the library scales the window to 1 at u = 0 and the correction by
    # prod_d psi_d(0) to match
    return float(np.prod([float(onfft.psi(0.0, p.m, b)) for b in p.b]))


def test_pruned_path_selection():
    from paper_2208_00049_gb300 import binding as B
    cases = [
        ((128, 128, 128), "c64", 0, 2.0, True),
        ((128, 128, 128), "c64", B.NFFT_FLAG_LIBRARY_FFT, 2.0, False),
        ((128, 128, 128), "c128", 0, 2.0, False),
        ((128, 128, 64), "c64", 0, 2.0, False),
        ((128, 128, 128), "c64", 0, 1.5, False),
        ((128, 128, 128), "c64", 0, 1.25, True),
        ((128, 128, 128), "c64", B.NFFT_FLAG_LIBRARY_FFT, 1.25, False),
        ((128, 128), "c64", 0, 2.0, False),
        ((256, 256), "c64", 0, 2.0, True),
        ((256, 256), "c64", B.NFFT_FLAG_LIBRARY_FFT, 2.0, False),
        ((256, 256), "c128", 0, 2.0, False),
        ((256, 128), "c64", 0, 2.0, False),
    ]
    for N, dt, flags, sigma, want in cases:
        plan = _plan(N, 8, dt, flags, sigma)
        assert plan.paths()["pruned_fft"] is want, (N, dt, flags, sigma)
        plan.close()


def test_pad_fft_matches_oracle():
    """Algorithm 1's correction, zero-pad and FFT steps on the full grid."""
    rng = np.random.default_rng(2208)
    f = inputs.complex_normal(rng, N3)
    p = onfft.Params(N3, 2.0, 4)
    plan = _plan(N3, 8)
    assert plan.paths()["pruned_fft"]
    plan.step_pad_fft(to_dev(f, torch.complex64))
    got = plan.grid_tensor().cpu().numpy().astype(np.complex128) / _peak(p)
    want = onfft.fft_forward(onfft.correction_pad(p, f))
    assert_close(got, want, tol_for(N3, 2.0, 4, "c64"), "pad_fft", tol_max_for(N3, 2.0, 4, "c64"))
    plan.close()


def test_fft_crop_matches_oracle():
    """Algorithm 2's inverse FFT, crop and correction steps on an arbitrary grid."""
    rng = np.random.default_rng(49)
    p = onfft.Params(N3, 2.0, 4)
    G = inputs.complex_normal(rng, p.Nt)
    plan = _plan(N3, 8)
    plan.grid_tensor().copy_(torch.from_numpy(G.astype(np.complex64)))
    y = torch.empty(N3, dtype=torch.complex64, device="cuda")
    plan.step_fft_crop(y)
    got = y.cpu().numpy().astype(np.complex128) / _peak(p)
    want = onfft.crop_correction(p, onfft.fft_adjoint(G))
    assert_close(got, want, tol_for(N3, 2.0, 4, "c64"), "fft_crop", tol_max_for(N3, 2.0, 4, "c64"))
    plan.close()


def test_pruned_and_library_fft_agree():
    """Both FP32 forms of the same steps agree to FP32 rounding."""
    from paper_2208_00049_gb300 import binding as B
    rng = np.random.default_rng(7)
    f = to_dev(inputs.complex_normal(rng, N3), torch.complex64)
    grids = []
    for flags in (0, B.NFFT_FLAG_LIBRARY_FFT):
        plan = _plan(N3, 8, flags=flags)
        plan.step_pad_fft(f)
        grids.append(plan.grid_tensor().cpu().numpy())
        plan.close()
    assert rel_l2(grids[0], grids[1]) <= 2e-6


@pytest.mark.parametrize("M", [1, 20000])
def test_transforms_through_pruned_fft(M):
    """nfft_forward / nfft_adjoint at N = 128^3 (pruned path) against the oracle."""
    rng = np.random.default_rng(1000 + M)
    k = inputs.uniform_nodes(rng, M, 3)
    f = inputs.complex_normal(rng, N3)
    w = inputs.complex_normal(rng, (M,))
    plan = _plan(N3, M)
    assert plan.paths()["pruned_fft"]
    plan.set_nodes(to_dev(k, torch.float64))
    fh = plan.forward(to_dev(f, torch.complex64)).cpu().numpy()
    y = plan.adjoint(to_dev(w, torch.complex64)).cpu().numpy()
    plan.close()
    tol, tmax = tol_for(N3, 2.0, 4, "c64"), tol_max_for(N3, 2.0, 4, "c64")
    assert_close(fh, onfft.forward(k, f, 2.0, 4), tol, "forward", tmax)
    assert_close(y, onfft.adjoint(k, w, N3, 2.0, 4), tol, "adjoint", tmax)


def test_grad_through_pruned_fft():
    """nfft_grad (ghat from the pruned FFT) against the oracle's node gradient."""
    M = 3000
    rng = np.random.default_rng(77)
    k = inputs.uniform_nodes(rng, M, 3)
    f = inputs.complex_normal(rng, N3)
    cot = inputs.complex_normal(rng, (M,))
    plan = _plan(N3, M)
    plan.set_nodes(to_dev(k, torch.float64))
    gk = plan.grad(to_dev(f, torch.complex64), to_dev(cot, torch.complex64)).cpu().numpy()
    plan.close()
    want = onfft.node_grad(k, f, cot, 2.0, 4)
    # the complex64 node-gradient tolerance of the other gradient tests
    assert_close(gk, want, 1e-4, "grad")


def test_direct_sum_selection():
    from paper_2208_00049_gb300 import binding as B
    cases = [
        ((256,), "c128", 0, "direct"),
        ((300,), "c128", 0, "direct"),
        ((2048,), "c128", 0, "library"),         # N N~ = 2^23 > 2^20
        ((256,), "c64", 0, "library"),
        ((256,), "c128", B.NFFT_FLAG_LIBRARY_FFT, "library"),
        ((64, 64), "c128", 0, "library"),
    ]
    for N, dt, flags, want in cases:
        plan = _plan(N, 8, dt, flags)
        assert plan.paths()["fft_form"] == want, (N, dt, flags)
        plan.close()


@pytest.mark.parametrize("N,sigma", [((256,), 2.0), ((257,), 2.0), ((300,), 1.5), ((800,), 1.25)])
def test_direct_sum_steps_match_oracle(N, sigma):
    """Small 1D complex128 plans: correction + pad + FFT and inverse FFT +
    crop + correction as direct sums, element by element against the oracle's
    steps, and the whole transforms against the oracle."""
    rng = np.random.default_rng(211)
    p = onfft.Params(N, sigma, 4)
    plan = _plan(N, 600, "c128", 0, sigma)
    assert plan.paths()["fft_form"] == "direct"
    f = inputs.complex_normal(rng, N)
    plan.step_pad_fft(to_dev(f, torch.complex128))
    got = plan.grid_tensor().cpu().numpy() / _peak(p)
    assert_close(got, onfft.fft_forward(onfft.correction_pad(p, f)), 1e-13, "direct pad_fft")
    G = inputs.complex_normal(rng, p.Nt)
    plan.grid_tensor().copy_(torch.from_numpy(G))
    y = torch.empty(N, dtype=torch.complex128, device="cuda")
    plan.step_fft_crop(y)
    assert_close(y.cpu().numpy() / _peak(p), onfft.crop_correction(p, onfft.fft_adjoint(G)), 1e-13,
                 "direct fft_crop")
    case = inputs.small_case(N, 600, seed=223, sigma=sigma, m=4)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    fh = plan.forward(to_dev(case["f"], torch.complex128)).cpu().numpy()
    ya = plan.adjoint(to_dev(case["w"], torch.complex128)).cpu().numpy()
    assert_close(fh, onfft.forward(case["k"], case["f"], sigma, 4), 1e-12, "forward")
    assert_close(ya, onfft.adjoint(case["k"], case["w"], N, sigma, 4), 1e-12, "adjoint")
    plan.close()


N2 = (256, 256)


def test_pruned_2d_steps_match_oracle():
    """The 2D pruned form (N~ = 2N = 512): correction + pad + FFT and inverse
    FFT + crop + correction element by element on the full grid / output,
    the whole transforms against the oracle, and agreement with the library
    form."""
    from paper_2208_00049_gb300 import binding as B
    rng = np.random.default_rng(227)
    p = onfft.Params(N2, 2.0, 4)
    plan = _plan(N2, 8)
    assert plan.paths()["pruned_fft"]
    f = inputs.complex_normal(rng, N2)
    plan.step_pad_fft(to_dev(f, torch.complex64))
    got = plan.grid_tensor().cpu().numpy().astype(np.complex128) / _peak(p)
    tol, tmax = tol_for(N2, 2.0, 4, "c64"), tol_max_for(N2, 2.0, 4, "c64")
    assert_close(got, onfft.fft_forward(onfft.correction_pad(p, f)), tol, "2D pad_fft", tmax)
    G = inputs.complex_normal(rng, p.Nt)
    plan.grid_tensor().copy_(torch.from_numpy(G.astype(np.complex64)))
    y = torch.empty(N2, dtype=torch.complex64, device="cuda")
    plan.step_fft_crop(y)
    got = y.cpu().numpy().astype(np.complex128) / _peak(p)
    assert_close(got, onfft.crop_correction(p, onfft.fft_adjoint(G)), tol, "2D fft_crop", tmax)
    plan.close()
    grids = []
    fd = to_dev(f, torch.complex64)
    for flags in (0, B.NFFT_FLAG_LIBRARY_FFT):
        pl = _plan(N2, 8, flags=flags)
        pl.step_pad_fft(fd)
        grids.append(pl.grid_tensor().cpu().numpy())
        pl.close()
    assert rel_l2(grids[0], grids[1]) <= 2e-6
    case = inputs.small_case(N2, 20000, seed=229, m=4)
    plan = _plan(N2, 20000)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    fh = plan.forward(to_dev(case["f"], torch.complex64)).cpu().numpy()
    ya = plan.adjoint(to_dev(case["w"], torch.complex64)).cpu().numpy()
    assert_close(fh, onfft.forward(case["k"], case["f"], 2.0, 4), tol, "2D forward")
    assert_close(ya, onfft.adjoint(case["k"], case["w"], N2, 2.0, 4), tol, "2D adjoint")
    plan.close()


def test_pruned_160_steps_against_single_precision_floor():
    """The sigma = 1.25 form (N~ = 160, N = 128): correction + pad + FFT and
    inverse FFT + crop + correction on the full grid / output against the
    oracle's FP64 steps, within 1.5x the error of the library's (cuFFT)
    single-precision FFT on the same data: the deconvolution amplifies FFT
    rounding at the band edges, so the bound is a single-precision FFT's own
    floor, not a fixed number.  (numpy's complex64 FFT is not that floor: its
    error on random data, 5e-8, is close to the rounding of the output alone.)
    The whole transforms at this size run in test_gpu_parity's lean-variant
    tests."""
    rng = np.random.default_rng(233)
    p = onfft.Params(N3, 1.25, 6)
    plan = _plan(N3, 8, sigma=1.25, m=6)
    assert plan.paths()["pruned_fft"]
    f = inputs.complex_normal(rng, N3)
    plan.step_pad_fft(to_dev(f, torch.complex64))
    got = plan.grid_tensor().cpu().numpy().astype(np.complex128) / _peak(p)
    g = onfft.correction_pad(p, f)
    want = onfft.fft_forward(g)
    g32 = torch.fft.fftn(torch.from_numpy(g.astype(np.complex64)).cuda()).cpu().numpy()
    e_lib = rel_l2(g32.astype(np.complex128), want)
    assert rel_l2(got, want) <= 1.5 * e_lib, (rel_l2(got, want), e_lib)
    G = inputs.complex_normal(rng, p.Nt)
    plan.grid_tensor().copy_(torch.from_numpy(G.astype(np.complex64)))
    y = torch.empty(N3, dtype=torch.complex64, device="cuda")
    plan.step_fft_crop(y)
    got = y.cpu().numpy().astype(np.complex128) / _peak(p)
    want = onfft.crop_correction(p, onfft.fft_adjoint(G))
    G32 = torch.fft.ifftn(torch.from_numpy(G.astype(np.complex64)).cuda(), norm="forward").cpu().numpy()
    e_lib = rel_l2(onfft.crop_correction(p, G32.astype(np.complex128)), want)
    assert rel_l2(got, want) <= 1.5 * e_lib, (rel_l2(got, want), e_lib)
    plan.close()
