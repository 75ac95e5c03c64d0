"""GPU parity of the node gradient (nfft_grad, Re(conj(cot) dfhat/dk)) and of
the torch.autograd wrappers, against the FP64 oracle and finite differences.

Tolerances (relative L2): complex64 1e-4, complex128 1e-10 against the
oracle's derivative of the same approximation; the exact NDFT derivative at
m = 8 (complex128) to 1e-10; central differences (h = 1e-4, FP64) to 1e-2,
the size of their own truncation error h^2 (pi N)^2 / 6 at N = 256.
"""
import numpy as np
import pytest

from oracle import ndft as ondft
from oracle import nfft as onfft
from paper_2208_00049_gb300 import inputs

from gpu_helpers import assert_close, cdtype, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAD_TOL = {"c64": 1e-4, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _plan(N, M, m, dt, sigma=2.0):
    from paper_2208_00049_gb300.nfft import Plan
    return Plan(N, M, sigma=sigma, m=m, dtype=cdtype(dt))


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("N,M,m", [((300,), 700, 4), ((40, 36), 2500, 4), ((20, 18, 16), 4000, 4),
                                   ((33, 29), 1200, 6), ((12, 10, 14), 900, 3)])
def test_grad_matches_oracle(N, M, m, dt):
    case = inputs.small_case(N, M, seed=41, m=m)
    cot = inputs.complex_normal(np.random.default_rng(3), (M,))
    plan = _plan(N, M, m, dt)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    gk = plan.grad(to_dev(case["f"], cdtype(dt)), to_dev(cot, cdtype(dt))).cpu().numpy()
    plan.close()
    want = onfft.node_grad(case["k"], case["f"], cot, 2.0, m)
    assert_close(gk, want, GRAD_TOL[dt], "node gradient")


@pytest.mark.parametrize("tile", [(9, 9, 8), (5, 7, 9), (8, 8, 1), (16, 4, 3)])
def test_grad_3d_m4_tiles(tile):
    """3D m = 4 complex64: the gather-layout gradient kernel (value and
    derivative from the POLYNOMIAL window) on several tiles, and the generic
    kernel where the tile does not fit it (16 x 4 x 3), against the oracle."""
    N, M = (24, 20, 28), 5000
    case = inputs.small_case(N, M, seed=47, m=4)
    cot = inputs.complex_normal(np.random.default_rng(5), (M,))
    plan = _plan(N, M, 4, "c64")
    plan.set_tile(tile)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    gk = plan.grad(to_dev(case["f"], torch.complex64), to_dev(cot, torch.complex64)).cpu().numpy()
    plan.close()
    assert_close(gk, onfft.node_grad(case["k"], case["f"], cot, 2.0, 4), GRAD_TOL["c64"], "node gradient")


def test_grad_against_exact_ndft_derivative():
    N, M = (24, 20), 600
    case = inputs.small_case(N, M, seed=43, m=8)
    cot = inputs.complex_normal(np.random.default_rng(4), (M,))
    plan = _plan(N, M, 8, "c128")
    plan.set_nodes(to_dev(case["k"], torch.float64))
    gk = plan.grad(to_dev(case["f"], torch.complex128), to_dev(cot, torch.complex128)).cpu().numpy()
    plan.close()
    assert rel_l2(gk, ondft.ndft_node_grad(case["k"], case["f"], cot)) <= 1e-10


def _loss_grads(wl, dt):
    from paper_2208_00049_gb300.nfft import nfft
    plan = _plan(wl["N"], wl["M"], wl["m"], dt)
    f = to_dev(wl["f"], cdtype(dt)).requires_grad_(True)
    k = to_dev(wl["k"], torch.float64).requires_grad_(True)
    y = to_dev(wl["y"], cdtype(dt))
    r = nfft(f, k, plan) - y
    loss = (r.real ** 2 + r.imag ** 2).sum()
    loss.backward()
    out = (float(loss.detach()), f.grad.cpu().numpy(), k.grad.cpu().numpy())
    plan.close()
    return out


def test_differentiation_workload_against_oracle():
    """Workload 5: jittered radial set on 256 x 256, L = ||A(x) f - y||^2."""
    wl = inputs.differentiation()
    for dt in ("c64", "c128"):
        loss, gf, gk = _loss_grads(wl, dt)
        fh = onfft.forward(wl["k"], wl["f"], 2.0, 4)
        r = fh - wl["y"]
        assert loss == pytest.approx(float(np.sum(np.abs(r) ** 2)), rel=1e-5 if dt == "c64" else 1e-12)
        want_gf = onfft.adjoint(wl["k"], 2 * r, wl["N"], 2.0, 4)
        want_gk = onfft.node_grad(wl["k"], wl["f"], 2 * r, 2.0, 4)
        assert_close(gf, want_gf, 1e-5 if dt == "c64" else 1e-12, "grad f")
        assert_close(gk, want_gk, GRAD_TOL[dt], "grad k")


def test_differentiation_workload_finite_differences():
    """Central differences of the FP64 loss (h = 1e-4) on 64 (j, d) entries
    and along one random direction over all nodes."""
    from paper_2208_00049_gb300.nfft import Plan
    wl = inputs.differentiation()
    _, _, gk = _loss_grads(wl, "c128")
    plan = Plan(wl["N"], wl["M"], sigma=2.0, m=4, dtype=torch.complex128)
    f = to_dev(wl["f"], torch.complex128)
    y = to_dev(wl["y"], torch.complex128)

    def loss_at(k):
        plan.set_nodes(to_dev(k, torch.float64))
        r = plan.forward(f) - y
        return float((r.real ** 2 + r.imag ** 2).sum())

    h = 1e-4
    rng = np.random.default_rng(47)
    js = rng.choice(wl["M"], 32, replace=False)
    fd, an = [], []
    for j in js:
        for d in range(2):
            kp = wl["k"].copy()
            km = wl["k"].copy()
            kp[j, d] += h
            km[j, d] -= h
            fd.append((loss_at(kp) - loss_at(km)) / (2 * h))
            an.append(gk[j, d])
    assert rel_l2(np.array(an), np.array(fd)) <= 1e-2
    direction = rng.standard_normal(wl["k"].shape)
    direction /= np.linalg.norm(direction)
    dd = (loss_at(wl["k"] + h * direction) - loss_at(wl["k"] - h * direction)) / (2 * h)
    assert float(np.sum(gk * direction)) == pytest.approx(dd, rel=1e-2)
    plan.close()


def test_adjoint_autograd_against_oracle():
    """y = A(x)^H w: grad_w = A Y and grad_x = Re(conj(w) d(A Y)/dx) for upstream Y."""
    from paper_2208_00049_gb300.nfft import nfft_adjoint
    N, M = (32, 28), 2000
    case = inputs.small_case(N, M, seed=53, m=4)
    Y = inputs.complex_normal(np.random.default_rng(9), N)
    plan = _plan(N, M, 4, "c128")
    w = to_dev(case["w"], torch.complex128).requires_grad_(True)
    k = to_dev(case["k"], torch.float64).requires_grad_(True)
    yv = nfft_adjoint(w, k, plan)
    Yd = to_dev(Y, torch.complex128)
    L = (yv.real * Yd.real + yv.imag * Yd.imag).sum()   # dL/dy = Y (PyTorch convention)
    L.backward()
    assert_close(w.grad.cpu().numpy(), onfft.forward(case["k"], Y, 2.0, 4), 1e-12, "grad w")
    assert_close(k.grad.cpu().numpy(), onfft.node_grad(case["k"], Y, case["w"], 2.0, 4), 1e-10, "grad k")
    plan.close()
