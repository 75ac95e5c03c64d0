"""The spreading entry point that allocates nothing (nfft_spread_noalloc).

Callers that cannot call cudaMalloc (code under another framework's caching
allocator, latency-critical loops that cannot take its implicit
synchronisation, fixed memory budgets) use this call; its scratch is a static
device array.  Checked through the C ABI against the oracle's adjoint
resampling step (scaled by the window peak, the normalisation the library
uses) and against the plan path's scatter step, on calls in a row with
different sizes (nothing of one call's scratch may leak into the next),
including 1D, 3D at m = 8 (the generic kernel with a region above 48 KB of
shared memory) and M = 0.  Kept in its own file, collected last."""
import numpy as np
import pytest

from oracle import nfft as onfft
from paper_2208_00049_gb300 import inputs

from gpu_helpers import assert_close, require_gpu

torch = pytest.importorskip("torch")


def _nt(N, sigma):
    return tuple(int(2 * np.ceil(sigma * n / 2.0 - 1e-12)) for n in N)


def _oracle_spread(N, m, k, w):
    p = onfft.Params(N, 2.0, m)
    peak = np.prod([float(onfft.psi(0.0, m, b)) for b in p.b])
    return onfft.resample_adjoint(p, k, w) / peak


@pytest.mark.gpu
def test_spread_noalloc_matches_oracle_and_plan_scatter():
    require_gpu()
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan

    stream = torch.cuda.current_stream().cuda_stream
    cases = [((24, 20, 28), 6000, 31, 4), ((64, 48), 3000, 37, 4), ((300,), 900, 41, 4),
             ((12, 10, 14), 1500, 43, 8), ((24, 20, 28), 6000, 31, 4)]
    for N, M, seed, m in cases:
        case = inputs.small_case(N, M, seed=seed, m=m)
        k = torch.from_numpy(case["k"]).cuda()
        w = torch.from_numpy(case["w"]).to(torch.complex64).cuda()
        out = torch.full(_nt(N, 2.0), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        s = B.nfft_spread_noalloc(len(N), N, 2.0, m, M, k.data_ptr(), w.data_ptr(), out.data_ptr(), stream)
        assert s == B.NFFT_OK, B.strerror(s)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        want = _oracle_spread(N, m, case["k"], case["w"].astype(np.complex64).astype(np.complex128))
        assert_close(got, want, 1e-5, "spread vs oracle %s m=%d" % (N, m))
        plan = Plan(N, M, sigma=2.0, m=m, dtype=torch.complex64)
        plan.set_nodes(k)
        plan.step_scatter(w)
        ref = plan.grid_tensor().clone()
        torch.cuda.synchronize()
        assert_close(got, ref.cpu().numpy(), 1e-5, "spread vs plan scatter %s" % (N,))
        plan.close()

    # no nodes: an all-zero grid (the call clears what was there)
    g0 = torch.full(_nt((20, 18), 2.0), 3.0 - 1.0j, dtype=torch.complex64, device="cuda")
    assert B.nfft_spread_noalloc(2, (20, 18), 2.0, 4, 0, 0, 0, g0.data_ptr(), stream) == B.NFFT_OK
    torch.cuda.synchronize()
    assert not torch.any(g0 != 0)

    # sizes beyond the static scratch are rejected before any work
    big = B.NFFT_NOALLOC_MAX_NODES + 1
    kb = torch.zeros((big, 1), dtype=torch.float64, device="cuda")
    wb = torch.zeros(big, dtype=torch.complex64, device="cuda")
    g = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 4, big, kb.data_ptr(), wb.data_ptr(), g.data_ptr(),
                                 stream) == B.NFFT_ERR_UNSUPPORTED
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 0, 4, kb.data_ptr(), wb.data_ptr(), g.data_ptr(),
                                 stream) == B.NFFT_ERR_INVALID_ARG
