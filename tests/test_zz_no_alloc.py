"""The spreading entry point that allocates nothing (nfft_spread_noalloc),
checked through the C ABI against the plan path's scatter step on two calls
in a row.  Kept in its own file, collected last."""
import numpy as np
import pytest

from paper_2208_00049_gb300 import inputs

from gpu_helpers import assert_close, require_gpu

torch = pytest.importorskip("torch")


def _nt(N, sigma):
    return tuple(int(2 * np.ceil(sigma * n / 2.0 - 1e-12)) for n in N)


@pytest.mark.gpu
def test_spread_noalloc_matches_plan_scatter_twice():
    require_gpu()
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan

    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different sizes and data: nothing of the first
    # call's scratch may leak into the second
    for N, M, seed in [((24, 20, 28), 6000, 31), ((64, 48), 3000, 37)]:
        case = inputs.small_case(N, M, seed=seed, m=4)
        k = torch.from_numpy(case["k"]).cuda()
        w = torch.from_numpy(case["w"]).to(torch.complex64).cuda()
        out = torch.full(_nt(N, 2.0), 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
        s = B.nfft_spread_noalloc(len(N), N, 2.0, 4, M, k.data_ptr(), w.data_ptr(), out.data_ptr(), stream)
        assert s == B.NFFT_OK, B.strerror(s)
        plan = Plan(N, M, sigma=2.0, m=4, dtype=torch.complex64)
        plan.set_nodes(k)
        plan.step_scatter(w)
        ref = plan.grid_tensor().clone()
        torch.cuda.synchronize()
        assert_close(out.cpu().numpy(), ref.cpu().numpy(), 1e-5, "spread %s" % (N,))
        plan.close()

    # sizes beyond the static scratch are rejected before any work
    big = B.NFFT_NOALLOC_MAX_NODES + 1
    kb = torch.zeros((big, 1), dtype=torch.float64, device="cuda")
    wb = torch.zeros(big, dtype=torch.complex64, device="cuda")
    g = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 4, big, kb.data_ptr(), wb.data_ptr(), g.data_ptr(),
                                 stream) == B.NFFT_ERR_UNSUPPORTED
    assert B.nfft_spread_noalloc(1, (32,), 2.0, 0, 4, kb.data_ptr(), wb.data_ptr(), g.data_ptr(),
                                 stream) == B.NFFT_ERR_INVALID_ARG
