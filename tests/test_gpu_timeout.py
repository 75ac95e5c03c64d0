"""The bounded wait of the 3D gather's region copy, made to run out on purpose.

The test hook NFFT_GB300_TEST_TX_EXTRA makes each CTA's mbarrier expect 16
bytes more than the TMA box delivers: the copy completes (nothing stays in
flight), the barrier's phase never does, and the wait gives up after its time
bound.  The CTA then sets the device flag and returns, and nfft_plan_sync
reports NFFT_ERR_TIMEOUT.  No fault, trap or unbounded loop is involved.
Afterwards the context must still be usable and the flag cleared.
"""
import time

import numpy as np
import pytest

from oracle import nfft as onfft
from paper_2208_00049_gb300 import inputs

from gpu_helpers import TOL, assert_close, require_gpu, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _plan(N, M):
    from paper_2208_00049_gb300.nfft import Plan
    return Plan(N, M, sigma=2.0, m=4, dtype=torch.complex64)


def test_region_copy_wait_runs_out_and_reports_timeout(monkeypatch):
    from paper_2208_00049_gb300 import binding as B
    N, M = (32, 32, 32), 20000
    case = inputs.small_case(N, M, seed=113, m=4)
    plan = _plan(N, M)
    assert plan.paths()["fast_gather"]
    plan.set_nodes(to_dev(case["k"], torch.float64))
    f = to_dev(case["f"], torch.complex64)
    fh = torch.empty(M, dtype=torch.complex64, device="cuda")
    monkeypatch.setenv("NFFT_GB300_TEST_TX_EXTRA", "16")
    t0 = time.time()
    assert B.nfft_forward(plan.handle, f.data_ptr(), fh.data_ptr()) == B.NFFT_OK
    s = B.nfft_plan_sync(plan.handle)
    elapsed = time.time() - t0
    monkeypatch.delenv("NFFT_GB300_TEST_TX_EXTRA")
    assert s == B.NFFT_ERR_TIMEOUT, B.strerror(s)
    assert elapsed < 30.0
    # the error is sticky for this plan
    assert B.nfft_forward(plan.handle, f.data_ptr(), fh.data_ptr()) == B.NFFT_ERR_TIMEOUT
    plan.close()
    # the context is intact, the flag was cleared, and a new plan is correct
    plan = _plan(N, M)
    plan.set_nodes(to_dev(case["k"], torch.float64))
    plan.forward(f, out=fh)
    assert B.nfft_plan_sync(plan.handle) == B.NFFT_OK
    assert_close(fh.cpu().numpy(), onfft.forward(case["k"], case["f"], 2.0, 4), TOL["c64"], "after timeout")
    plan.close()
    assert np.isfinite(elapsed)
