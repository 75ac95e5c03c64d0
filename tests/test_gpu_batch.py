"""Batched transforms (nfft_batch_*): 64 uneven 2D problems and 32 right-hand
sides on one radial node set, in one persistent launch per step, with CUDA
graph replay and the autotuner, against the FP64 oracle.

The oracle runs every problem's forward on 64 sampled nodes (the grid steps
at full size), the full adjoint on a few problems, and both transforms of two
right-hand sides in full; the adjoint identity <A f, w> = <f, A^H w> is
checked on every problem."""
import numpy as np
import pytest

from oracle import nfft as onfft
from paper_2208_00049_gb300 import inputs

from gpu_helpers import assert_close, require_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _flat(arrs, dtype):
    return torch.cat([torch.from_numpy(np.ascontiguousarray(a).ravel()) for a in arrs]).to(dtype).cuda()


def _split(t, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(t[o:o + n])
        o += n
    return out


def test_uneven_problems_against_oracle():
    from paper_2208_00049_gb300.nfft import Batch
    probs = inputs.batched_problems(n_problems=64)
    Ns = [p["N"] for p in probs]
    Ms = [p["M"] for p in probs]
    b = Batch(Ns, list(range(64)), Ms, sigma=2.0, m=4, dtype=torch.complex64)
    k_all = torch.from_numpy(np.concatenate([p["k"] for p in probs])).cuda()
    b.set_nodes(k_all)
    info = b.info()
    assert info["fft_classes"] <= 16 and info["n_items"] > 64
    f_all = _flat([p["f"] for p in probs], torch.complex64)
    w_all = _flat([p["w"] for p in probs], torch.complex64)
    fh = _split(b.forward(f_all).cpu().numpy(), Ms)
    y = _split(b.adjoint(w_all).cpu().numpy(), [int(np.prod(n)) for n in Ns])
    rng = np.random.default_rng(61)
    for i, p in enumerate(probs):
        sel = rng.choice(p["M"], 64, replace=False)
        assert_close(fh[i][sel], onfft.forward(p["k"][sel], p["f"], 2.0, 4), 1e-5, "forward %d" % i)
        lhs = np.vdot(p["w"], fh[i])
        rhs = np.vdot(y[i], p["f"].ravel())
        assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(p["w"]) * np.linalg.norm(fh[i])
    small = sorted(range(64), key=lambda i: Ms[i])[:3] + [int(np.argmax(Ms))]
    for i in small:
        p = probs[i]
        assert_close(y[i].reshape(p["N"]), onfft.adjoint(p["k"], p["w"], p["N"], 2.0, 4), 1e-5, "adjoint %d" % i)
    b.close()


def test_uneven_problems_register_scatter_tile():
    """The 2D register-accumulating scatter (tile 9 x 25, regions of 16 x 32)
    on the uneven batch: full adjoint on the smallest problems and the
    largest, the adjoint identity on all."""
    from paper_2208_00049_gb300.nfft import Batch
    probs = inputs.batched_problems(n_problems=24, salt=3)
    Ns = [p["N"] for p in probs]
    Ms = [p["M"] for p in probs]
    b = Batch(Ns, list(range(24)), Ms, sigma=2.0, m=4, dtype=torch.complex64)
    b.set_tile((9, 25))
    b.set_nodes(torch.from_numpy(np.concatenate([p["k"] for p in probs])).cuda())
    assert b.info()["tile"] == (9, 25)
    f_all = _flat([p["f"] for p in probs], torch.complex64)
    w_all = _flat([p["w"] for p in probs], torch.complex64)
    fh = _split(b.forward(f_all).cpu().numpy(), Ms)
    y = _split(b.adjoint(w_all).cpu().numpy(), [int(np.prod(n)) for n in Ns])
    for i, p in enumerate(probs):
        lhs = np.vdot(p["w"], fh[i])
        rhs = np.vdot(y[i], p["f"].ravel())
        assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(p["w"]) * np.linalg.norm(fh[i])
    for i in sorted(range(24), key=lambda i: Ms[i])[:3] + [int(np.argmax(Ms))]:
        p = probs[i]
        assert_close(y[i].reshape(p["N"]), onfft.adjoint(p["k"], p["w"], p["N"], 2.0, 4), 1e-5, "adjoint %d" % i)
    b.close()


def test_shared_node_set_rhs_graph_and_autotune():
    from paper_2208_00049_gb300.nfft import Batch
    rad = inputs.radial_rhs(n_rhs=32)
    k = rad["k"]
    M = k.shape[0]
    b = Batch([rad["N"]] * 32, [0] * 32, [M], sigma=2.0, m=4, dtype=torch.complex64)
    kd = torch.from_numpy(k).cuda()
    tile = b.autotune(kd)
    assert len(tile) == 2
    b.set_graph(True)
    f_all = _flat(list(rad["f"]), torch.complex64)
    w_all = _flat(list(rad["w"]), torch.complex64)
    out_f = torch.empty(32 * M, dtype=torch.complex64, device="cuda")
    out_y = torch.empty(32 * int(np.prod(rad["N"])), dtype=torch.complex64, device="cuda")
    for _ in range(3):                      # captured once, replayed
        b.forward(f_all, out_f)
        b.adjoint(w_all, out_y)
    fh = _split(out_f.cpu().numpy(), [M] * 32)
    y = _split(out_y.cpu().numpy(), [int(np.prod(rad["N"]))] * 32)
    for r in (0, 31):
        assert_close(fh[r], onfft.forward(k, rad["f"][r], 2.0, 4), 1e-5, "rhs forward %d" % r)
        assert_close(y[r].reshape(rad["N"]), onfft.adjoint(k, rad["w"][r], rad["N"], 2.0, 4), 1e-5,
                     "rhs adjoint %d" % r)
    # graph replay with new data in the same buffers
    f_all.mul_(2.0)
    b.forward(f_all, out_f)
    torch.cuda.synchronize()
    assert_close(out_f[:M].cpu().numpy(), 2 * fh[0], 1e-6, "replay")
    b.close()


def test_batch_matches_single_plans_fp64():
    """complex128 batch equals per-problem plans to 1e-12 on mixed sizes."""
    from paper_2208_00049_gb300.nfft import Batch, Plan
    probs = inputs.batched_problems(n_problems=6, sizes=(16, 32, 48))
    Ns = [p["N"] for p in probs]
    Ms = [p["M"] for p in probs]
    b = Batch(Ns, list(range(6)), Ms, sigma=2.0, m=4, dtype=torch.complex128)
    b.set_nodes(torch.from_numpy(np.concatenate([p["k"] for p in probs])).cuda())
    fh = _split(b.forward(_flat([p["f"] for p in probs], torch.complex128)).cpu().numpy(), Ms)
    y = _split(b.adjoint(_flat([p["w"] for p in probs], torch.complex128)).cpu().numpy(),
               [int(np.prod(n)) for n in Ns])
    for i, p in enumerate(probs):
        assert_close(fh[i], onfft.forward(p["k"], p["f"], 2.0, 4), 1e-12, "forward %d" % i)
        assert_close(y[i].reshape(p["N"]), onfft.adjoint(p["k"], p["w"], p["N"], 2.0, 4), 1e-12, "adjoint %d" % i)
    b.close()


def test_rank_split_sub_batches_match_full_batch():
    """The batched workload split over 2 ranks (bench.py's split, emulated
    one rank after the other on this GPU): each rank's sub-batch gives, for
    its problems, the full batch's outputs."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2208_00049_gb300.nfft import Batch
    probs = inputs.batched_problems(n_problems=64)

    def run(idx):
        ps = [probs[i] for i in idx]
        Ms = [p["M"] for p in ps]
        b = Batch([p["N"] for p in ps], list(range(len(ps))), Ms, sigma=2.0, m=4, dtype=torch.complex64)
        b.set_tile((9, 25))
        b.set_nodes(torch.from_numpy(np.concatenate([p["k"] for p in ps])).cuda())
        fh = _split(b.forward(_flat([p["f"] for p in ps], torch.complex64)).cpu().numpy(), Ms)
        y = _split(b.adjoint(_flat([p["w"] for p in ps], torch.complex64)).cpu().numpy(),
                   [int(np.prod(p["N"])) for p in ps])
        b.close()
        return dict(zip(idx, zip(fh, y)))

    full = run(list(range(64)))
    w = bench.batch_weights(probs)
    seen = set()
    for rank in range(2):
        mine = bench.split_problems(w, 2, rank)
        part = run(mine)
        for i in mine:
            assert i not in seen
            seen.add(i)
            assert_close(part[i][0], full[i][0], 1e-6, "forward %d" % i)
            assert_close(part[i][1], full[i][1], 1e-6, "adjoint %d" % i)
    assert seen == set(range(64))
