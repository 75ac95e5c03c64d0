"""Benchmark: NFFT forward + adjoint nodes/s on one GB300 (or N replicas).

A step is one pass of the whole path over one batch: Algorithm 1
(correction + zero pad + FFT -> gather) and Algorithm 2 (scatter -> inverse
FFT + crop + correction), the FFT steps pruned and fused with the correction
where the plan qualifies (3D, complex64, N~ = 2N = 256; cuFFT between the
separate correction kernels otherwise), every kernel launched through the C
ABI, on
device-resident inputs (nodes set once: the plan's precomputation, timed
separately as set_nodes).  value = M / (mean step time) nodes/s, summed over
ranks; each rank runs an independent replica of the same workload (a single
transform does not shard: "replicas only", weak scaling).

Default workload: 3D, N = 128^3, M = 2097152 uniform nodes, sigma = 2, m = 4,
complex64 (FP32 arithmetic).  Between timed steps L2 is flushed by writing a
256 MiB buffer.  e2e repeats the step through the same C-ABI calls with
pinned HOST buffers (host<->device copies inside the timed region), pipelined
with nfft_plan_set_async; its synchronous form is reported beside it.

--impl reference times the FP64 CPU oracle (plain numpy Algorithms 1/2) on a
bounded node sample of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "NFFT fwd+adj nodes/s at 3D 128^3 (FP32, rel err <=1e-5) vs FP64 form; % HBM roofline"
UNIT = "nodes/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE_DIR = os.path.join(ROOT, "profiles")

WORKLOADS = {
    "accuracy": "accuracy",
    "batched": "batched",
    "diff": "diff",
    "tiles": "tiles",
    "3d": "3d",
    "3d_lean": "3d_lean",
    "2d_c64": "2d_c64",
    "2d_c128": "2d_c128",
    "1d": "1d",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="3d", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile", default=None,
                    help="batched workload: fixed tile shape (e.g. 9,25) instead of the autotuner's choice; "
                         "for profiling, where timings taken under the profiler would steer the autotuner")
    ap.add_argument("--cpu-sample", type=int, default=131072,
                    help="nodes in the oracle's bounded sample")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the complex128 (FP64) comparison run")
    ap.add_argument("--no-full-form", action="store_true",
                    help="skip the FULL sparse-matrix (cuSPARSE) comparison run")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="default line only: skip the other workloads measured in the same run")
    ap.add_argument("--other-steps", type=int, default=20,
                    help="timed steps of each other workload in the default line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_desc(wl):
    N = "x".join(str(n) for n in wl["N"])
    return "%s N=%s M=%d sigma=%g m=%d %s" % (wl["name"], N, wl["M"], wl["sigma"], wl["m"], wl["dtype"])


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _strip_comments(src):
    """C/C++ source without comments and with whitespace runs collapsed:
    what the compiler sees, so that editing a comment keeps the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":  # string or character literal, copied whole
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(files=None):
    """Hash of kernel sources (comments and layout excluded), recorded in the
    committed ncu summaries beside the counters taken from that code: the
    named files of the source directory (those that define the profiled
    kernels and their launch configuration), or all of them."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2208_00049_gb300", "csrc")
    names = sorted(files) if files else sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    for f in names:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary for this kernel
    and workload, or None if absent or taken on different kernel sources."""
    path = os.path.join(PROFILE_DIR, "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    mf = re.search(r"source_files:\s*([^\n]+)", text)
    files = mf.group(1).split() if mf else None
    if not mh or not mt:
        return None
    try:
        if mh.group(1) != kernel_source_hash(files):
            return None
    except OSError:
        return None
    return float(mt.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region
    (one nvidia-smi process in loop mode, every 100 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.samples = []
        self._proc = None
        self._thread = None

    def _read(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._thread = threading.Thread(target=self._read, daemon=True)
            self._thread.start()
            time.sleep(0.15)  # first sample before the timed work starts
        except Exception:
            self._proc = None
        return self

    def __exit__(self, *a):
        if self._proc is not None:
            time.sleep(0.15)
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            if self._thread is not None:
                self._thread.join(timeout=5)

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                mx = float(s[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, s[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_throughput(wl, sample):
    """Time the plain FP64 oracle (numpy, Algorithms 1/2) on the full grid with
    a node sample; returns (full-workload nodes/s, details).  Grid steps
    (deconvolution, two FFTs) run once at full size; node steps (gather,
    scatter) scale linearly in the number of nodes, so the full-workload time
    is t_grid + t_nodes * M / sample."""
    import numpy as np
    from oracle import nfft as onfft
    Ms = min(int(sample), wl["M"])
    k = wl["k"][:Ms]
    w = wl["w"][:Ms]
    p = onfft.Params(wl["N"], wl["sigma"], wl["m"])
    t0 = time.perf_counter()
    g = onfft.correction_pad(p, wl["f"])
    t1 = time.perf_counter()
    gh = onfft.fft_forward(g)
    t2 = time.perf_counter()
    onfft.resample(p, k, gh)
    t3 = time.perf_counter()
    ga = onfft.resample_adjoint(p, k, w)
    t4 = time.perf_counter()
    gg = onfft.fft_adjoint(ga)
    t5 = time.perf_counter()
    onfft.crop_correction(p, gg)
    t6 = time.perf_counter()
    t_grid = (t1 - t0) + (t2 - t1) + (t5 - t4) + (t6 - t5)
    t_nodes = (t3 - t2) + (t4 - t3)
    full = t_grid + t_nodes * wl["M"] / Ms
    del np
    return wl["M"] / full, {
        "sample": "full %s grid, %d of %d nodes; node steps scaled by M/sample" % (
            "x".join(str(n) for n in wl["N"]), Ms, wl["M"]),
        "t_grid_s": round(t_grid, 3), "t_nodes_s": round(t_nodes, 3), "t_full_est_s": round(full, 3),
        "wall_s": round(t6 - t0, 3)}


def cpu_cores_used():
    # numpy's FFT (pocketfft) and element-wise kernels run on one thread.
    return 1


def host_cpu():
    """CPU model name and the cores this process may use."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return {"model": model or "unknown", "nproc": cores}


def _oracle_node_worker(task):
    """One process of the all-core oracle: the oracle's gather and scatter
    steps on a chunk of nodes; the gather reads the shared grid, the scatter
    writes this worker's partial grid into its own shared block."""
    import numpy as np
    from multiprocessing import shared_memory
    from oracle import nfft as onfft
    grid_name, part_name, shape, N, sigma, m, k, w = task
    gsh = shared_memory.SharedMemory(name=grid_name)
    psh = shared_memory.SharedMemory(name=part_name)
    try:
        gh = np.ndarray(shape, dtype=np.complex128, buffer=gsh.buf)
        part = np.ndarray(shape, dtype=np.complex128, buffer=psh.buf)
        p = onfft.Params(N, sigma, m)
        fh = onfft.resample(p, k, gh)
        part[...] = onfft.resample_adjoint(p, k, w)
        return int(fh.shape[0])
    finally:
        del gh, part
        gsh.close()
        psh.close()


def _oracle_warm(_):
    from oracle import nfft  # noqa: F401  (import once per worker before timing)
    return 0


def oracle_all_cores(wl, procs=None, max_nodes=None):
    """The unchanged FP64 oracle on every host core: the grid steps
    (correction + pad, FFT, inverse FFT, crop + correction; numpy, one core)
    at full size, and the node steps (gather and scatter) on the node set split
    into one chunk per process (spawned processes, the grid in shared memory),
    the partial grids of the scatter summed at the end.  Times the full node
    set unless max_nodes caps it (then scaled by M / nodes).  Returns
    (nodes/s for the full workload, details)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    from oracle import nfft as onfft
    info = host_cpu()
    P = max(1, min(int(procs or info["nproc"]), 64))
    M = wl["M"]
    n = M if not max_nodes else min(M, int(max_nodes))
    p = onfft.Params(wl["N"], wl["sigma"], wl["m"])
    t0 = time.perf_counter()
    g = onfft.correction_pad(p, wl["f"])
    gh = onfft.fft_forward(g)
    t_grid_fwd = time.perf_counter() - t0
    shape = gh.shape
    nbytes = gh.nbytes
    gsh = shared_memory.SharedMemory(create=True, size=nbytes)
    parts = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(P)]
    try:
        np.ndarray(shape, dtype=np.complex128, buffer=gsh.buf)[...] = gh
        bounds = np.linspace(0, n, P + 1).astype(int)
        tasks = [(gsh.name, parts[i].name, shape, wl["N"], wl["sigma"], wl["m"],
                  wl["k"][bounds[i]:bounds[i + 1]], wl["w"][bounds[i]:bounds[i + 1]]) for i in range(P)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(P) as pool:
            pool.map(_oracle_warm, range(P))
            t1 = time.perf_counter()
            pool.map(_oracle_node_worker, tasks)
            acc = np.zeros(shape, dtype=np.complex128)
            for ps in parts:
                acc += np.ndarray(shape, dtype=np.complex128, buffer=ps.buf)
            t_nodes = time.perf_counter() - t1
        t2 = time.perf_counter()
        onfft.crop_correction(p, onfft.fft_adjoint(acc))
        t_grid_adj = time.perf_counter() - t2
    finally:
        for sh in [gsh] + parts:
            sh.close()
            sh.unlink()
    t_full = t_grid_fwd + t_grid_adj + t_nodes * M / n
    return M / t_full, {
        "cores": P, "cpu_model": info["model"], "nproc": info["nproc"],
        "sample": ("full %s grid, %s; node steps in %d spawned processes (grid in shared memory, partial "
                   "scatter grids summed), grid steps on one core" % (
                       "x".join(str(v) for v in wl["N"]),
                       "all %d nodes" % M if n == M else "%d of %d nodes scaled by M/sample" % (n, M), P)),
        "t_grid_s": round(t_grid_fwd + t_grid_adj, 3), "t_nodes_s": round(t_nodes, 3),
        "t_full_s": round(t_full, 3)}


REF_BUDGET_S = 90.0  # timed part of a --impl reference run, whatever --steps asks for


def _oracle_grid_s(wl, p):
    """Seconds for the oracle's full-size grid steps (correction + pad, FFT,
    adjoint FFT, crop + correction)."""
    from oracle import nfft as onfft
    t0 = time.perf_counter()
    g = onfft.correction_pad(p, wl["f"])
    gh = onfft.fft_forward(g)
    gg = onfft.fft_adjoint(gh)
    onfft.crop_correction(p, gg)
    return time.perf_counter() - t0, gh


def _oracle_nodes_s(wl, p, gh, lo, n):
    """Seconds for the oracle's node steps (gather, scatter) on nodes lo .. lo + n."""
    from oracle import nfft as onfft
    k = wl["k"][lo:lo + n]
    w = wl["w"][lo:lo + n]
    t0 = time.perf_counter()
    onfft.resample(p, k, gh)
    onfft.resample_adjoint(p, k, w)
    return time.perf_counter() - t0


def reference_plan(t_grid, t_fixed, s_per_node, steps, M, cap, budget=REF_BUDGET_S):
    """How a --impl reference run fits its time budget: whether the grid steps
    are re-timed in every step (while steps x t_grid stays within a quarter of
    the budget; otherwise their one full-size timing is used for every step)
    and how many nodes each step's node sample holds (what is left of the
    budget per step after the grid steps and the node steps' fixed part,
    between 1024 and min(cap, M) nodes)."""
    steps = max(1, int(steps))
    grid_each = steps * t_grid <= 0.25 * budget
    per_step = budget / steps - (t_grid if grid_each else 0.0) - t_fixed
    n = int(per_step / max(s_per_node, 1e-12))
    return grid_each, max(1024, min(n, int(cap), int(M)))


def reference_estimate(t_grid, t_fixed, t_nodes, n, M):
    """Full-workload oracle seconds from one step: the grid steps, the node
    steps' fixed part (the adjoint's full-grid allocation, once per call) and
    their per-node part measured on n nodes, scaled to M."""
    per_node = max(t_nodes - t_fixed, 0.0) / n
    return t_grid + t_fixed + per_node * M


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (plain numpy Algorithms 1/2) on
    the host cores, timed like the GPU arm's steps.  A step is the full-size
    grid steps plus the node steps on a node sample, scaled to M; the sample
    size (and whether the grid steps are re-timed each step) follows from a
    fixed time budget, so the run ends within minutes for any --steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import nfft as onfft
    from paper_2208_00049_gb300 import inputs
    # single-problem workloads time the oracle on themselves; the others
    # (batched, accuracy, tiles, diff) on the default 3D workload
    single = ("1d", "2d_c64", "2d_c128", "3d", "3d_lean")
    wl = inputs.workload(args.workload if args.workload in single else "3d")
    M = wl["M"]
    p = onfft.Params(wl["N"], wl["sigma"], wl["m"])
    _oracle_grid_s(wl, p)  # first touch of the full-size arrays and FFT set-up, not timed
    t_grid, gh = _oracle_grid_s(wl, p)
    # node steps = fixed part + per-node part: two sample sizes, best of two each
    na, nb = min(1024, M), min(4096, M)
    ta = min(_oracle_nodes_s(wl, p, gh, 0, na) for _ in range(2))
    tb = min(_oracle_nodes_s(wl, p, gh, 0, nb) for _ in range(2))
    s_per_node = max((tb - ta) / (nb - na), 1e-9) if nb > na else tb / nb
    t_fixed = max(ta - s_per_node * na, 0.0)
    grid_each, Ms = reference_plan(t_grid, t_fixed, s_per_node, args.steps, M, args.cpu_sample)
    for i in range(max(1, args.warmup)):
        _oracle_nodes_s(wl, p, gh, 0, min(Ms, 4096))
    vals = []
    t_loop = time.perf_counter()
    for i in range(max(1, args.steps)):
        tg = _oracle_grid_s(wl, p)[0] if grid_each else t_grid
        lo = (i * Ms) % max(1, M - Ms + 1)
        tn = _oracle_nodes_s(wl, p, gh, lo, Ms)
        vals.append(M / reference_estimate(tg, t_fixed, tn, Ms, M))
    t_loop = time.perf_counter() - t_loop
    value = statistics.median(vals)
    # a step is the bounded sample actually run (its wall time), not the
    # full-workload time that value extrapolates to
    ms_step = 1e3 * t_loop / max(1, args.steps)
    sample = ("full %s grid (grid steps %s), %d of %d nodes per step; the node steps' per-node part "
              "scaled by M/sample, their fixed part (%.3f s) counted once" % (
                  "x".join(str(n) for n in wl["N"]),
                  "timed each step" if grid_each else "timed once at full size", Ms, M, t_fixed))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64, uniform nodes)",
        "config": {"workload": workload_desc(wl), "parallelism": "none (host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": sample, "cpu_model": host_cpu()["model"], "nproc": host_cpu()["nproc"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_detail": {"t_grid_s": round(t_grid, 3), "t_node_fixed_s": round(t_fixed, 4),
                          "s_per_node": s_per_node, "nodes_per_step": Ms, "grid_timed_each_step": grid_each,
                          "full_workload_s_per_step_estimate": round(M / value, 3),
                          "timed_loop_s": round(t_loop, 3)},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def algorithmic_bytes(wl, kernel):
    """Bytes a kernel must move at minimum (complex64 = 8 B, FP32 coordinate
    = 4 B): the grid once, the nodes' coordinates once, fhat once."""
    import numpy as np
    grid = 8 * int(np.prod([2 * int(np.ceil(wl["sigma"] * n / 2.0 - 1e-12)) for n in wl["N"]]))
    M, D = wl["M"], len(wl["N"])
    nvals = 8 * int(np.prod(wl["N"]))
    if kernel in ("gather", "scatter"):
        return grid + M * (4 * D + 8)
    if kernel in ("deconv_pad", "pad_fft", "fft_crop"):
        # f read (or y written) once and the grid written (or read) once
        return grid + nvals
    if kernel == "crop_deconv":
        return 2 * nvals
    raise KeyError(kernel)


def aggregate_replicas(local_ms_total, units_per_rank, steps):
    """Whole-job numbers for independent replicas (one per rank): the slowest
    rank's total time (max over ranks, as the timing rules ask) and the units
    of all ranks over it.  Works with any initialised process group (NCCL on
    GPUs, gloo in the CPU tests); world size 1 needs none."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    total = float(local_ms_total)
    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    ms_per_step = total / steps
    return {"world": world, "ms_total_max": total, "ms_per_step": ms_per_step,
            "value": world * units_per_rank / (ms_per_step * 1e-3)}


def split_problems(weights, world, rank):
    """Indices of the independent problems rank `rank` of `world` runs: each
    problem goes to exactly one rank, largest first to the least-loaded rank
    (ties to the lower rank), so every rank's share of the total weight is
    within one problem of the mean.  Host logic only."""
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    load = [0.0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += float(weights[i])
    return [i for i in range(len(weights)) if owner[i] == rank]


def aggregate_split(local_ms_total, local_units, steps):
    """Whole-job numbers when ranks share one workload (strong scaling): the
    slowest rank's total time and the units of all ranks over it.  Works with
    any initialised process group; world size 1 needs none."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    total, units = float(local_ms_total), float(local_units)
    if world > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([units], dtype=torch.float64, device=dev)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        total, units = float(t.item()), float(u.item())
    ms_per_step = total / steps
    return {"world": world, "ms_total_max": total, "ms_per_step": ms_per_step, "units": units,
            "value": units / (ms_per_step * 1e-3)}


def time_steps(step_fn, steps, warmup, stream, flush):
    """Mean ms of step_fn over `steps` event-timed runs (L2 flushed before each)."""
    import torch
    for _ in range(warmup):
        flush.zero_()
        step_fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        step_fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def fp64_form(wl, fhat32, steps, warmup, flush):
    """The FP64 form (complex128 plan: the generic gather in FP64 and the
    FP64 scatter that owns region points by residue class) on the same
    workload: throughput and the FP32 result's distance to it."""
    import numpy as np
    import torch
    from paper_2208_00049_gb300.nfft import Plan
    stream = torch.cuda.current_stream()
    plan = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=torch.complex128)
    plan.set_nodes(torch.from_numpy(wl["k"]).cuda())
    f = torch.from_numpy(wl["f"]).cuda()
    w = torch.from_numpy(wl["w"]).cuda()
    fh = torch.empty(wl["M"], dtype=torch.complex128, device="cuda")
    y = torch.empty(wl["N"], dtype=torch.complex128, device="cuda")

    def step():
        plan.forward(f, fh)
        plan.adjoint(w, y)
    ms = time_steps(step, steps, warmup, stream, flush)
    ref = fh.cpu().numpy()
    plan.close()
    err = float(np.linalg.norm(fhat32.astype(np.complex128) - ref) / np.linalg.norm(ref))
    return {"value": wl["M"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": round(ms, 3), "dtype": "f64",
            "steps": steps}, ref, err


def full_matrix_form(wl, steps, warmup, flush):
    """The FULL-precomputation form (the paper's GPU prototype: the sparse
    matrix B on the device, applied with cuSPARSE) on the same workload."""
    import torch
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan
    stream = torch.cuda.current_stream()
    dt = torch.complex64 if wl["dtype"] == "c64" else torch.complex128
    plan = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=dt, flags=B.NFFT_FLAG_FULL_MATRIX)
    k = torch.from_numpy(wl["k"]).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plan.set_nodes(k)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    f = torch.from_numpy(wl["f"]).to(dt).cuda()
    w = torch.from_numpy(wl["w"]).to(dt).cuda()
    fh = torch.empty(wl["M"], dtype=dt, device="cuda")
    y = torch.empty(wl["N"], dtype=dt, device="cuda")
    h = plan.handle

    def step():
        B.check(B.nfft_step_pad_fft(h, f.data_ptr()))
        B.check(B.nfft_step_gather(h, fh.data_ptr()))
        B.check(B.nfft_step_scatter(h, w.data_ptr()))
        B.check(B.nfft_step_fft_crop(h, y.data_ptr()))
    ms = time_steps(step, steps, warmup, stream, flush)
    plan.close()
    nnz = wl["M"] * (2 * wl["m"]) ** len(wl["N"])
    return {"value": wl["M"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": round(ms, 3), "steps": steps,
            "set_nodes_ms_incl_matrix_build": round(build_ms, 2), "nnz": nnz}


def ndft_sample_error(wl, fhat, n=48, seed=11):
    """Relative L2 error of fhat against the exact FP64 NDFT (oracle) on n sampled nodes."""
    import numpy as np
    from oracle import ndft as ondft
    rng = np.random.default_rng(seed)
    sel = rng.choice(wl["M"], n, replace=False)
    ex = ondft.ndft(wl["k"][sel], wl["f"])
    return float(np.linalg.norm(fhat[sel] - ex) / np.linalg.norm(ex))


def batch_weights(probs):
    """Work of each batched problem: its nodes plus its oversampled grid points."""
    return [p["M"] + 4 * p["N"][0] * p["N"][1] for p in probs]


def measure_batched(steps, warmup, flush, tile=None, which=None, clock_gpu=None):
    """Workload 4: the given problems (default: all 64) of the uneven 2D batch
    in one persistent launch per step, graph-captured, tile from the
    autotuner unless given.  Returns a dict (ms per step, nodes, ...)."""
    import numpy as np
    import torch
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Batch
    probs = inputs.batched_problems(n_problems=64)
    which = list(range(len(probs))) if which is None else list(which)
    probs = [probs[i] for i in which]
    Ns = [p["N"] for p in probs]
    Ms = [p["M"] for p in probs]
    b = Batch(Ns, list(range(len(probs))), Ms, sigma=2.0, m=4, dtype=torch.complex64)
    k_all = torch.from_numpy(np.concatenate([p["k"] for p in probs])).cuda()
    if tile:
        b.set_tile(tile)
        b.set_nodes(k_all)
    else:
        tile = b.autotune(k_all)
    b.set_graph(True)
    f_all = torch.cat([torch.from_numpy(p["f"].ravel()) for p in probs]).to(torch.complex64).cuda()
    w_all = torch.cat([torch.from_numpy(p["w"]) for p in probs]).to(torch.complex64).cuda()
    fh = torch.empty(sum(Ms), dtype=torch.complex64, device="cuda")
    y = torch.empty(f_all.numel(), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        b.forward(f_all, fh)
        b.adjoint(w_all, y)
    clocks = None
    if clock_gpu is not None:
        with ClockSampler(clock_gpu) as clk:
            ms = time_steps(step, steps, max(3, warmup), stream, flush)
        clocks = clk.summary()
    else:
        ms = time_steps(step, steps, max(3, warmup), stream, flush)
    info = b.info()
    b.close()
    return {"ms": ms, "M": sum(Ms), "problems": which, "tile": list(tile), "info": info, "clocks": clocks}


def run_batched(args):
    """Workload 4: 64 uneven 2D problems in one persistent launch per step,
    graph-captured, autotuned tile (nodes/s summed over the problems).  With
    N ranks the problems are split over the ranks (no collective on the data
    path): each rank runs its share as one batch, the job time is the max
    over ranks and the value sums all ranks' nodes (strong scaling)."""
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_00049_gb300 import inputs
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    which = split_problems(batch_weights(inputs.batched_problems(n_problems=64)), world, rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile else None
    if world > 1:
        dist.barrier()
    r = measure_batched(args.steps, args.warmup, flush, tile=tile, which=which, clock_gpu=local)
    agg = aggregate_split(r["ms"] * args.steps, r["M"], args.steps)
    if rank == 0:
        line = {"metric": "batched NFFT fwd+adj nodes/s (64 uneven 2D problems, one launch per step)",
                "value": agg["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(agg["ms_per_step"], 4), "higher_is_better": True,
                "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded PCG64)",
                "config": {"workload": "batched 64 x 2D N in {64..512}^2, M = N1 N2 U(0.5,2), total M = %d"
                           % int(agg["units"]),
                           "split": "problems split over ranks (largest first to the least-loaded rank)"
                                    if world > 1 else "one batch",
                           "rank0_problems": len(r["problems"]), "tile": r["tile"],
                           "tile_from": "--tile" if args.tile else "autotuner",
                           "work_items": r["info"]["n_items"], "fft_classes": r["info"]["fft_classes"],
                           "graph": True, "l2": "flushed between steps (256 MiB write)"},
                "clocks": r["clocks"]}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def measure_diff(steps, warmup, flush, clock_gpu=None):
    """Workload 5 (differentiation): one loss-and-gradient step on the 2D
    256 x 256 problem with the jittered 402 x 512 radial node set:
    r = A(x) f - y (nfft_forward), then grad_f = A^H (2 r) (nfft_adjoint)
    and grad_x = Re(conj(2 r) d(A(x) f)/dx) (nfft_grad), all through the C
    ABI; the residual 2 (fhat - y) is the caller's loss, computed with torch.
    complex64 beside complex128, and the complex64 gradients' relative L2
    error against the complex128 ones."""
    import numpy as np
    import torch
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan
    wl = inputs.differentiation()
    M, N = wl["M"], wl["N"]
    stream = torch.cuda.current_stream()
    k = torch.from_numpy(wl["k"]).cuda()
    ms, grads, clocks = {}, {}, None
    for name, dt in (("c64", torch.complex64), ("c128", torch.complex128)):
        plan = Plan(N, M, sigma=wl["sigma"], m=wl["m"], dtype=dt)
        plan.set_nodes(k)
        f = torch.from_numpy(wl["f"]).to(dt).cuda()
        y = torch.from_numpy(wl["y"]).to(dt).cuda()
        fh = torch.empty(M, dtype=dt, device="cuda")
        cot = torch.empty(M, dtype=dt, device="cuda")
        gf = torch.empty(N, dtype=dt, device="cuda")
        gk = torch.empty((M, 2), dtype=plan.real_dtype, device="cuda")

        def step():
            plan.forward(f, out=fh)
            torch.sub(fh, y, out=cot)
            cot.mul_(2)
            plan.adjoint(cot, out=gf)
            plan.grad(f, cot, out=gk)
        n = steps if name == "c64" else max(10, min(steps, 50))
        if name == "c64" and clock_gpu is not None:
            with ClockSampler(clock_gpu) as clk:
                ms[name] = time_steps(step, n, max(3, warmup), stream, flush)
            clocks = clk.summary()
        else:
            ms[name] = time_steps(step, n, max(3, warmup), stream, flush)
        plan.sync()
        grads[name] = (gf.cpu().numpy().astype(np.complex128), gk.cpu().numpy().astype(np.float64))
        plan.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"M": M, "ms": ms, "clocks": clocks,
            "accuracy": {"rel_l2_grad_f_fp32_vs_fp64": rel(grads["c64"][0], grads["c128"][0]),
                         "rel_l2_grad_x_fp32_vs_fp64": rel(grads["c64"][1], grads["c128"][1])}}


def run_diff(args):
    """Workload 5 as its own line (see measure_diff)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    r = measure_diff(args.steps, args.warmup, flush, clock_gpu=local)
    M, ms = r["M"], r["ms"]
    line = {"metric": "NFFT loss + gradients (f and nodes) nodes/s, 2D 256^2, jittered radial set",
            "value": M / (ms["c64"] * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms["c64"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded PCG64)",
            "config": {"workload": "differentiation 2D N=256x256 M=%d (402 spokes x 512, angle jitter 1e-3) "
                                   "sigma=2 m=4" % M,
                       "step": "nfft_forward, residual, nfft_adjoint, nfft_grad",
                       "l2": "flushed between steps (256 MiB write)"},
            "fp64_form": {"value": M / (ms["c128"] * 1e-3), "unit": UNIT, "ms_per_step": round(ms["c128"], 4),
                          "dtype": "f64"},
            "accuracy": r["accuracy"], "clocks": r["clocks"]}
    print(json.dumps(line))


def api_timing(plan, f, w, fh, y, steps, flush, stream):
    """One forward + one adjoint through the public calls (nfft_forward,
    nfft_adjoint) on device buffers, from an idle GPU (synchronised before
    each pair), so that the time includes the host's launch latency: direct
    launches against one graph replay per call (nfft_plan_set_graph), and
    the relative L2 difference of the two modes' results."""
    import torch
    out = {}
    res = {}
    for mode in ("direct", "graph"):
        plan.set_graph(mode == "graph")
        for _ in range(3):
            plan.forward(f, out=fh)
            plan.adjoint(w, out=y)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.forward(f, out=fh)
            plan.adjoint(w, out=y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[mode + "_ms"] = round(statistics.median(ms), 4)
        res[mode] = (fh.clone(), y.clone())
    plan.set_graph(False)
    # atomics make the adjoint's summation order vary between runs
    out["graph_vs_direct_rel_l2"] = max(
        float((res["graph"][i] - res["direct"][i]).abs().pow(2).sum().sqrt()
              / res["direct"][i].abs().pow(2).sum().sqrt()) for i in range(2))
    return out


def measure_single(name, steps, warmup, flush, clock_gpu=None, cpu_oracle=False):
    """One single-problem workload through the step ABI (correction + pad +
    FFT, gather, scatter, inverse FFT + crop + correction), like the default
    line: ms per step and per kernel, nodes/s, accuracy against the exact
    NDFT on sampled nodes / outputs, the complex64 result against the
    complex128 form of the same workload, and (cpu_oracle) the FP64 oracle
    timed on the full workload on one core."""
    import numpy as np
    import torch
    from oracle import ndft as ondft
    from oracle import nfft as onfft
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan
    wl = inputs.workload(name)
    dt = torch.complex64 if wl["dtype"] == "c64" else torch.complex128
    stream = torch.cuda.current_stream()
    N, M = wl["N"], wl["M"]

    def build(dtype):
        plan = Plan(N, M, sigma=wl["sigma"], m=wl["m"], dtype=dtype)
        plan.set_nodes(torch.from_numpy(wl["k"]).cuda())
        return plan
    plan = build(dt)
    h = plan.handle
    f_d = torch.from_numpy(wl["f"]).to(dt).cuda()
    w_d = torch.from_numpy(wl["w"]).to(dt).cuda()
    fh = torch.empty(M, dtype=dt, device="cuda")
    y = torch.empty(N, dtype=dt, device="cuda")
    names = ["pad_fft", "gather", "scatter", "fft_crop"]

    def step(evs):
        evs[0].record(stream)
        B.check(B.nfft_step_pad_fft(h, f_d.data_ptr()))
        evs[1].record(stream)
        B.check(B.nfft_step_gather(h, fh.data_ptr()))
        evs[2].record(stream)
        B.check(B.nfft_step_scatter(h, w_d.data_ptr()))
        evs[3].record(stream)
        B.check(B.nfft_step_fft_crop(h, y.data_ptr()))
        evs[4].record(stream)
    for _ in range(max(3, warmup)):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(5)])
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]

    def timed():
        for e in evs:
            flush.zero_()
            step(e)
        torch.cuda.synchronize()
    clocks = None
    if clock_gpu is not None:
        with ClockSampler(clock_gpu) as clk:
            timed()
        clocks = clk.summary()
    else:
        timed()
    B.check(B.nfft_plan_sync(h))
    step_ms = statistics.mean(e[0].elapsed_time(e[-1]) for e in evs)
    kern = {n: round(statistics.mean(e[j].elapsed_time(e[j + 1]) for e in evs), 4) for j, n in enumerate(names)}
    fh_np, y_np = fh.cpu().numpy().astype(np.complex128), y.cpu().numpy().astype(np.complex128)
    api = api_timing(plan, f_d, w_d, fh, y, steps, flush, stream)
    plan.close()
    # accuracy: exact NDFT on sampled nodes and outputs
    rng = np.random.default_rng(11)
    ns = min(M, 16 if len(N) == 3 else 64)
    sel = rng.choice(M, ns, replace=False)
    ex = ondft.ndft(wl["k"][sel], wl["f"])
    flat = rng.choice(int(np.prod(N)), ns, replace=False)
    idx = np.unravel_index(flat, N)
    nn = np.stack([idx[d] - N[d] // 2 for d in range(len(N))], axis=1).astype(float)
    exa = np.empty(ns, complex)
    for a in range(0, ns, 8):
        ph = nn[a:a + 8] @ wl["k"].T
        ph -= np.floor(ph)
        exa[a:a + 8] = np.exp(2j * np.pi * ph) @ wl["w"]
    acc = {"rel_l2_fwd_vs_ndft_sampled": float(np.linalg.norm(fh_np[sel] - ex) / np.linalg.norm(ex)),
           "rel_l2_adj_vs_ndft_sampled": float(np.linalg.norm(y_np[idx] - exa) / np.linalg.norm(exa)),
           "ndft_samples": ns}
    fp64 = None
    if dt == torch.complex64:
        p64 = build(torch.complex128)
        ref = p64.forward(torch.from_numpy(wl["f"]).cuda()).cpu().numpy()
        p64.close()
        acc["rel_l2_fwd_fp32_vs_fp64_form"] = float(np.linalg.norm(fh_np - ref) / np.linalg.norm(ref))
    out = {"workload": workload_desc(wl), "steps": steps, "ms_per_step": round(step_ms, 4),
           "nodes_per_s": M / (step_ms * 1e-3), "kernels_ms": kern, "accuracy": acc, "clocks": clocks,
           "dtype": "f32" if dt == torch.complex64 else "f64", "api_forward_adjoint": api}
    if cpu_oracle:
        t0 = time.perf_counter()
        onfft.forward(wl["k"], wl["f"], wl["sigma"], wl["m"])
        onfft.adjoint(wl["k"], wl["w"], N, wl["sigma"], wl["m"])
        t = time.perf_counter() - t0
        out["cpu_oracle"] = {"value": M / t, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "full workload (all %d nodes), forward + adjoint" % M}
    del fp64
    return out


def compensated_form(name, steps, warmup, flush):
    """NFFT_FLAG_COMPENSATED beside the plain form on one workload: the
    scatter step's time (L2 flushed) and the spread grid's relative L2
    distance to the complex128 plan's grid (FP64 sums of the same terms)."""
    import numpy as np
    import torch
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan
    wl = inputs.workload(name)
    stream = torch.cuda.current_stream()
    k = torch.from_numpy(wl["k"]).cuda()
    w32 = torch.from_numpy(wl["w"]).to(torch.complex64).cuda()
    ref = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=torch.complex128)
    ref.set_nodes(k)
    ref.step_scatter(w32.to(torch.complex128))
    g64 = ref.grid_tensor().cpu().numpy()
    ref.close()
    out = {"workload": workload_desc(wl)}
    for label, flags in (("plain", 0), ("compensated", B.NFFT_FLAG_COMPENSATED)):
        plan = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=torch.complex64, flags=flags)
        plan.set_nodes(k)
        h = plan.handle
        ms = time_steps(lambda: B.check(B.nfft_step_scatter(h, w32.data_ptr())), steps, warmup, stream, flush)
        g = plan.grid_tensor().cpu().numpy().astype(np.complex128)
        out[label] = {"scatter_ms": round(ms, 4), "fast_kernel": plan.paths()["fast_scatter"],
                      "grid_rel_l2_vs_fp64_sums": float(np.linalg.norm(g - g64) / np.linalg.norm(g64))}
        plan.close()
    return out


def window_modes_form(wl, steps, warmup, flush, ref64=None):
    """The window modes of Sec. 3.7.4 on one workload: DIRECT, LINEAR and
    POLYNOMIAL on the same (generic) kernels (plan flags), beside the default
    plan's specialised kernels (POLYNOMIAL): gather and scatter step times
    and the forward's relative L2 distance to the FP64 form (if given)."""
    import numpy as np
    import torch
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300.nfft import Plan
    dt = torch.complex64 if wl["dtype"] == "c64" else torch.complex128
    stream = torch.cuda.current_stream()
    k = torch.from_numpy(wl["k"]).cuda()
    f = torch.from_numpy(wl["f"]).to(dt).cuda()
    w = torch.from_numpy(wl["w"]).to(dt).cuda()
    fh = torch.empty(wl["M"], dtype=dt, device="cuda")
    out = {"workload": workload_desc(wl)}
    modes = (("default (specialised kernels, POLYNOMIAL)", 0), ("DIRECT", B.NFFT_FLAG_WINDOW_DIRECT),
             ("LINEAR", B.NFFT_FLAG_WINDOW_LINEAR), ("POLYNOMIAL", B.NFFT_FLAG_WINDOW_POLYNOMIAL))
    for name, flag in modes:
        try:
            plan = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=dt, flags=flag)
        except Exception as exc:
            out[name] = {"unavailable": str(exc)}
            continue
        plan.set_nodes(k)
        h = plan.handle
        B.check(B.nfft_step_pad_fft(h, f.data_ptr()))
        tg = time_steps(lambda: B.check(B.nfft_step_gather(h, fh.data_ptr())), steps, warmup, stream, flush)
        res = fh.cpu().numpy().astype(np.complex128)
        ts = time_steps(lambda: B.check(B.nfft_step_scatter(h, w.data_ptr())), steps, warmup, stream, flush)
        entry = {"gather_ms": round(tg, 4), "scatter_ms": round(ts, 4), "paths": plan.paths()}
        if ref64 is not None:
            entry["rel_l2_fwd_vs_fp64_form"] = float(np.linalg.norm(res - ref64) / np.linalg.norm(ref64))
        out[name] = entry
        plan.close()
    return out


def other_configs(steps, warmup, flush, gpu):
    """The other workloads, measured in the same run as the headline line."""
    import torch
    out = {}
    for name in ("3d_lean", "2d_c64", "2d_c128", "1d"):
        try:
            out[name] = measure_single(name, steps, warmup, flush, clock_gpu=gpu,
                                       cpu_oracle=name in ("2d_c64", "2d_c128", "1d"))
        except Exception as exc:
            out[name] = {"unavailable": str(exc)}
        torch.cuda.synchronize()
    try:
        out["2d_c64"]["compensated_form"] = compensated_form("2d_c64", steps, 2, flush)
    except Exception as exc:
        out["2d_c64"]["compensated_form"] = {"unavailable": str(exc)}
    try:
        r = measure_batched(steps, warmup, flush, clock_gpu=gpu)
        out["batched"] = {"workload": "64 uneven 2D problems, graph replay, autotuned tile %s" % (r["tile"],),
                          "ms_per_step": round(r["ms"], 4), "nodes_per_s": r["M"] / (r["ms"] * 1e-3),
                          "M": r["M"], "work_items": r["info"]["n_items"], "clocks": r["clocks"]}
    except Exception as exc:
        out["batched"] = {"unavailable": str(exc)}
    try:
        r = measure_diff(steps, warmup, flush, clock_gpu=gpu)
        out["diff"] = {"workload": "differentiation 2D 256^2, %d jittered radial nodes" % r["M"],
                       "ms_per_step": round(r["ms"]["c64"], 4), "nodes_per_s": r["M"] / (r["ms"]["c64"] * 1e-3),
                       "fp64_form_nodes_per_s": r["M"] / (r["ms"]["c128"] * 1e-3), "accuracy": r["accuracy"],
                       "clocks": r["clocks"]}
    except Exception as exc:
        out["diff"] = {"unavailable": str(exc)}
    return out


def run_accuracy(args):
    """Figs. 1-2 analogue on the GPU: relative errors (L2 and the paper's
    infinity norm) of the direct and adjoint NFFT against the exact NDFT for
    m = 2..10, 2D N = 128^2 with M = |I_N| random nodes, sigma = 2, complex64
    and complex128: 2m points (default kernels, and the DIRECT, LINEAR and
    POLYNOMIAL window modes on the generic kernels) and the (2m+2)-point
    variant (m <= 8)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from oracle import ndft as ondft
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan
    N = (128, 128)
    case = inputs.small_case(N, 128 * 128, seed=2208)
    sel = np.random.default_rng(1).choice(case["M"], 1024, replace=False)
    ex = ondft.ndft(case["k"][sel], case["f"])
    nsel = np.random.default_rng(2).choice(int(np.prod(N)), 1024, replace=False)
    idx = np.unravel_index(nsel, N)
    n = np.stack([idx[d] - N[d] // 2 for d in range(2)], axis=1).astype(float)
    ph = n @ case["k"].T
    ph -= np.floor(ph)
    exa = np.exp(2j * np.pi * ph) @ case["w"]
    rows = []
    variants = [("2m", 0), ("2m+2", B.NFFT_FLAG_WIDE_WINDOW), ("2m LINEAR", B.NFFT_FLAG_WINDOW_LINEAR),
                ("2m POLYNOMIAL", B.NFFT_FLAG_WINDOW_POLYNOMIAL), ("2m DIRECT", B.NFFT_FLAG_WINDOW_DIRECT)]
    for dt, name in ((torch.complex64, "c64"), (torch.complex128, "c128")):
        for taps, flags in variants:
            for m in range(2, 11):
                if m > 8 and flags == B.NFFT_FLAG_WIDE_WINDOW:
                    continue  # K = 2m + 2 > 18: not built
                plan = Plan(N, case["M"], sigma=2.0, m=m, dtype=dt, flags=flags)
                plan.set_nodes(torch.from_numpy(case["k"]).cuda())
                fh = plan.forward(torch.from_numpy(case["f"]).to(dt).cuda()).cpu().numpy()[sel]
                y = plan.adjoint(torch.from_numpy(case["w"]).to(dt).cuda()).cpu().numpy()[idx]
                plan.close()
                rows.append({"dtype": name, "taps": taps, "m": m,
                             "fwd_l2": float(np.linalg.norm(fh - ex) / np.linalg.norm(ex)),
                             "fwd_inf": float(np.max(np.abs(fh - ex)) / np.max(np.abs(ex))),
                             "adj_l2": float(np.linalg.norm(y - exa) / np.linalg.norm(exa)),
                             "adj_inf": float(np.max(np.abs(y - exa)) / np.max(np.abs(exa)))})
    print(json.dumps({"metric": "NFFT relative error vs exact NDFT (1024 sampled outputs each way)",
                      "config": {"workload": "2D N=128^2 M=16384 sigma=2 uniform nodes"}, "rows": rows}))


def run_tiles(args):
    """Tile-shape sweep (the GPU analogue of the block-size study of Sec. 5.2):
    gather and scatter time per tile shape across dimension, m, sigma and node
    density, including a clustered (non-uniform) node set."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(2208)
    t3 = [(4, 4, 4), (8, 8, 8), (9, 9, 8), (9, 9, 9), (8, 8, 4), (4, 8, 8), (6, 8, 8), (16, 8, 8), (16, 16, 16)]
    n3 = 128 ** 3
    clustered = inputs.wrap_half(0.12 * rng.standard_normal((n3, 3)))
    cases = [
        ("3d sigma=2 m=4 uniform M=|I_N|/4", (128,) * 3, 2.0, 4, inputs.uniform_nodes(rng, n3 // 4, 3), t3),
        ("3d sigma=2 m=4 uniform M=|I_N|", (128,) * 3, 2.0, 4, inputs.uniform_nodes(rng, n3, 3), t3),
        ("3d sigma=2 m=4 uniform M=2|I_N|", (128,) * 3, 2.0, 4, inputs.uniform_nodes(rng, 2 * n3, 3), t3),
        ("3d sigma=2 m=4 clustered (normal, sd 0.12) M=|I_N|", (128,) * 3, 2.0, 4, clustered, t3),
        ("3d sigma=1.25 m=6 uniform M=|I_N|", (128,) * 3, 1.25, 6, inputs.uniform_nodes(rng, n3, 3),
         [(4, 4, 4), (5, 5, 5), (5, 5, 4), (4, 5, 5), (8, 8, 8), (8, 8, 4), (16, 8, 8)]),
        ("2d sigma=2 m=4 uniform M=|I_N|", (256, 256), 2.0, 4, inputs.uniform_nodes(rng, 256 * 256, 2),
         [(8, 8), (16, 16), (32, 32), (64, 64), (16, 32), (32, 16), (9, 25), (8, 25)]),
    ]
    rows = []
    for name, N, sigma, m, k, tiles in cases:
        M = k.shape[0]
        plan = Plan(N, M, sigma=sigma, m=m, dtype=torch.complex64)
        kd = torch.from_numpy(k).cuda()
        w = torch.ones(M, dtype=torch.complex64, device="cuda")
        fh = torch.empty(M, dtype=torch.complex64, device="cuda")
        f = torch.ones(N, dtype=torch.complex64, device="cuda")
        h = plan.handle
        for tile in tiles:
            try:
                plan.set_tile(tile)
                plan.set_nodes(kd)
            except Exception as exc:  # tile not admissible for this plan
                rows.append({"case": name, "tile": list(tile), "unavailable": str(exc)})
                continue
            B.check(B.nfft_step_pad_fft(h, f.data_ptr()))
            tg = time_steps(lambda: B.check(B.nfft_step_gather(h, fh.data_ptr())), 10, 2, stream, flush)
            ts = time_steps(lambda: B.check(B.nfft_step_scatter(h, w.data_ptr())), 10, 2, stream, flush)
            rows.append({"case": name, "M": M, "tile": list(tile), "gather_ms": round(tg, 4),
                         "scatter_ms": round(ts, 4), "nodes_per_s": M / ((tg + ts) * 1e-3),
                         "fast_gather": plan.paths()["fast_gather"],
                         "fast_scatter": plan.paths()["fast_scatter"]})
        plan.close()
    print(json.dumps({"metric": "gather + scatter time per tile shape", "unit": "ms",
                      "data": "synthetic (seeded PCG64)", "rows": rows}))


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2208_00049_gb300 import binding as B
    from paper_2208_00049_gb300 import inputs
    from paper_2208_00049_gb300.nfft import Plan

    wl = inputs.workload(WORKLOADS[args.workload])
    dt = torch.complex64 if wl["dtype"] == "c64" else torch.complex128
    stream = torch.cuda.current_stream()
    plan = Plan(wl["N"], wl["M"], sigma=wl["sigma"], m=wl["m"], dtype=dt)
    k_d = torch.from_numpy(wl["k"]).cuda()
    f_d = torch.from_numpy(wl["f"]).to(dt).cuda()
    w_d = torch.from_numpy(wl["w"]).to(dt).cuda()
    fhat_d = torch.empty(wl["M"], dtype=dt, device="cuda")
    y_d = torch.empty(wl["N"], dtype=dt, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # set_nodes (precomputation), timed separately
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    plan.set_nodes(k_d)
    torch.cuda.synchronize()
    ev[0].record(stream)
    plan.set_nodes(k_d)
    ev[1].record(stream)
    torch.cuda.synchronize()
    set_nodes_ms = ev[0].elapsed_time(ev[1])
    info = plan.info()

    h = plan.handle
    paths = plan.paths()
    # Algorithm 1: correction + zero pad + FFT | resampling; Algorithm 2:
    # adjoint resampling | inverse FFT + crop + correction
    names = ["pad_fft", "gather", "scatter", "fft_crop"]
    nev = len(names) + 1

    def step(evs):
        evs[0].record(stream)
        B.check(B.nfft_step_pad_fft(h, f_d.data_ptr()))
        evs[1].record(stream)
        B.check(B.nfft_step_gather(h, fhat_d.data_ptr()))
        evs[2].record(stream)
        B.check(B.nfft_step_scatter(h, w_d.data_ptr()))
        evs[3].record(stream)
        B.check(B.nfft_step_fft_crop(h, y_d.data_ptr()))
        evs[4].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(nev)])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    all_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            step(all_ev[i])
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    B.check(B.nfft_plan_sync(h))

    per = {n: [] for n in names}
    steps_ms = []
    for evs in all_ev:
        steps_ms.append(evs[0].elapsed_time(evs[-1]))
        for j, n in enumerate(names):
            per[n].append(evs[j].elapsed_time(evs[j + 1]))
    agg = aggregate_replicas(sum(steps_ms), wl["M"], args.steps)
    ms_per_step = agg["ms_per_step"]
    value = agg["value"]
    mean = {n: statistics.mean(v) for n, v in per.items()}
    resample_ms = mean["gather"] + mean["scatter"]

    # roofline of the dominant kernel
    dom = "gather" if mean["gather"] >= mean["scatter"] else "scatter"
    peak, peak_kind = measured_peak()
    abytes = algorithmic_bytes(wl, dom)
    achieved = abytes / (mean[dom] * 1e-3) / 1e9
    traffic = profiled_traffic(dom, args.workload)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "algorithmic_bytes": abytes}
    # on-chip bounds of the resampling kernels (they are not HBM-bound at 3D):
    # useful FP32 FMAs ((2m)^D complex x real products = 2 (2m)^D FMAs per node)
    # against the FP32 peak (SMs x 128 FMA/clk), and the shared-memory floor of
    # reading each of the (2m)^D complex64 taps once (8 B; 128 B per wavefront)
    # against one wavefront per clock per SM; clock = the SM maximum
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    taps = (2 * wl["m"]) ** len(wl["N"])
    fmas = 2 * taps * wl["M"]
    wavefronts = wl["M"] * taps * (8 if dt == torch.complex64 else 16) / 128.0
    clk_hz = 2070e6
    onchip = {"clock_mhz": clk_hz / 1e6, "sms": sms,
              "fp32_peak_tflops": round(2 * sms * 128 * clk_hz / 1e12, 1),
              "shared_peak_wavefronts_per_s": sms * clk_hz}
    for n in ("gather", "scatter"):
        t = mean[n] * 1e-3
        onchip[n] = {"useful_fma_tflops": round(2 * fmas / t / 1e12, 2),
                     "fma_frac": round(fmas / t / (sms * 128 * clk_hz), 4),
                     "shared_floor_frac": round(wavefronts / t / (sms * clk_hz), 4)}
    roofline["onchip"] = onchip
    kernel_table = {}
    for n in names:
        ab = algorithmic_bytes(wl, n)
        kernel_table[n] = {"ms": round(mean[n], 4), "GBps": round(ab / (mean[n] * 1e-3) / 1e9, 1),
                           "hbm_frac": round(ab / (mean[n] * 1e-3) / 1e9 / peak, 4)}

    # the same FFT steps of Algorithms 1 and 2 as separate correction kernels
    # around cuFFT (the form the pruned FFT replaces)
    def lib_fwd():
        B.check(B.nfft_step_deconv_pad(h, f_d.data_ptr()))
        B.check(B.nfft_step_fft(h, -1))

    def lib_adj():
        B.check(B.nfft_step_fft(h, +1))
        B.check(B.nfft_step_crop_deconv(h, y_d.data_ptr()))

    nlib = min(20, max(3, args.steps // 4))
    fft_forms = {"pruned_fft_used": paths["pruned_fft"],
                 "pad_fft_ms": round(mean["pad_fft"], 4), "fft_crop_ms": round(mean["fft_crop"], 4),
                 "library_pad_fft_ms": round(time_steps(lib_fwd, nlib, 2, stream, flush), 4),
                 "library_fft_crop_ms": round(time_steps(lib_adj, nlib, 2, stream, flush), 4)}

    # node gradient (row a8) through nfft_grad on the same workload: the
    # forward's pad_fft plus the derivative gather
    gk_d = torch.empty((wl["M"], len(wl["N"])), dtype=torch.float32 if dt == torch.complex64 else torch.float64,
                       device="cuda")
    grad_ms = time_steps(lambda: B.check(B.nfft_grad(h, f_d.data_ptr(), w_d.data_ptr(), gk_d.data_ptr())),
                         min(20, max(3, args.steps // 4)), 2, stream, flush)
    grad_form = {"nodes_per_s": world * wl["M"] / (grad_ms * 1e-3), "ms": round(grad_ms, 4)}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        f_h = torch.from_numpy(wl["f"]).to(dt).pin_memory()
        w_h = torch.from_numpy(wl["w"]).to(dt).pin_memory()
        fh_h = torch.empty(wl["M"], dtype=dt).pin_memory()
        y_h = torch.empty(wl["N"], dtype=dt).pin_memory()
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for _ in range(2):
            plan.forward(f_h, out=fh_h)
            plan.adjoint(w_h, out=y_h)
        times = []
        for _ in range(min(50, max(3, args.steps // 2))):
            flush.zero_()
            ee[0].record(stream)
            plan.forward(f_h, out=fh_h)
            plan.adjoint(w_h, out=y_h)
            ee[1].record(stream)
            torch.cuda.synchronize()
            times.append(ee[0].elapsed_time(ee[1]))
        sync_ms = statistics.mean(times)
        # pipelined: nfft_plan_set_async lets each step's copies overlap the
        # previous step's kernels; steps back to back (the device working set,
        # grid + nodes + stage buffers, exceeds L2), wall clock over K steps
        plan.set_async(True)
        for _ in range(3):
            plan.forward(f_h, out=fh_h)
            plan.adjoint(w_h, out=y_h)
        plan.sync()
        K = min(50, max(5, args.steps // 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            plan.forward(f_h, out=fh_h)
            plan.adjoint(w_h, out=y_h)
        plan.sync()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / K
        plan.set_async(False)
        if world > 1:
            t = torch.tensor([e2e_ms, sync_ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms, sync_ms = float(t[0].item()), float(t[1].item())
        nb = f_h.numel() * f_h.element_size() + w_h.numel() * w_h.element_size()
        ob = fh_h.numel() * fh_h.element_size() + y_h.numel() * y_h.element_size()
        e2e = {"value": world * wl["M"] / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": ob, "ms_per_step": round(e2e_ms, 3),
               "mode": "nfft_forward + nfft_adjoint on pinned host buffers, nfft_plan_set_async (copies of "
                       "one step overlap the kernels of the previous one), %d steps back to back, wall clock; "
                       "device working set larger than L2" % K,
               "synchronous": {"value": world * wl["M"] / (sync_ms * 1e-3), "ms_per_step": round(sync_ms, 3),
                               "mode": "each step waits for its outputs; L2 flushed between steps; CUDA events"}}

    # FP64 form on the same workload, and the FP32 result's accuracy
    fhat32 = fhat_d.cpu().numpy()
    fp64 = None
    ref64 = None
    accuracy = {}
    if rank == 0 and not args.no_fp64_form and dt == torch.complex64:
        fp64, ref64, err = fp64_form(wl, fhat32, min(10, max(3, args.steps // 4)), 2, flush)
        accuracy["rel_l2_fp32_vs_fp64_form"] = err
    wmodes = None
    if rank == 0 and world == 1 and not args.no_other_configs:
        try:
            wmodes = window_modes_form(wl, min(5, max(3, args.steps // 4)), 1, flush, ref64)
        except Exception as exc:
            wmodes = {"unavailable": str(exc)}
    full = None
    if rank == 0 and not args.no_full_form:
        try:
            full = full_matrix_form(wl, min(10, max(3, args.steps // 4)), 2, flush)
        except Exception as exc:  # e.g. too many nonzeros for 32-bit CSR indices
            full = {"unavailable": str(exc)}

    comp = None
    if rank == 0 and world == 1 and dt == torch.complex64 and not args.no_other_configs:
        try:
            comp = compensated_form(args.workload, min(10, max(3, args.steps // 4)), 2, flush)
        except Exception as exc:
            comp = {"unavailable": str(exc)}
    other = None
    if rank == 0 and world == 1 and not args.no_other_configs and args.workload == "3d":
        other = other_configs(max(3, args.other_steps), 3, flush, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v1, det1 = oracle_throughput(wl, args.cpu_sample)
        hc = host_cpu()
        one = {"value": v1, "unit": UNIT, "cores": cpu_cores_used(), "kind": "oracle",
               "sample": det1["sample"], "detail": det1}
        try:
            va, deta = oracle_all_cores(wl)
            cpu = {"value": va, "unit": UNIT, "cores": deta["cores"], "kind": "oracle",
                   "sample": deta["sample"], "cpu_model": hc["model"], "nproc": hc["nproc"],
                   "detail": deta, "one_core": one}
        except Exception as exc:  # e.g. no shared memory for the process pool
            cpu = dict(one, cpu_model=hc["model"], nproc=hc["nproc"], all_cores_unavailable=str(exc))
        accuracy["rel_l2_vs_ndft_48_sampled_nodes"] = ndft_sample_error(wl, fhat32)

    # pruned FFT: 3 + 3 line-DFT kernels; else deconv_pad and crop_deconv
    # (cuFFT's kernels and the grid memset not counted); gather and scatter
    launches_per_step = (8 if paths["pruned_fft"] else 4)
    plan.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if dt == torch.complex64 else "f64",
            "data": "synthetic (seeded PCG64, uniform nodes)",
            "config": {"workload": workload_desc(wl), "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "tile": list(info["tile"]), "work_items": info["n_items"]},
            "nodes_per_s_resampling_only": world * wl["M"] / (resample_ms * 1e-3),
            # the three ways of the measurement definition: forward (Algorithm 1),
            # adjoint (Algorithm 2) and both, with and without the FFT steps;
            # min / median over the timed steps beside the mean of `value`
            "per_direction": {
                "forward_nodes_per_s": world * wl["M"] / ((mean["pad_fft"] + mean["gather"]) * 1e-3),
                "adjoint_nodes_per_s": world * wl["M"] / ((mean["scatter"] + mean["fft_crop"]) * 1e-3),
                "gather_nodes_per_s": world * wl["M"] / (mean["gather"] * 1e-3),
                "scatter_nodes_per_s": world * wl["M"] / (mean["scatter"] * 1e-3),
                "step_ms_min": round(min(steps_ms), 4),
                "step_ms_median": round(statistics.median(steps_ms), 4),
            },
            "set_nodes_ms": round(set_nodes_ms, 3),
            "kernels": kernel_table,
            "fft_forms": fft_forms,
            "grad_form": grad_form,
            "roofline": roofline,
            "fp64_form": fp64,
            "full_matrix_form": full,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "compensated_form": comp,
            "window_modes": wmodes,
            "other_configs": other,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    del np


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "diff":
        run_diff(args)
    elif args.workload == "accuracy":
        run_accuracy(args)
    elif args.workload == "tiles":
        run_tiles(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
