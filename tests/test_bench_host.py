"""Host-side logic of bench.py that needs no GPU."""
import json
import os
import subprocess
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_source_hash_ignores_comments_and_layout():
    import bench
    code = 'int f(int x) {\n  return x + 1;  // add one\n}\nconst char* s = "a // b /* c */";\n'
    edited = '/* header */\nint f(int x) {\n    return x + 1;  /* one */\n}\n' \
             'const char* s = "a // b /* c */";  // same string\n'
    assert bench._strip_comments(code) == bench._strip_comments(edited)
    assert '"a // b /* c */"' in bench._strip_comments(code)
    assert bench._strip_comments("x = '\\'' ; // q\ny") == "x = '\\'' ; y"
    assert bench._strip_comments("a = 1;") != bench._strip_comments("a = 2;")


def test_source_hash_is_stable():
    import bench
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


def test_source_hash_over_named_files():
    import bench
    one = bench.kernel_source_hash(["resample3d.cu"])
    assert one == bench.kernel_source_hash(["resample3d.cu"])
    assert one != bench.kernel_source_hash(["resample3d.cu", "nfft_plan.cu"])
    assert one != bench.kernel_source_hash()


def test_reference_arm_prints_one_contract_line():
    """--impl reference times the CPU oracle (no GPU involved) and prints one
    JSON line with the contract's keys; run here on the small 1D workload."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "1d", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=root,
                         env=dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0"))
    assert out.returncode == 0, out.stderr
    lines = [x for x in out.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "nodes/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("1d N=256 M=1024")


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle; other ranks print nothing."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "1d", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=300, cwd=root,
                         env=dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1"))
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def test_reference_plan_fits_the_budget():
    """The reference arm sizes each step so that --steps K ends within the
    budget: many steps reuse one full-size grid timing and take small node
    samples; few steps re-time the grid and take large samples (up to the cap)."""
    import bench
    grid_each, n = bench.reference_plan(t_grid=0.7, t_fixed=0.03, s_per_node=4e-5, steps=300, M=2097152,
                                        cap=131072, budget=90.0)
    assert not grid_each
    assert n == int((90.0 / 300 - 0.03) / 4e-5)
    assert 300 * (0.03 + n * 4e-5) <= 90.0 + 1e-6
    grid_each, n = bench.reference_plan(t_grid=0.7, t_fixed=0.03, s_per_node=4e-5, steps=20, M=2097152,
                                        cap=131072, budget=90.0)
    assert grid_each and n == int((90.0 / 20 - 0.7 - 0.03) / 4e-5)
    assert 20 * (0.7 + 0.03 + n * 4e-5) <= 90.0 + 1e-6
    assert bench.reference_plan(0.7, 0.03, 4e-5, 5, 2097152, 131072, 90.0) == (True, 131072)
    # never below 1024 nodes, never above M
    assert bench.reference_plan(5.0, 1.0, 1e-3, 10000, 2097152, 131072, 90.0)[1] == 1024
    assert bench.reference_plan(0.001, 0.0, 1e-7, 1, 1024, 131072, 90.0)[1] == 1024


def test_reference_estimate_counts_the_fixed_part_once():
    import bench
    est = bench.reference_estimate(t_grid=1.0, t_fixed=0.1, t_nodes=0.1 + 1000 * 1e-4, n=1000, M=2000000)
    assert abs(est - (1.0 + 0.1 + 1e-4 * 2000000)) < 1e-6
    # a step faster than the calibrated fixed part contributes no negative time
    assert bench.reference_estimate(1.0, 0.1, 0.05, 1000, 2000000) == 1.1


def test_split_problems_covers_each_problem_once_and_balances():
    import bench
    from paper_2208_00049_gb300 import inputs
    w = bench.batch_weights(inputs.batched_problems(n_problems=64))
    for world in (1, 2, 3, 4, 8):
        parts = [bench.split_problems(w, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(w[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(w)   # within one problem of each other
        assert all(p == sorted(p) for p in parts)


def test_split_aggregation_single_process():
    import bench
    agg = bench.aggregate_split(40.0, 1000, 4)
    assert agg["world"] == 1 and agg["ms_per_step"] == 10.0 and agg["value"] == 1000 / 0.010
