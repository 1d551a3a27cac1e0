"""bench.py's reference arm, on the CPU: the FP64 oracle timed on a bounded sample
of the D_cut = 64 workload, reported as one JSON line with the GPU arm's metric.

The arm needs no GPU (it runs only `oracle/` and numpy), so its contract is
checked here: one line, the keys the driver reads, the oracle as its own
cpu_baseline and end-to-end figure, and quiet exit on ranks other than 0.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, rank=None):
    env = dict(os.environ)
    if rank is not None:
        env["RANK"] = str(rank)
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=600, env=env)


def json_lines(out):
    return [json.loads(x) for x in out.splitlines() if x.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "workload" in d["config"] and "D_cut=64" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"] and cb["cores"] >= 1
    assert cb["sample"] and cb["detail"]["x_columns"] == 4
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], rank=1)
    assert r.returncode == 0, r.stderr[-2000:]
    assert json_lines(r.stdout) == []


def test_single_core_sample_runs_on_one_thread():
    # the bench's cpu_baseline.single_core: the nx = 1 sample in a child process with one-thread pools
    import bench
    from paper_2609_20536_b300.workloads import headline_points
    p = headline_points(1, d_cut=bench.D_CUT, n_max=bench.N_MAX, n_steps=bench.N_STEPS)[0]
    out = bench.oracle_sample_one_thread(p.beta, p.delta)
    assert out is not None
    s1, u1, threads = out
    assert threads == 1 and s1 > 0 and 0 < u1 < 1
