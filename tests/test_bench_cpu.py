"""bench.py's contract pieces that run without a GPU: the reference arm (the FP64
oracle timed on host cores) and its JSON line, the silence of the other ranks under
a multi-process launch, and the clock sampler's fallback."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=timeout, cwd=ROOT, env=env)


def test_reference_arm_json_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "qaoa_n20_p3_depol_damp_K4096"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                  env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_sampler_without_samples():
    sys.path.insert(0, ROOT)
    import bench

    s = bench.ClockSampler(0)
    s.proc = None  # as when nvidia-smi cannot be started
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]
    s.proc = object()  # started, but nothing arrived within the timed region
    assert s.summary()["reasons"] == ["no sample: timed region under 200 ms"]


def test_sweep_counts_follow_the_window_schedules():
    """bench.py's byte counts use the library's window schedules: the fused forward layers
    (the window list the GPU test mirrors) and the tiled adjoint (qubits 0-9, then windows of
    at most six, the cost diagonal on the last; below 12 qubits register windows of 2-4 plus a
    diagonal sweep)."""
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    from test_gpu_fused import fused_windows

    for n in range(2, 33):
        assert bench.fused_window_count(n) == len(fused_windows(n)), n
    assert [bench.fused_window_count(n) for n in (16, 20, 26, 30)] == [2, 3, 3, 4]
    assert [bench.adjoint_window_count(n) for n in (8, 10, 11, 12, 16, 17, 22, 23)] == [4, 4, 5, 2, 2, 3, 3, 4]
