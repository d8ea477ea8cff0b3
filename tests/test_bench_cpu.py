"""The reference arm of bench.py (the oracle on every host core) on the CPU: its JSON line carries
the contract's keys and the number of cores used, its step time fits in the run's own wall clock,
and under a multi-rank launch only rank 0 prints it (the others exit 0)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_workers():
    sys.path.insert(0, ROOT)
    import bench
    return bench.host_workers()


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--oracle-rows", "2", "--workload", "disc1000_p12_ns512"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    import time
    t0 = time.perf_counter()
    res = _run({})
    elapsed = time.perf_counter() - t0
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"] == "disc1000_p12_ns512"
    cb = line["cpu_baseline"]
    assert cb["cores"] == bench_workers() and line["steps"] == 1
    # the step time is what a step took: the run fits in its own wall clock
    assert line["ms_per_step"] * line["steps"] < 1e3 * elapsed


def test_reference_arm_other_ranks_exit_quietly():
    res = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert res.returncode == 0, res.stderr[-2000:]
    assert res.stdout.strip() == ""


def test_a_failing_further_workload_keeps_the_headline(capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    assert bench.guarded("ok", lambda a, b: a + b, 2, 3) == 5

    def boom():
        raise RuntimeError("no convergence")
    out = bench.guarded("example1", boom)
    assert out == {"error": "RuntimeError: no convergence"}
    assert "section example1 failed" in capsys.readouterr().err


def test_roofline_arithmetic():
    # the headline kernel's algorithmic work: 5000 discs, p = 14 (P = 29): 8 P^2 N (N - 1) flop per
    # translation = 1.68e11; the derived FP32 peak: 152 SMs x 128 lanes x 2 flop x 2070 MHz
    import sys
    sys.path.insert(0, ROOT)
    import bench

    assert bench.translation_flop(5000, 14) == 8 * 29 * 29 * 5000 * 4999 == 168166360000
    assert bench.translation_flop(2000, 12, 64) == 8 * 25 * 25 * 2000 * 1999 * 64
    assert bench.translation_flop(1, 14) == 0
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54784) < 1e-9
