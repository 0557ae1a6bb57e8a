"""The reference arm of bench.py (the CPU FP64 oracle) runs without a GPU:
its one JSON line keeps the benchmark contract, and only rank 0 prints it."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = _run({}, "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "unknowns/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # four V-cycles of the diagonal hierarchy do not reach 1e-10; the cycle
    # count to reach it comes from the measured contraction (about 0.06 per
    # cycle for this workload, so about nine cycles)
    assert 7 <= d["config"]["cycles_to_rtol"] <= 12


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_traffic_counters_belong_to_the_current_kernels():
    """The DRAM traffic bench.py reports for the dominant kernels was captured
    on the kernel source it names by hash; a kernel edited since reports no
    traffic (null) until it is captured again.  Both are current."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for t in (bench.TRAFFIC, bench.TRAFFIC3):
        assert bench.kernel_source_sha1(t["kernel"], t["file"]) == t["source_sha1"], t["kernel"]
        assert bench.measured_traffic(t) == t["bytes"] > 0
    stale = dict(bench.TRAFFIC, source_sha1="0" * 40)
    assert bench.measured_traffic(stale) is None
