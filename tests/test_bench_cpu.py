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
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    assert cb["nproc"] == os.cpu_count() and 1 <= cb["cores"] <= cb["nproc"] and cb["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # a step is a full oracle solve to 1e-10: about nine cycles of the
    # diagonal hierarchy (contraction about 0.06 per cycle for this workload)
    assert 7 <= d["config"]["cycles_to_rtol"] <= 12 and d["config"]["relres"] <= 1e-10


def _bench_module():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench


def test_cpu_baseline_legs_on_all_cores_and_one_core():
    """bench.py's cpu_baseline: the oracle solve of the benchmark workload on
    all host cores, with the one-core leg beside it; the two solutions are
    the same bits (the threads split only per-point loops)."""
    import numpy as np

    from paper_math_9907190_gb300 import inputs as I
    bench = _bench_module()
    cb, u = bench.oracle_cpu_baseline(I.square_large(bench.N_SIDE))
    for key in ("value", "unit", "cores", "kind", "sample", "nproc", "cpu_model", "single_core"):
        assert key in cb, key
    assert cb["single_core"]["cores"] == 1 and cb["value"] > 0 and cb["single_core"]["value"] > 0
    assert np.isfinite(u).all()


def test_main_line_carries_the_roofline_and_e2e_keys():
    """The keys of the GPU arm's line (built on a GPU only): the cycle-level
    HBM fraction, the FP64 path's roofline, the C-ABI end-to-end number with
    its pipelined variant, and the all-cores CPU baseline."""
    bench = _bench_module()
    src = open(os.path.join(ROOT, "bench.py")).read()
    for key in ('"cycle_frac"', '"cycle"', '"roofline_fp64"', '"cycle_roofline"', '"pipelined"', '"api"', '"link"',
                '"single_core"', '"cpu_model"', '"nproc"', '"roofline"', '"cpu_baseline"', '"e2e"', '"clocks"',
                '"configs"', '"cube255"', '"batch512_subset"', '"grad64x127_subset"',
                '"gpu_launches"'):
        assert key in src, key
    r = bench.cycle_roofline(4095**2, 9, 2.0, 6746.3)
    assert r["bytes_per_unknown"] == 40 + 36 * 9
    assert abs(r["frac"] - 364 * 4095**2 / 2e-3 / 1e9 / 6746.3) < 1e-12


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3")
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_traffic_counters_belong_to_the_current_kernels():
    """The DRAM traffic bench.py reports for the dominant kernels was captured
    on the kernel source it names by hash; a kernel edited since reports no
    traffic (null) until it is captured again.  Both are current."""
    bench = _bench_module()
    for t in (bench.TRAFFIC, bench.TRAFFIC3):
        assert bench.kernel_source_sha1(t["kernel"], t["file"]) == t["source_sha1"], t["kernel"]
        assert bench.measured_traffic(t) == t["bytes"] > 0
    stale = dict(bench.TRAFFIC, source_sha1="0" * 40)
    assert bench.measured_traffic(stale) is None
