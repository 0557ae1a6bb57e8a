#!/usr/bin/env python3
"""Benchmark: unknowns/s to a 1e-10 relative residual for the diagonally
oriented multigrid solve of Poisson's equation on one GB300 per rank.

A step is one complete solve, from u = 0 to ||f - L u|| / ||f|| <= 1e-10, of
the 2D unit-square problem with h = 1/4096 (4095^2 = 16.8M unknowns, f ~
U[-1,1] seed 1) by the diagonal V-cycle in mixed precision (FP64 residual and
update, FP32 levels).  Under torchrun every rank solves its own replica
(weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU FP64 oracle (the reference arm of this
benchmark) on the host cores: each step is one oracle V-cycle on the same
problem, and the metric is extrapolated from the cycles the oracle needs.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "unknowns/s to 1e-10 rel. residual (2D 4096², 3D 256³), % HBM roofline"
UNIT = "unknowns/s"
N_SIDE = 4095
RTOL = 1e-10
WORKLOAD = "2D unit square, h=1/4096 (4095^2 = 16.8M unknowns), f ~ U[-1,1] seed 1, zero Dirichlet; " \
           "diagonal V-cycle (p=1.052), mixed FP64/FP32, solve from u=0 to 1e-10 relative residual"

# The dominant kernel of the mixed solve is the finest pair fused with u += v
# and the next residual (k_up_ff_2d<RR>, probe family 1).  Algorithmic bytes per
# finest unknown: reads u (8), the carried residual as a float-float pair
# (hi 4 + lo 4), the red residual (N/2 x 4 B = 2) and the blue correction
# (N/4 x 4 B = 1); writes u (8) and the new pair (4 + 4): 35 B.  FP64 pipe
# operations per point: 1 (u + v; the residual update runs in FP32 pairs).
PROBE = {
    "family": 1,
    "name": "k_up_ff_2d<RR>: finest Jacobi prolongation + u += v + carried float-float residual r -= L v",
    "bytes_per_point": 35,
    "fp64_pipe_ops_per_point": 1,
}
# The dominant kernel of the 3D mixed solve: the finest triple's green-red
# sweep fused with u += v and the carried residual (k_green_ff_3d, probe
# family 1).  Bytes per finest unknown: reads u (8), hi 4, lo 4, the red
# correction (N/2 x 4 B = 2); writes u (8), hi 4, lo 4: 34 B.
PROBE3 = {
    "name": "k_green_ff_3d<RR>: finest green-red sweep + u += v + carried float-float residual r -= L v",
    "bytes_per_point": 34,
}
# DRAM traffic of one launch on the 4095^2 workload from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); reported only while the
# kernel's source is the one that was captured.
TRAFFIC = {"kernel": "k_up_ff_2d", "file": "mg_fast2d.cuh", "bytes": 333.867008e6 + 210.874368e6,
           "source_sha1": "a13e9d4e6d101062bdd195c4b7b5b6fdfaee6922"}
# the same for the dominant 3D kernel on the 255^3 workload
TRAFFIC3 = {"kernel": "k_green_ff_3d", "file": "mg_fast3d.cuh", "bytes": 326.936832e6 + 213.631232e6,
            "source_sha1": "d3cc2abc3f1704b3286d2f0682dc9c363a98f5bf"}


# Whole-solve traffic model of the mixed path (the algorithmic bytes the
# method must move per finest unknown): the outer FP64 step -- u and f read,
# u written, the FP32 residual and correction -- about 40 B, and every inner
# FP32 V-cycle about 36 B (finest level two passes, coarse levels ~N points
# of r and v written and read).  A solve of c cycles: 40 + 36 c bytes.
CYCLE_MODEL = {"outer_bytes": 40, "per_cycle_bytes": 36}
# The paper's flop count of one diagonal V-cycle per finest unknown (2D,
# second order; Section 2.3), used for the FP64 path's arithmetic roofline.
PAPER_FLOPS_2D = 25.0


def cycle_roofline(n_unknowns, cycles, ms, peak):
    bpu = CYCLE_MODEL["outer_bytes"] + CYCLE_MODEL["per_cycle_bytes"] * cycles
    ach = bpu * n_unknowns / (ms * 1e-3) / 1e9
    return {"bytes_per_unknown": bpu, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "model": "40 B (outer FP64 step) + 36 B x cycles (FP32 V-cycles) per finest unknown, "
                     "over the whole solve time"}


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# nominal FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PIPE_OPS_PEAK = 152 * 2 * 2.07e9  # FP64 pipe operations per second (an FMA counts once)


def kernel_source_sha1(name: str, file: str = "mg_fast2d.cuh") -> str | None:
    """sha1 of a kernel's source text (from its template line to the end of its body)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "paper_math_9907190_gb300", "csrc", file)
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"template <[^>]*>\s*__global__ void __launch_bounds__\([^)]*\) " + name + r"\(.*?\n}\n", text, re.S)
    return hashlib.sha1(m.group(0).encode()).hexdigest() if m else None


def measured_traffic(t):
    """ncu DRAM bytes of one launch, while the kernel's source is the one captured."""
    sha = kernel_source_sha1(t["kernel"], t["file"])
    return t["bytes"] if (t["bytes"] and sha == t["source_sha1"]) else None


def cuda_timed(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def extra_measurements(dev, stream):
    """The other measured configurations: the FP64 path on the same problem,
    the 3D unit cube, the 512-problem batch and the differentiable 3D batch."""
    import torch

    from paper_math_9907190_gb300 import Batch, Context, PoissonSolve
    from paper_math_9907190_gb300 import inputs as I
    out = {}
    f = torch.from_numpy(I.square_large(N_SIDE)).to(dev)
    with Context(2, N_SIDE, precision="fp64") as c:
        u = c.new_grid()
        ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f, u, from_zero=True, rtol=RTOL, max_cycles=60), 5, stream)
        out["square4095_fp64"] = {"unknowns_per_s": N_SIDE**2 / (ms * 1e-3), "ms": ms, "cycles": cyc, "relres": rel}
        # the FP64 path's arithmetic roofline: its finest residual kernel
        # (k_res0_2d: 5 FP64 operations per point, probed live inside the
        # solve) and the whole solve at the paper's 25 flops per unknown and
        # cycle, against this device's measured FP64 pipe rate
        rate = c.fp64_rate()
        c.probe_set(0)
        for _ in range(3):
            c.solve(f, u, from_zero=True, rtol=RTOL, max_cycles=60)
        k, pms = c.probe_read()
        c.probe_set(-1)
        avg = pms / max(k, 1)
        ops = 5 * N_SIDE**2 / (avg * 1e-3)
        peak_hbm = read_peaks().get("hbm_gbs", 6800.0)
        flops = PAPER_FLOPS_2D * N_SIDE**2 * cyc / (ms * 1e-3)
        out["square4095_fp64"]["roofline_fp64"] = {
            "bound": "fp64", "kernel": "k_res0_2d<double>: finest residual r = f - L u, FP64 (5 FP64 ops per point)",
            "avg_launch_ms": avg, "launches_probed": k, "achieved": ops, "peak": rate, "unit": "FP64 ops/s",
            "frac": ops / rate, "hbm_frac": 24 * N_SIDE**2 / (avg * 1e-3) / 1e9 / peak_hbm,
            "peak_source": "measured on this device by mg_fp64_rate (independent FP64 FMA chains on every SM; "
                           "an FMA counts one operation)",
            "solve": {"paper_flops_per_unknown_cycle": PAPER_FLOPS_2D, "achieved_flop_s": flops,
                      "peak_flop_s": 2 * rate, "frac": flops / (2 * rate)}}
    for prec in ("mixed", "fp64"):  # the conventional 2^-l V-cycle the paper compares with
        with Context(2, N_SIDE, hierarchy="usual", precision=prec) as c:
            u = c.new_grid()
            ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f, u, from_zero=True, rtol=RTOL, max_cycles=80), 3, stream)
            out[f"square4095_usual_{prec}"] = {"unknowns_per_s": N_SIDE**2 / (ms * 1e-3), "ms": ms, "cycles": cyc,
                                               "relres": rel, "workload": "same problem, conventional V-cycle "
                                               "(full weighting, bilinear + red-black Jacobi, p = 1.121)"}
    # fourth-order residual (2D Mehrstellen, p = 1.2), and the two-stage solve:
    # second-order cycles to 1e-4, then fourth-order cycles to 1e-10
    for prec in ("mixed", "fp64"):
        with Context(2, N_SIDE, order=4, precision=prec) as c:
            u = c.new_grid()
            ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f, u, from_zero=True, rtol=RTOL, max_cycles=80, raise_on_fail=False), 3, stream)
            out[f"square4095_order4_{prec}"] = {"unknowns_per_s": N_SIDE**2 / (ms * 1e-3), "ms": ms, "cycles": cyc,
                                                "relres": rel, "workload": "same f, fourth-order residual "
                                                "(Mehrstellen right-hand side), diagonal V-cycle p = 1.2"}
            if prec == "mixed":
                ms, (_, c2, c4, rel) = cuda_timed(lambda: c.solve_two_stage(f, u.zero_(), rtol=RTOL, max_cycles=80, raise_on_fail=False),
                                                  3, stream)
                out["square4095_two_stage_mixed"] = {"unknowns_per_s": N_SIDE**2 / (ms * 1e-3), "ms": ms,
                                                     "cycles_order2": c2, "cycles_order4": c4, "relres": rel,
                                                     "workload": "same f, second-order cycles (p = 1.052) to "
                                                     "1e-4, then fourth-order cycles to 1e-10"}
    # one extra Jacobi sweep per level (the extension the paper leaves open;
    # per-stage kernels, p = 1.052 as the headline)
    with Context(2, N_SIDE, precision="mixed") as c:
        c.set_sweeps(1)
        u = c.new_grid()
        ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f, u, from_zero=True, rtol=RTOL, max_cycles=60, raise_on_fail=False),
                                          3, stream)
        out["square4095_sweeps1_mixed"] = {"unknowns_per_s": N_SIDE**2 / (ms * 1e-3), "ms": ms, "cycles": cyc,
                                           "relres": rel, "workload": "same problem, one extra Jacobi sweep per "
                                           "level (mg_set_sweeps), per-stage kernels"}
    del f
    f3 = torch.from_numpy(I.cube(255)).to(dev)
    for prec in ("mixed", "fp64"):  # fourth-order residual in 3D (19-point, Eq. Efos4)
        with Context(3, 255, order=4, precision=prec) as c:
            u = c.new_grid()
            ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f3, u, from_zero=True, rtol=RTOL, max_cycles=80, raise_on_fail=False), 3, stream)
            out[f"cube255_order4_{prec}"] = {"unknowns_per_s": 255**3 / (ms * 1e-3), "ms": ms, "cycles": cyc,
                                             "relres": rel, "workload": "3D unit cube 255^3, same f, 19-point "
                                             "fourth-order residual, diagonal V-cycle (0.91, 0.80, 0.70, 1.77)"}
    for prec in ("mixed", "fp64"):
        with Context(3, 255, precision=prec) as c:
            u = c.new_grid()
            ms, (_, cyc, rel, _) = cuda_timed(lambda: c.solve(f3, u, from_zero=True, rtol=RTOL, max_cycles=60), 5, stream)
            out[f"cube255_{prec}"] = {"unknowns_per_s": 255**3 / (ms * 1e-3), "ms": ms, "cycles": cyc, "relres": rel,
                                      "workload": "3D unit cube 255^3, f = -6 pi^2 sin sin sin(2 pi z) + N(0,1e-6), "
                                                  "diagonal V-cycle (1.11, 1.42, 1.08, 0.99)"}
            if prec == "mixed":
                out["cube255_mixed"]["cycle_roofline"] = cycle_roofline(255**3, cyc, ms,
                                                                         read_peaks().get("hbm_gbs", 6800.0))
            if prec == "mixed":  # the dominant 3D kernel, probed inside the solve as the headline's
                c.probe_set(PROBE["family"])
                for _ in range(3):
                    c.solve(f3, u, from_zero=True, rtol=RTOL, max_cycles=60)
                k, pms = c.probe_read()
                c.probe_set(-1)
                avg = pms / max(k, 1)
                ach = PROBE3["bytes_per_point"] * 255**3 / (avg * 1e-3) / 1e9
                peak = read_peaks().get("hbm_gbs", 6800.0)
                out["cube255_roofline"] = {"kernel": PROBE3["name"], "bound": "hbm", "avg_launch_ms": avg,
                                           "launches_probed": k, "bytes_per_point": PROBE3["bytes_per_point"],
                                           "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                           "traffic": measured_traffic(TRAFFIC3)}
    del f3
    sides = I.batch_sides(512)
    fs = [torch.from_numpy(I.batch_f(n, b)).to(dev) for b, n in enumerate(sides)]
    us = [torch.zeros_like(x) for x in fs]
    tot = sum(n * n for n in sides)
    for prec in ("mixed", "fp64"):
        with Batch(2, sides, precision=prec) as bt:
            def run():
                for x in us:
                    x.zero_()
                return bt.solve(fs, us, rtol=RTOL, max_cycles=60)
            ms, (_, cyc, rel) = cuda_timed(run, 3, stream)
            out[f"batch512_{prec}"] = {"unknowns_per_s": tot / (ms * 1e-3), "ms": ms, "unknowns": tot,
                                       "max_cycles": max(cyc), "max_relres": max(rel),
                                       "workload": "512 2D problems, n_b = 2^k - 1, k ~ U{5..10} (seed 3), "
                                                   "f_b ~ U[-1,1] (seed 4+b); one graph launch"}
    del fs, us
    n = 127
    F = torch.stack([torch.from_numpy(I.grad_f(n, b)) for b in range(64)]).to(dev)
    ut = torch.from_numpy(I.grad_target(n)).to(dev)

    def fwd_bwd():
        x = F.detach().requires_grad_(True)
        U = PoissonSolve.apply(x, RTOL, "mixed")
        ((U - ut) ** 2).sum().backward()
        return x.grad
    ms, _ = cuda_timed(fwd_bwd, 3, stream)
    out["grad64x127_mixed"] = {"solves_per_s": 2 * 64 / (ms * 1e-3), "ms_fwd_bwd": ms,
                               "unknowns_per_s": 2 * 64 * n**3 / (ms * 1e-3),
                               "workload": "64 3D problems at 127^3, f ~ N(0,1), loss sum (u - u_t)^2; "
                                           "forward solve + adjoint solve (autograd), mixed, 1e-10"}
    return out


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 7 and p[0].replace(".", "").isdigit():
                    rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][1]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())}


def oracle_cpu_baseline(f):
    """The oracle as it stands (C, FP64) solving the full workload from u = 0
    to 1e-10, on all host cores (its per-point loops under OpenMP; sums and
    the coarsest solve serial, so the result does not depend on the thread
    count) and on one core.  Returns the baseline dict and its solution."""
    import oracle as O
    nproc = os.cpu_count() or 1
    legs = {}
    u = None
    for threads in (nproc, 1):
        used = O.set_threads(threads)
        t0 = time.perf_counter()
        u, cycles, rel, _ = O.solve(f, omega=[1.052], rtol=RTOL, max_cycles=40)
        dt = time.perf_counter() - t0
        legs[threads] = {"value": N_SIDE**2 / dt, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"one full oracle solve of the benchmark workload ({cycles} FP64 V-cycles to "
                                   f"relres {rel:.2e}, {dt:.2f} s on {used} host thread(s))"}
    O.set_threads(1)
    out = dict(legs[nproc])
    out["nproc"] = nproc
    out["cpu_model"] = cpu_model()
    out["single_core"] = legs[1]
    return out, u


def oracle_cpu_configs():
    """The oracle (C, FP64) on all host cores on the other configurations of
    the measurement table: the 3D unit cube 255^3 in full, and seeded subsets
    of the 512-problem batch (16 problems) and of the 64 x 127^3 gradient
    batch (2 problems, forward and adjoint solve); per-unknown rates, the
    subsets stated.  About 5 s of host time."""
    import numpy as np

    import oracle as O
    from paper_math_9907190_gb300 import inputs as I
    used = O.set_threads(os.cpu_count() or 1)
    out = {}
    f3 = I.cube(255)
    t0 = time.perf_counter()
    _, cyc, rel, _ = O.solve(f3, omega=[1.11, 1.42, 1.08, 0.99], rtol=RTOL, max_cycles=40)
    dt = time.perf_counter() - t0
    out["cube255"] = {"value": 255**3 / dt, "unit": UNIT, "cores": used, "kind": "oracle",
                      "sample": f"one full oracle solve of the 3D 255^3 workload ({cyc} FP64 V-cycles to relres "
                                f"{rel:.2e}, {dt:.2f} s)"}
    del f3
    sides = I.batch_sides(512)
    pick = sorted(np.random.default_rng(3).choice(len(sides), 16, replace=False).tolist())
    tot, dt = 0, 0.0
    for b in pick:
        fb = I.batch_f(sides[b], b)
        t0 = time.perf_counter()
        O.solve(fb, rtol=RTOL, max_cycles=40)
        dt += time.perf_counter() - t0
        tot += sides[b] ** 2
    out["batch512_subset"] = {"value": tot / dt, "unit": UNIT, "cores": used, "kind": "oracle",
                              "sample": f"16 of the 512 problems (seed 3: sides {[sides[b] for b in pick]}), "
                                        f"each solved in full one after the other, {tot} unknowns in {dt:.2f} s"}
    n = 127
    ut = I.grad_target(n)
    dt = 0.0
    for b in range(2):
        fb = I.grad_f(n, b)
        t0 = time.perf_counter()
        u, _, _, _ = O.solve(fb, omega=[1.11, 1.42, 1.08, 0.99], rtol=RTOL, max_cycles=40)
        g = I.zero_ring(2.0 * (u - ut))
        O.solve(g, omega=[1.11, 1.42, 1.08, 0.99], rtol=RTOL, max_cycles=40)  # the adjoint (L is symmetric)
        dt += time.perf_counter() - t0
    out["grad64x127_subset"] = {"solves_per_s": 4 / dt, "unknowns_per_s": 4 * n**3 / dt, "cores": used,
                                "kind": "oracle",
                                "sample": f"2 of the 64 problems at 127^3, forward and adjoint solve each, "
                                          f"{dt:.2f} s"}
    O.set_threads(1)
    return out


def run_reference(args):
    """Reference arm: the CPU FP64 oracle on all host cores, rank 0 only; a
    step is one full oracle solve of the workload from u = 0 to 1e-10."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from paper_math_9907190_gb300 import inputs as I
    f = I.square_large(N_SIDE)
    nproc = os.cpu_count() or 1
    used = O.set_threads(nproc)
    times, cycles, rel = [], 0, 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, cycles, rel, _ = O.solve(f, omega=[1.052], rtol=RTOL, max_cycles=40)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    t_step = statistics.mean(times)
    value = N_SIDE**2 / t_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("mixed FP64/FP32", "FP64 CPU oracle"),
                       "step": "one full oracle solve", "cycles_to_rtol": cycles, "relres": rel},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "nproc": nproc, "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": f"{args.warmup + args.steps} full oracle solves of the workload "
                                       f"({cycles} V-cycles each to 1e-10) on {used} host thread(s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 3D, batched and gradient measurements")
    ap.add_argument("--ncu", action="store_true", help="short run (warm-up + one solve) for an ncu launch list")
    ap.add_argument("--ncu-workload", default="square4095", choices=["square4095", "cube255"],
                    help="workload of the --ncu run")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_math_9907190_gb300 import Context
    from paper_math_9907190_gb300 import dist as D
    from paper_math_9907190_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    if args.ncu and args.ncu_workload == "cube255":
        f_host = I.cube(255)
        N = 255**3
        ctx = Context(3, 255, hierarchy="diag", order=2, precision="mixed")
    else:
        f_host = I.square_large(N_SIDE)
        N = N_SIDE**2
        ctx = Context(2, N_SIDE, hierarchy="diag", order=2, precision="mixed", omega=(1.052,))
    f = torch.from_numpy(f_host).to(dev)
    u = ctx.new_grid()
    stream = torch.cuda.current_stream(dev)

    def step():  # a solve from u = 0 (mg_solve_zero: u is output only, zeroed inside the solve's graph)
        return ctx.solve(f, u, rtol=RTOL, max_cycles=60, from_zero=True)

    warm = max(args.warmup, 3)  # at least three untimed warm-up steps
    for _ in range(warm):
        step()
    if args.ncu:  # short run for an ncu launch list: the warm-up solves plus one solve
        step()
        torch.cuda.synchronize()
        print(json.dumps({"ncu_run": True, "launches": ctx.launch_count()}))
        ctx.close()
        return 0
    barrier()
    launches0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        cycles = []
        for _ in range(args.steps):
            _, cyc, rel, hist = step()
            cycles.append(cyc)
        ev1.record(stream)
        barrier()
    launches = ctx.launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = D.max_over_ranks(ms, dev)
    value = world * N / (ms_max * 1e-3)

    # end to end through the C ABI, pipelined (mg_solve_host_many): the K
    # steps' problems in one call; every problem's f is copied in from pinned
    # host memory and its u copied back to pinned host memory inside the timed
    # region, overlapped with the other problems' solves (two device buffer
    # pairs); wall-clock time of the call over K
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pins = [torch.empty_like(f_pin).pin_memory() for _ in range(2)]

    def e2e_many(k):
        t0 = time.perf_counter()
        ctx.solve_host_many([f_pin] * k, [u_pins[i % 2] for i in range(k)], rtol=RTOL, max_cycles=60)
        return (time.perf_counter() - t0) * 1e3 / k

    e2e_many(2)
    barrier()
    e2e_pipe_ms = D.max_over_ranks(e2e_many(args.steps), dev)
    barrier()

    # end to end through the C ABI with HOST buffers (mg_solve_host): every
    # step copies f from pinned host memory to the device, solves from u = 0
    # and copies u back to pinned host memory, one call after the other (no
    # overlap between steps); wall-clock time per call
    u_host = torch.empty_like(f_pin).pin_memory()
    for _ in range(2):
        ctx.solve_host(f_pin, u_host, rtol=RTOL, max_cycles=60)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, e2e_cyc, e2e_rel = ctx.solve_host(f_pin, u_host, rtol=RTOL, max_cycles=60)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = D.max_over_ranks(e2e_ms, dev)
    e2e_ok = bool(np.array_equal(u_host.numpy(), u.cpu().numpy()))
    barrier()
    # the host link's own speed on the same buffers (best of 5 single copies,
    # CUDA events on the stream): the end-to-end step's floor is the device
    # solve plus one copy each way at these rates
    def copy_ms(dst, src):
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best
    h2d_ms, d2h_ms = copy_ms(f, f_pin), copy_ms(u_host, u)
    e2e_floor_ms = ms_max + h2d_ms + d2h_ms

    # live probe of the dominant kernel inside the same solve: every launch of
    # its family bracketed by CUDA events on the launching stream (the solver
    # runs its host-driven loop while probed; the kernels are the same)
    ctx.probe_set(PROBE["family"])
    for _ in range(args.steps):
        step()
    nprobe, probe_ms = ctx.probe_read()
    ctx.probe_set(-1)
    avg_ms = probe_ms / max(nprobe, 1)
    peaks = read_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    bytes_ = PROBE["bytes_per_point"] * N
    achieved = bytes_ / (avg_ms * 1e-3) / 1e9
    pipe = PROBE["fp64_pipe_ops_per_point"] * N / (avg_ms * 1e-3)
    traffic = measured_traffic(TRAFFIC)
    roofline = {"bound": "hbm", "kernel": PROBE["name"], "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "algorithmic_bytes": bytes_,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback",
                "avg_launch_ms": avg_ms, "launches_probed": nprobe,
                "cycle_frac": cycle_roofline(N, cycles[-1], ms_max, hbm_peak)["frac"],
                "cycle": cycle_roofline(N, cycles[-1], ms_max, hbm_peak),
                "fp64_pipe": {"ops_per_point": PROBE["fp64_pipe_ops_per_point"], "achieved_ops_s": pipe,
                              "peak_ops_s": FP64_PIPE_OPS_PEAK, "frac": pipe / FP64_PIPE_OPS_PEAK,
                              "peak_note": "152 SMs x 2 FP64 ops/clk x 2.07 GHz (nominal, derived)"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dim": 2, "n": N_SIDE, "hierarchy": "diag", "precision": "mixed",
                       "rtol": RTOL, "cycles": cycles[-1], "relres": rel,
                       "vcycles_per_s": world * cycles[-1] / (ms_max * 1e-3),
                       "l2": "inputs larger than L2 (f and u 134 MB each; ~1 GB moved per cycle)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk.summary(),
            "e2e": {"value": world * N / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(f_pin.numel() * 8), "d2h_bytes_per_step": int(u_host.numel() * 8),
                    "api": "mg_solve_host (C ABI): f from pinned host memory, solve from u = 0, u back to pinned "
                           "host memory; one call per step, copies not overlapped, wall-clock time",
                    "cycles": e2e_cyc, "relres": e2e_rel, "same_u_as_device_solve": e2e_ok,
                    "link": {"h2d_gbs": f_pin.numel() * 8 / (h2d_ms * 1e-3) / 1e9,
                             "d2h_gbs": u_host.numel() * 8 / (d2h_ms * 1e-3) / 1e9,
                             "floor_ms": e2e_floor_ms, "frac": e2e_floor_ms / e2e_ms,
                             "how": "one pinned-host copy each way on the step's buffers, timed alone; "
                                    "floor = device solve + both copies at those rates, one after the other "
                                    "(the copy back overlaps the solve's closing residual, so frac can "
                                    "exceed 1)"},
                    "pipelined": {"value": world * N / (e2e_pipe_ms * 1e-3), "ms_per_step": e2e_pipe_ms,
                                  "how": "mg_solve_host_many (C ABI): the steps' problems in one call, each f "
                                         "copied in and each u copied back (pinned host memory) inside the "
                                         "timed region, overlapped with the other problems' solves on two "
                                         "device buffer pairs; wall-clock time of the call over the steps"}},
            "gpu_launches": int(launches),
            "roofline": roofline}

    if not args.no_extra:
        line["extra"] = extra_measurements(dev, stream)
        line["extra"]["mixed_vs_fp64_speedup_square4095"] = (
            line["extra"]["square4095_fp64"]["ms"] / ms_max)
        line["extra"]["mixed_vs_fp64_speedup_batch512"] = (
            line["extra"]["batch512_fp64"]["ms"] / line["extra"]["batch512_mixed"]["ms"])
        line["extra"]["diag_vs_usual_speedup_square4095_mixed"] = (
            line["extra"]["square4095_usual_mixed"]["ms"] / ms_max)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, u_orc = oracle_cpu_baseline(f_host)
        if not args.no_extra:  # the oracle on the other configurations of the measurement table
            cb["configs"] = oracle_cpu_configs()
        line["cpu_baseline"] = cb
        ug = u.cpu().numpy()
        line["config"]["rel_err_vs_oracle"] = float(np.linalg.norm(ug - u_orc) / np.linalg.norm(u_orc))
        line["config"]["max_pointwise_err_vs_oracle"] = float(np.abs(ug - u_orc).max() / np.abs(u_orc).max())
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
