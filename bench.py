#!/usr/bin/env python
"""Throughput of the coupled CH + NS lattice Boltzmann step on GB300.

Workload: the disk + droplet lattice of the cylinder experiment (Sec. 4.3) at
1024 x 1024 nodes, D2Q9, solid disk of radius 160 lu, droplet of radius 120 lu
on its top, density and viscosity ratio 10, contact angle swept over
{30, 60, 90, 120, 150} deg.  The five angles are five independent instances
advanced by one launch per time step.  A "step" is one time step of all five
instances (5 x 1024^2 lattice updates); the metric is million lattice updates
per second (MLUPS) over the whole job.

Rank 0 prints one JSON line.  Under torchrun every rank runs the same batch on
its own GPU (independent instances, no collective on the data path; weak
scaling), timing is the maximum over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled CH+NS LBM MLUPS on 1 GB300, % of HBM roofline, time-to-equilibrium"
BYTES_PER_LU = 188   # f, g read+write 144; phi0 4; history (phi1, u, S) read 20 + write 20
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="target CPU time of the oracle sample")
    ap.add_argument("--size", type=int, default=1024, help="lattice side (default: the 1024^2 workload)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idxs = sorted({r[0] for r in rows})
        want = idxs[0] if len(idxs) == 1 else (vis.split(",")[0] if vis.split(",")[0].isdigit() else idxs[0])
        rows = [r for r in rows if r[0] == want and len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1].split()[0]) for r in rows]
        smax = float(rows[0][2].split()[0])
        reasons = sorted({n for r in rows for n, v in zip(self.NAMES, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(sm),
                "power_w_max": max(float(r[3].split()[0]) for r in rows if r[3].split()[0].replace(".", "").isdigit())
                if any(r[3].split()[0].replace(".", "").isdigit() for r in rows) else None}


def traffic_from_profile(lu_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel."""
    import hashlib
    src = os.path.join(ROOT, "paper_2311_05091_gb300", "csrc", "lbm_d2q9.cu")
    summ = os.path.join(ROOT, "profiles", "d2q9_step_disk1024x5.md")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        kv = {}
        for line in open(summ):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("kernel_source_sha256_16") != sha:
            return None
        per_lu = float(kv["dram_bytes_per_lu"])
        return per_lu * lu_per_launch
    except Exception:
        return None


def oracle_sample(size_nodes, steps, theta=30.0):
    """Time the FP64 oracle on a square crop of one instance of the workload (single thread)."""
    code = f"""
import os, sys, time, json, math
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import lbm, model
from synthetic.workloads import disk_sweep
n = {int(size_nodes)}
wl = disk_sweep(n=n, Rs=160.0 * n / 1024, R0=120.0 * n / 1024, thetas=({theta},))
prm = dict(wl["params"][0])
st = lbm.init_state("D2Q9", wl["phi0"][0].astype(np.float64), wl["phi1"][0].astype(np.float64),
                    model.Params(**prm), (True, True))
c = model.constants(model.Params(**prm))
lbm.step(st, c, 1)
t = time.perf_counter()
lbm.step(st, c, {int(steps)})
dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt, "lu": n * n * {int(steps)}}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["lu"] / d["seconds"] / 1e6, d["seconds"]


def oracle_sample_size(cpu_seconds, steps):
    """Square crop whose `steps` oracle steps take about cpu_seconds (about 2 us per node-step)."""
    nodes = cpu_seconds / (2.0e-6 * max(steps, 1))
    side = int(math.sqrt(max(nodes, 1024)))
    return max(32, min(1024, side - side % 8))


def dist_setup(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    total = args.steps + args.warmup
    side = oracle_sample_size(120.0, total)
    mlups, secs = oracle_sample(side, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 oracle on a {side}x{side} crop of one instance of the 1024^2 disk+droplet "
                                   f"workload (theta 30 deg); each step one oracle time step of that crop"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of a {side}x{side} crop, 1 thread"},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if world > 1:
        line["note"] = "rank 0 alone runs the CPU reference"
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    world, rank, local = dist_setup(args.gpus)
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_2311_05091_gb300.build import build
    build()
    from paper_2311_05091_gb300 import _lbm as L
    from synthetic.workloads import disk_sweep

    n = args.size
    wl = disk_sweep(n=n, Rs=160.0 * n / 1024, R0=120.0 * n / 1024)
    nb = len(wl["params"])
    lu = wl["nx"] * wl["ny"] * nb
    stream = torch.cuda.Stream()
    ctx = L.Context(L.LBM_D2Q9, wl["nx"], wl["ny"], 1, periodic=(True, True, False),
                    batch=[L.lbm_default_params(**p) for p in wl["params"]])
    ctx.set_stream(stream.cuda_stream)

    # pinned host copies of the inputs and outputs (used by the end-to-end leg)
    def pinned(shape):
        return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()
    h_phi0, h_phi1 = pinned(wl["phi0"].shape), pinned(wl["phi1"].shape)
    h_phi0[...] = wl["phi0"]
    h_phi1[...] = wl["phi1"]
    o_phi1, o_u, o_p = pinned((nb, n * n)), pinned((nb, 2, n * n)), pinned((nb, n * n))

    ctx.set_solid(h_phi0)
    ctx.set_phase(h_phi1)
    ctx.step(args.warmup)
    ctx.sync()

    # ---- device-resident timed region: K steps replayed from CUDA graphs ----
    clocks = Clocks()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    ev0.record(stream)
    ctx.step(args.steps)          # one step-kernel launch per step
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ctx.sync()
    ms = max_over_ranks(world, ms)
    value = world * lu * args.steps / (ms * 1e-3) / 1e6
    launches = args.steps

    # cross-check: the same kernel with a CUDA-event pair around every launch
    nchk = min(args.steps, 500)
    ctx.set_profiling(True)
    ctx.kernel_time()
    ctx.step(nchk)
    kernel_ms, nk = ctx.kernel_time()
    ctx.set_profiling(False)
    ctx.sync()

    # ---- end to end through the public API with host buffers ----
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.set_solid(h_phi0)
    ctx.set_phase(h_phi1)
    ctx.step(args.steps)
    ctx.get_fields(o_phi1, o_u, o_p)
    e2e_s = time.perf_counter() - t0
    barrier(world)
    e2e_s = max_over_ranks(world, e2e_s)
    e2e = world * lu * args.steps / e2e_s / 1e6
    obs = ctx.observables(0)
    ctx.close()

    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    per_launch_ms = ms / args.steps          # timed region / launches (gaps included)
    achieved = BYTES_PER_LU * lu / (per_launch_ms * 1e-3) / 1e9
    traffic = traffic_from_profile(lu)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "lattice": "D2Q9", "nx": n, "ny": n, "instances": nb,
                   "thetas": [p["theta_deg"] for p in wl["params"]], "density_ratio": 10, "viscosity_ratio": 10,
                   "d0": 0.5, "W": 4.0, "lu_per_step": lu, "bytes_per_lu": BYTES_PER_LU,
                   "l2": f"no flush: each step reads {lu * 96 / 1e9:.2f} GB and writes {lu * 92 / 1e9:.2f} GB "
                         f"(> 129 MB L2)",
                   "parallelism": f"weak, {world} x independent 5-instance batches"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "kernel": "d2q9_step", "kernel_ms_per_launch": per_launch_ms, "launches": launches,
                     "bytes_per_lu": BYTES_PER_LU,
                     "event_bracketed_ms_per_launch": kernel_ms / max(nk, 1)},
        "e2e": {"value": e2e, "unit": "MLUPS", "h2d_bytes_per_step": 8 * lu / args.steps,
                "d2h_bytes_per_step": 16 * lu / args.steps,
                "note": "set_solid + set_phase from pinned host, K steps, get_fields to pinned host"},
        "gpu_launches": launches,
        "clocks": clk,
        "check": {"mass1": obs["mass1"], "umax": obs["umax"], "dp": obs["dp"]},
    }
    if world == 1 and not args.no_cpu_baseline:
        steps = 8
        side = oracle_sample_size(args.cpu_seconds, steps)
        try:
            mlups, secs = oracle_sample(side, steps)
            line["cpu_baseline"] = {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                    "sample": f"FP64 oracle, {steps} steps of a {side}x{side} crop of one instance "
                                              f"(theta 30 deg), {secs:.1f} s, 1 thread"}
        except Exception as e:   # the GPU number stands on its own
            line["cpu_baseline"] = {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                    "sample": f"failed: {str(e)[:200]}"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
