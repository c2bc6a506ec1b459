#!/usr/bin/env python3
"""Benchmark of the two-temperature cooling step (cool_step) on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: 256^3 = 16.8M cells, FP32 SoA fields (rho, B, H, u_e, u_i) of the
two-region synthetic MAD-like recipe (cold-thin ~1e7 K and hot ~1e10 K
regions), a 64^4 (+64, 64^2) FP32 log2 rate table (67 MB, L2-resident),
8 sub-cycles, explicit limited mode.  One step = one cool_step over all
cells.  Inputs (336 MB) exceed the 126 MB L2, so no flush is needed
between steps; the table is meant to stay in L2.

Prints ONE JSON line (rank 0).  Under torchrun each rank steps its own
256^3 problem (weak scaling, no data-path collective); the timing is the
max over ranks.  --impl reference times the FP64 CPU oracle on host cores
(the baseline arm), on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s of cool_step (fwd), 1 step = 16.8M cells x 8 sub-cycles"
UNIT = "cell-updates/s"
WORKLOAD = "two_region_256c"
TABLE_N = (64, 64, 64, 64, 64)
N_SUB = 8
BYTES_PER_CELL = 28  # FP32: read rho, B, H, u_e, u_i; write u_e, u_i


def config_dict(n_cells, world):
    return {"workload": "256^3 two-region MAD-like cells (synthetic, seeded)",
            "cells_per_gpu": n_cells, "table": "64^4 syn + 64 brems + 64^2 Coulomb, FP32 log2",
            "n_sub": N_SUB, "mode": "explicit-limited", "field_dtype": "f32",
            "l2": "inputs 336 MB > L2 (no flush needed); table L2-resident by design",
            "parallelism": f"cells sharded, {world} rank(s), no collective"}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


KERNEL_SOURCES = ("cool_step.cu", "cool_step_common.cuh", "cool_internal.cuh")


def kernel_source_sha():
    """sha256 (16 hex digits) over the sources the timed kernel is built from."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2505_08855_b300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (kernel_source_sha); else None."""
    sha = kernel_source_sha()
    for f in sorted(os.listdir(os.path.join(ROOT, "profiles"))) if os.path.isdir(os.path.join(ROOT, "profiles")) else []:
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(ROOT, "profiles", f)).read()
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha256_16:\s*([0-9a-f]+)\s+workload:\s*(\S+)", txt)
        if m and m.group(2) == sha and m.group(3) == WORKLOAD:
            return float(m.group(1))
    return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(n_cells_sample, nthreads, seed_off=0, repeats=1):
    """The FP64 oracle's step on a sample of the workload, host cores.  The
    oracle builds its 64^4 table first (untimed, like the GPU table)."""
    import oracle as O
    from paper_2505_08855_b300 import inputs
    spec = O.Spec(n=TABLE_N)
    t0 = time.time()
    T = O.build_tables(spec, nthreads=nthreads)
    t_build = time.time() - t0
    F = inputs.make(WORKLOAD)
    rng = np.random.default_rng(99 + seed_off)
    idx = np.sort(rng.choice(F["rho"].size, n_cells_sample, replace=False))
    sub = inputs.subsample(F, idx)
    p = O.Params(n_sub=N_SUB)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        O.step(spec, T, p, **sub, nthreads=nthreads)
        times.append(time.perf_counter() - t0)
    return n_cells_sample / min(times), t_build, times


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cores = host_cores()
    sample = 1 << 20
    import oracle as O
    from paper_2505_08855_b300 import inputs
    spec = O.Spec(n=TABLE_N)
    T = O.build_tables(spec, nthreads=cores)
    F = inputs.make(WORKLOAD)
    rng = np.random.default_rng(123)
    p = O.Params(n_sub=N_SUB)
    subs = []
    for k in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(F["rho"].size, sample, replace=False))
        subs.append(inputs.subsample(F, idx))
    del F
    for k in range(args.warmup):
        O.step(spec, T, p, **subs[k], nthreads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        O.step(spec, T, p, **subs[args.warmup + k], nthreads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    value = sample / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(sample, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} random cells of the 256^3 workload per step, FP64 O2 oracle, "
                                       f"{cores} threads; 64^4 oracle table built once, untimed"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return rc

    torch.cuda.set_device(local)
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build, inputs
    build.build()
    table = cool.Table(cool.TableSpec(n=TABLE_N))
    F = inputs.make(WORKLOAD, seed=1002 + rank)
    n = F["rho"].size
    dev = torch.device("cuda", local)
    tf = {k: torch.from_numpy(v).to(dev) for k, v in F.items()}
    ue_o = torch.empty_like(tf["ue"])
    ui_o = torch.empty_like(tf["ui"])
    params = cool.Params(n_sub=N_SUB)
    stream = torch.cuda.current_stream()

    def one():
        cool.step(table, params, tf["rho"], tf["B"], tf["H"], tf["ue"], tf["ui"], ue_out=ue_o, ui_out=ui_o)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n / (ms * 1e-3)

    # end to end through the public API with host buffers: pinned H2D of the
    # five input fields, the step, D2H of u_e and u_i, every step
    host_in = {k: torch.from_numpy(v).pin_memory() for k, v in F.items()}
    host_out = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    dev_in = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in F}
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out)

    def e2e_one():
        for k in F:
            dev_in[k].copy_(host_in[k], non_blocking=True)
        a, b = cool.step(table, params, dev_in["rho"], dev_in["B"], dev_in["H"], dev_in["ue"], dev_in["ui"],
                         ue_out=ue_o, ui_out=ui_o)
        host_out[0].copy_(a, non_blocking=True)
        host_out[1].copy_(b, non_blocking=True)

    for _ in range(2):
        e2e_one()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.e2e_steps
    if world > 1:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    e2e_value = world * n / (ms_e2e * 1e-3)

    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_CELL * n / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_per_launch(), "peak_source": peak_kind,
            "kernel": "k_step_f32<true>", "bytes_per_cell": BYTES_PER_CELL}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = host_cores()
        sample = 1 << 21
        rate, t_build, times = cpu_oracle_rate(sample, cores, repeats=2)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sample} random cells of the 256^3 workload, one 8-sub-cycle step, FP64 O2 "
                         f"oracle on {cores} threads (best of 2, {min(times):.1f} s); its 64^4 table "
                         f"built once untimed ({t_build:.0f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(n, world), "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
                "gpu_launches": args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
