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


KERNEL_SOURCES = ("cool_step.cu", "cool_step_kernel.cuh", "cool_step_cell.cuh", "cool_step_common.cuh")


def kernel_source_sha():
    """sha256 (16 hex digits) over the files that hold the timed kernel's
    device code (the step kernel and its shared device functions), with
    comments and trailing blanks removed: a change of wording does not
    change the kernel."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, "paper_2505_08855_b300", "csrc", name)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.rstrip() for line in src.split("\n") if line.strip())
        h.update(src.encode())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (kernel_source_sha); else None."""
    sha = kernel_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, f)).read()
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha256_16:\s*([0-9a-f]+)"
                      r"\s+workload:\s*(\S+)", txt)
        if m and m.group(2) == sha and m.group(3) == WORKLOAD:
            return float(m.group(1))
    return None


def ncu_utilisation():
    """Utilisation of the units that bind the step kernel, from the committed
    ncu summary of the current kernel sources (same keying as
    traffic_per_launch): {"l1_data_pipe": f, "issue_active": f} as fractions
    of their peaks, or None."""
    sha = kernel_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, f)).read()
        m = re.search(r"ncu_utilisation:\s*l1_data_pipe\s+([0-9.]+)\s+issue_active\s+([0-9.]+)"
                      r"\s+source_sha256_16:\s*([0-9a-f]+)\s+workload:\s*(\S+)", txt)
        if m and m.group(3) == sha and m.group(4) == WORKLOAD:
            return {"l1_data_pipe": float(m.group(1)), "issue_active": float(m.group(2))}
    return None


def issue_roofline(ms, n_cells, clk):
    """The step kernel against its instruction-issue roof: warp instructions
    per launch from the committed ncu summary of the current kernel sources
    (same keying as traffic_per_launch) over the launch time, against 148 SMs
    x 4 schedulers x 1 warp instruction per clock at the SM clock sampled
    during the timed region (the maximum clock when no sample was taken)."""
    sha = kernel_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    inst = tinst = None
    for f in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not f.endswith(".md"):
            continue
        txt = open(os.path.join(pdir, f)).read()
        m = re.search(r"issue:\s*warp_instructions_per_launch\s+([0-9.eE+]+)\s+thread_instructions_per_launch\s+"
                      r"([0-9.eE+]+)\s+source_sha256_16:\s*([0-9a-f]+)\s+workload:\s*(\S+)", txt)
        if m and m.group(3) == sha and m.group(4) == WORKLOAD:
            inst, tinst = float(m.group(1)), float(m.group(2))
    if inst is None:
        return None
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    peak = 148 * 4 * mhz * 1e6
    achieved = inst / (ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "sm_mhz": mhz, "warp_instructions_per_launch": inst,
            "thread_instructions_per_cell": tinst / n_cells,
            "source": "ncu smsp__inst_executed.sum / smsp__thread_inst_executed.sum of the committed capture"}


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


def job_rate(dist, world, ms_local, cells_per_rank, device):
    """Whole-job rate of a weak-scaled step: the slowest rank's time (max
    over ranks, one all-reduce of a scalar) and all ranks' cells over it.
    Returns (ms, cell-updates/s)."""
    ms = ms_local
    if world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * cells_per_rank / (ms * 1e-3)


def cell_shard(n, rank, world):
    """(first, count) of rank's contiguous block when n cells are split over
    world ranks (sizes differ by at most one cell)."""
    base, extra = divmod(n, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def cpu_oracle_rate(n_cells_sample, nthreads, seed_off=0, repeats=1, extra=None):
    """The FP64 oracle's step on a sample of the workload, host cores.  The
    oracle builds its 64^4 table first (untimed, like the GPU table).  With
    `extra` (a dict, filled in): the same O2 step on one thread over 65,536
    of the cells, and the O1 step (every rate from the formulas, the paper's
    analytic path) on all threads over 2,048 of them."""
    import oracle as O
    from paper_2505_08855_b300 import inputs
    spec = O.Spec(n=TABLE_N)
    t0 = time.time()
    T = O.build_tables(spec, nthreads=nthreads)
    t_build = time.time() - t0
    F = inputs.make(WORKLOAD)
    rng = np.random.default_rng(99 + seed_off)
    if n_cells_sample >= F["rho"].size:
        sub = F
    else:
        idx = np.sort(rng.choice(F["rho"].size, n_cells_sample, replace=False))
        sub = inputs.subsample(F, idx)
    p = O.Params(n_sub=N_SUB)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        out = O.step(spec, T, p, **sub, nthreads=nthreads)
        times.append(time.perf_counter() - t0)
    if extra is not None:
        extra["_outputs"] = (out[0], out[1])     # u_e, u_i of every sampled cell (for the error report)
        extra["_tables"] = (spec, T)
    if extra is not None:
        for key, m, threads, direct in (("o2_one_thread", 65536, 1, False), ("o1_direct", 2048, nthreads, True)):
            idx = np.sort(rng.choice(F["rho"].size, m, replace=False))
            part = inputs.subsample(F, idx)
            t0 = time.perf_counter()
            O.step(spec, T, p, **part, direct=direct, nthreads=threads)
            dt = time.perf_counter() - t0
            extra[key] = {"value": m / dt, "unit": UNIT, "threads": threads,
                          "sample": f"{m} random cells, one 8-sub-cycle step ({dt:.2f} s)"}
    return n_cells_sample / min(times), t_build, times


def rel_err_report(got, want):
    """Per-field error of the GPU against the FP64 oracle: max and 99.99th
    percentile of |got - want| / |want|, and the cells beyond 1e-5."""
    r = np.abs(got.astype(np.float64) - want) / np.abs(want)
    return {"max": float(r.max()), "p9999": float(np.quantile(r, 0.9999)), "beyond_1e-5": int((r > 1e-5).sum())}


FWD_BWD_WORKLOAD = "uniform_128c"
FWD_BWD_BYTES_PER_CELL = 76   # forward 28 B + backward: read 5 fields + 2 output adjoints, write 5 (48 B)


def fwd_bwd_gpu(torch, cool, inputs, dev, table, steps):
    """Forward + adjoint (cool_step, cool_step_bwd) on the 128^3 uniform cells
    with the 64^4 table, 8 sub-cycles, CUDA events on the launching stream:
    returns the timing dict and the adjoint outputs of the last launch."""
    G = inputs.make(FWD_BWD_WORKLOAD)
    m = G["rho"].size
    tg = {k: torch.from_numpy(v).to(dev) for k, v in G.items()}
    gl = [tg[k] for k in ("rho", "B", "H", "ue", "ui")]
    p = cool.Params(n_sub=N_SUB)
    g_ue = torch.ones(m, device=dev)
    g_ui = torch.full((m,), 0.5, device=dev)
    nH, nB, nN, nT, nC = TABLE_N
    tgr = {"lb": torch.zeros(nT, device=dev), "ls": torch.zeros(nH * nB * nN * nT, device=dev),
           "lc": torch.zeros(nC * nC, device=dev)}
    stream = torch.cuda.current_stream()
    out = {}

    def fwd():
        cool.step(table, p, *gl)

    def bwd():
        out["g"] = cool.step_bwd(table, p, *gl, g_ue, g_ui)

    def bwd_t():
        cool.step_bwd(table, p, *gl, g_ue, g_ui, tgr)

    # the autograd path: the forward keeps each cell's 2x5 Jacobian, the
    # backward contracts it with the output adjoints
    uo, vo = torch.empty_like(gl[3]), torch.empty_like(gl[4])
    J = torch.empty((10, m), device=dev)

    def fwd_jac():
        cool.step_fwd_jac(table, p, *gl, ue_out=uo, ui_out=vo, jac=J)

    def bwd_jac():
        out["gj"] = cool.step_bwd_jac(J, g_ue, g_ui)

    ms_f = _timed(torch, fwd, steps, 3, stream)
    ms_b = _timed(torch, bwd, steps, 3, stream)
    ms_bt = _timed(torch, bwd_t, steps, 3, stream)
    ms_fj = _timed(torch, fwd_jac, steps, 3, stream)
    ms_bj = _timed(torch, bwd_jac, steps, 3, stream)
    grads = [t.cpu().numpy() for t in out["gj"]]
    same = all(torch.equal(a, b) for a, b in zip(out["gj"], out["g"]))
    del tg, gl, g_ue, g_ui, tgr, out, uo, vo, J
    torch.cuda.empty_cache()
    return {"cells": m, "ms_fwd": ms_f, "ms_bwd": ms_b, "ms_bwd_with_table_adjoints": ms_bt,
            "ms_fwd_jac": ms_fj, "ms_bwd_jac": ms_bj, "jac_grads_equal_step_bwd": same}, grads, G


def fwd_bwd_oracle(G, grads, spec, T, nthreads, n_sample=1024, seed=1003):
    """The oracle's forward + adjoint on a seeded sample of the same cells
    (the CPU baseline of the fwd+bwd metric) and the GPU adjoint's error on
    it: |g_gpu - g_oracle| |x| / |L| per input (L = sum(u_e + u_i/2), the
    loss whose adjoint the GPU launch computed; a scale-free measure, since
    an adjoint can vanish)."""
    import oracle as O
    from paper_2505_08855_b300 import inputs
    m = G["rho"].size
    idx = np.sort(np.random.default_rng(seed).choice(m, n_sample, replace=False))
    sub = inputs.subsample(G, idx)
    t0 = time.perf_counter()
    want = O.step_bwd(spec, T, O.Params(n_sub=N_SUB), **sub, g_ue=np.ones(n_sample), g_ui=np.full(n_sample, 0.5),
                      nthreads=nthreads)
    dt = time.perf_counter() - t0
    L = np.abs(want["ue"] + 0.5 * want["ui"])
    err = {}
    for k, (name, fld) in enumerate(zip(("g_rho", "g_B", "g_H", "g_ue", "g_ui"), ("rho", "B", "H", "ue", "ui"))):
        e = np.abs(grads[k][idx] - want[name]) * np.abs(sub[fld]) / np.maximum(L, 1e-30)
        err[name] = {"max": float(e.max()), "median": float(np.median(e)), "beyond_2e-4": int((e > 2e-4).sum())}
    cpu = {"value": n_sample / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
           "sample": f"{n_sample} cells (seed {seed}) of the 128^3 uniform workload: the FP64 O2 oracle's forward "
                     f"recomputation and adjoint of one 8-sub-cycle step ({dt:.2f} s)"}
    return cpu, {"cells": n_sample, "measure": "|g_gpu - g_oracle| |x| / |L| per input, L = sum(u_e + u_i / 2)",
                 **err}


def host_cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


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


# ---- secondary measurements (--suite perf): one JSON line per case ---------------

def _timed(torch, fn, steps, warmup, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _timed_graph(torch, fn, steps, warmup, calls=10):
    """CUDA-event time per call of `fn` captured `calls` times in a CUDA
    graph and replayed: for kernels shorter than the Python call that
    launches them, where back-to-back calls would time the host."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(calls):
            fn()
    g.replay()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    del g
    return e0.elapsed_time(e1) / (steps * calls)


def _suite_line(case, workload, n, ms, extra=None, bytes_per_cell=None, peak=None):
    line = {"suite": "perf", "case": case, "workload": workload, "cells": n, "ms_per_step": ms,
            "value": n / (ms * 1e-3), "unit": UNIT, "higher_is_better": True}
    if bytes_per_cell is not None and peak is not None:
        a = bytes_per_cell * n / (ms * 1e-3) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
                            "bytes_per_cell": bytes_per_cell}
    if extra:
        line.update(extra)
    print(json.dumps(line), flush=True)


SECTIONS = ("cfg2", "paper_size", "staging_bound", "l2_persist", "disk", "radiation", "scalar", "fp64", "adjoint",
            "direct", "surrogate", "placement", "host_link", "nsub")


def run_suite_perf(args, torch, cool, inputs, dev):
    """Secondary measurements, one JSON line per case, by section (--section,
    default all): step variants on the benchmark workload (formats, modes,
    texture paths), the paper-size table, the disk geometry, the radiation
    correction, unaligned and FP64 fields, the forward + adjoint and the
    direct-formula step on 128^3 uniform cells, and the surrogate step on the
    512 x 256 x 256 shell."""
    want = set(SECTIONS) if args.section == "all" else set(args.section.split(","))
    stream = torch.cuda.current_stream()
    peak, _ = measured_peak()
    steps, warm = max(args.steps // 10, 3), 3
    tables = {}

    def table(dtype=cool.F32, scaled=0):
        key = (dtype, scaled)
        if key not in tables:
            tables[key] = cool.Table(cool.TableSpec(n=TABLE_N, dtype=dtype, row_scaled=scaled))
        return tables[key]

    def counters(t, p, fields, outs):
        c = cool.new_counters(dev)
        cool.step(t, p, *fields, ue_out=outs[0], ui_out=outs[1], counters=c)
        torch.cuda.synchronize()
        return {k: v for k, v in cool.counters_dict(c).items() if v}

    if want & {"cfg2", "paper_size", "staging_bound", "l2_persist", "disk", "radiation", "scalar", "fp64"}:
        F = inputs.make(WORKLOAD)
        n = F["rho"].size
        tf = {k: torch.from_numpy(v).to(dev) for k, v in F.items()}
        fl = [tf[k] for k in ("rho", "B", "H", "ue", "ui")]
        ue_o, ui_o = torch.empty_like(tf["ue"]), torch.empty_like(tf["ui"])
        del F
    if "cfg2" in want:
        cases = [("explicit, FP32 table", cool.F32, 0, cool.Params(n_sub=N_SUB), steps),
                 ("explicit, fp64_critical", cool.F32, 0, cool.Params(n_sub=N_SUB, fp64_critical=1), steps),
                 ("implicit (Illinois, FP32)", cool.F32, 0, cool.Params(n_sub=N_SUB, mode=cool.IMPLICIT), steps),
                 ("implicit, fp64_critical", cool.F32, 0, cool.Params(n_sub=N_SUB, mode=cool.IMPLICIT,
                                                                        fp64_critical=1), 3),
                 ("explicit, BF16 table", cool.BF16, 0, cool.Params(n_sub=N_SUB), steps),
                 ("explicit, FP16 table", cool.F16, 0, cool.Params(n_sub=N_SUB), steps),
                 ("explicit, BF16 row-scaled table", cool.BF16, 1, cool.Params(n_sub=N_SUB), steps),
                 ("explicit, FP16 row-scaled table", cool.F16, 1, cool.Params(n_sub=N_SUB), steps),
                 ("explicit, N_sub = 1", cool.F32, 0, cool.Params(n_sub=1), steps),
                 ("explicit, TMA-staged fields (bulk copies, double-buffered)", cool.F32, 0,
                  cool.Params(n_sub=N_SUB, path=cool.PATH_TMA_SMEM), steps),
                 ("explicit, texture path: point fetches + FP32 lerp", cool.F32, 0,
                  cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_POINT), steps),
                 ("explicit, texture path: hardware trilinear filtering", cool.F32, 0,
                  cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_HWLERP), steps),
                 ("explicit, the paper's layout: one 4-D table of Q_total (bridge folded in)", cool.F32, 0,
                  cool.Params(n_sub=N_SUB, path=cool.PATH_QTOTAL), steps)]
        for name, dt, sc, p, k in cases:
            t = table(dt, sc)
            ms = _timed(torch, lambda: cool.step(t, p, *fl, ue_out=ue_o, ui_out=ui_o), k, warm, stream)
            _suite_line(name, WORKLOAD, n, ms, {"counters": counters(t, p, fl, (ue_o, ui_o)),
                                                "table_packed_bytes": t.packed_bytes()},
                        BYTES_PER_CELL, peak)
    if "paper_size" in want:
        # the paper's table size (100 nodes per axis): 457 MB packed, far beyond L2
        big = cool.Table(cool.TableSpec(n=(100,) * 5))
        for name, path in (("paper-size 100^4 table, L2 block layout", cool.PATH_L2WINDOW),
                           ("paper-size 100^4 table, the paper's layout (one Q_total table)", cool.PATH_QTOTAL),
                           ("paper-size 100^4 table, texture hardware filtering", cool.PATH_TEXTURE_HWLERP),
                           ("paper-size 100^4 table, texture point fetches", cool.PATH_TEXTURE_POINT)):
            p = cool.Params(n_sub=N_SUB, path=path)
            ms = _timed(torch, lambda: cool.step(big, p, *fl, ue_out=ue_o, ui_out=ui_o), steps, warm, stream)
            _suite_line(name, WORKLOAD, n, ms, {"table_packed_bytes": big.packed_bytes()}, BYTES_PER_CELL, peak)
        big.free()
        del big
        # the 16-bit storage formats at that size: half the table bytes (still
        # beyond L2), so fewer of the gathers' sectors miss L2
        for name, dt, sc in (("paper-size 100^4 table, BF16", cool.BF16, 0),
                             ("paper-size 100^4 table, FP16", cool.F16, 0),
                             ("paper-size 100^4 table, BF16 block-scaled", cool.BF16, 1),
                             ("paper-size 100^4 table, FP16 block-scaled", cool.F16, 1)):
            big = cool.Table(cool.TableSpec(n=(100,) * 5, dtype=dt, row_scaled=sc))
            p = cool.Params(n_sub=N_SUB)
            ms = _timed(torch, lambda: cool.step(big, p, *fl, ue_out=ue_o, ui_out=ui_o), steps, warm, stream)
            _suite_line(name, WORKLOAD, n, ms, {"table_packed_bytes": big.packed_bytes()}, BYTES_PER_CELL, peak)
            big.free()
            del big
    if "staging_bound" in want:
        # what staging the 4-D channel on chip could gain at most: the same
        # step with a 4-D channel of 2x2x2 (H, B, n_e) corners x 64 T_e nodes
        # (10 KB, L1-resident: every gather hits L1) against the 64^4 table
        # (75.5 MB, L2-resident), at 1 and 8 sub-cycles
        for nn, label in (((64, 64, 64, 64, 64), "64^4 table (L2-resident)"),
                          ((2, 2, 2, 64, 64), "2x2x2x64 4-D channel (L1-resident)")):
            tt = cool.Table(cool.TableSpec(n=nn))
            for ns in (1, N_SUB):
                p = cool.Params(n_sub=ns)
                ms = _timed(torch, lambda: cool.step(tt, p, *fl, ue_out=ue_o, ui_out=ui_o), steps, warm, stream)
                _suite_line(f"staging bound: {label}, N_sub = {ns}", WORKLOAD, n, ms,
                            {"table_packed_bytes": tt.packed_bytes()}, BYTES_PER_CELL, peak)
            tt.free()
            del tt
    if "l2_persist" in want:
        # the opt-in persisting-L2 reservation of the packed channel
        # (cool_table_l2_persist): the step with and without it, and the
        # radiation correction (a streaming kernel) run after it in the same
        # context
        thick = torch.empty(n, dtype=torch.uint8, device=dev)
        p = cool.Params(n_sub=N_SUB)
        t = table()
        for on in (False, True):
            t.l2_persist(on)
            ms = _timed(torch, lambda: cool.step(t, p, *fl, ue_out=ue_o, ui_out=ui_o), steps, warm, stream)
            _suite_line(f"L2 reservation {'on' if on else 'off'}: step, 64^4 table (75.5 MB)", WORKLOAD, n, ms,
                        None, BYTES_PER_CELL, peak)
            ms = _timed_graph(torch, lambda: cool.radiation_te(p, tf["rho"], tf["H"], tf["ue"], te_out=ue_o,
                                                               thick_out=thick), steps, warm)
            _suite_line(f"L2 reservation {'on' if on else 'off'}: radiation correction after it", WORKLOAD, n, ms,
                        {"timing": "CUDA graph of 10 calls, replayed"}, 17, peak)
        t.l2_persist(False)
        del thick
        # a table larger than L2: 128 x 128 x 64 x 64 FP32 (302 MB packed) on
        # the 448 x 192 x 192 shell
        S = inputs.make("shell_448x192x192")
        sf = [torch.from_numpy(S[k]).to(dev) for k in ("rho", "B", "H", "ue", "ui")]
        ns = sf[0].numel()
        del S
        so = (torch.empty_like(sf[3]), torch.empty_like(sf[4]))
        big = cool.Table(cool.TableSpec(n=(128, 128, 64, 64, 64)))
        for on in (False, True):
            big.l2_persist(on)
            ms = _timed(torch, lambda: cool.step(big, p, *sf, ue_out=so[0], ui_out=so[1]), steps, warm, stream)
            _suite_line(f"L2 reservation {'on' if on else 'off'}: step, 128x128x64x64 table (302 MB)",
                        "shell_448x192x192", ns, ms, {"table_packed_bytes": big.packed_bytes()}, BYTES_PER_CELL,
                        peak)
        big.free()
        del big, sf, so
    if "disk" in want:
        # the disk geometry fused into the step (H_th from the state, floor)
        r_dev = torch.from_numpy(inputs.make(WORKLOAD, with_r=True)["r"]).to(dev)
        for name, disk in (("disk geometry: H_th from the state (H not read)", cool.Disk(h_from_state=1)),
                           ("disk geometry: H_th from the state + temperature floor 0.1",
                            cool.Disk(h_from_state=1, h_floor=0.1))):
            p = cool.Params(n_sub=N_SUB)
            ms = _timed(torch, lambda: cool.step_disk(table(), p, disk, tf["rho"], tf["B"], None, tf["ue"],
                                                      tf["ui"], r_dev, ue_out=ue_o, ui_out=ui_o), steps, warm,
                        stream)
            c = cool.new_counters(dev)
            cool.step_disk(table(), p, disk, tf["rho"], tf["B"], None, tf["ue"], tf["ui"], r_dev, ue_out=ue_o,
                           ui_out=ui_o, counters=c)
            torch.cuda.synchronize()
            _suite_line(name, WORKLOAD, n, ms, {"counters": {k: v for k, v in cool.counters_dict(c).items() if v}},
                        BYTES_PER_CELL, peak)
        del r_dev
    if "radiation" in want:
        # radiation-pressure correction of T_e: an elementwise pass (12 B
        # read, 4 B T_e + 1 B flag written per cell), 285 MB per pass > L2
        thick = torch.empty(n, dtype=torch.uint8, device=dev)
        p = cool.Params(n_sub=N_SUB)
        ms = _timed_graph(torch, lambda: cool.radiation_te(p, tf["rho"], tf["H"], tf["ue"], te_out=ue_o,
                                                           thick_out=thick), steps, warm)
        _suite_line("radiation-pressure T_e correction (Sec. 5.2 quartic), elementwise", WORKLOAD, n, ms,
                    {"thick_cells": int(thick.sum().item()), "timing": "CUDA graph of 10 calls, replayed"}, 17,
                    peak)
        del thick
    if "scalar" in want:
        # unaligned fields: the scalar path
        off = {k: torch.cat([v[:1], v])[1:] for k, v in tf.items()}
        ofl = [off[k] for k in ("rho", "B", "H", "ue", "ui")]
        p = cool.Params(n_sub=N_SUB)
        ms = _timed(torch, lambda: cool.step(table(), p, *ofl), steps, warm, stream)
        _suite_line("explicit, fields not 16-byte aligned (scalar path)", WORKLOAD, n, ms, None, BYTES_PER_CELL,
                    peak)
        del off, ofl
    if "fp64" in want:
        # FP64 fields (all-FP64 kernel)
        p = cool.Params(n_sub=N_SUB)
        f64 = [v.double() for v in fl]
        o64 = [torch.empty_like(f64[3]), torch.empty_like(f64[4])]
        ms = _timed(torch, lambda: cool.step(table(), p, *f64, ue_out=o64[0], ui_out=o64[1]), 3, 1, stream)
        _suite_line("FP64 fields and arithmetic", WORKLOAD, n, ms, None, 56, peak)
        del f64, o64
    if want & {"cfg2", "paper_size", "staging_bound", "l2_persist", "disk", "radiation", "scalar", "fp64"}:
        del tf, fl, ue_o, ui_o
        torch.cuda.empty_cache()

    if want & {"adjoint", "direct"}:
        # forward + adjoint, 128^3 uniform cells
        G = inputs.make("uniform_128c")
        m = G["rho"].size
        tg = {k: torch.from_numpy(v).to(dev) for k, v in G.items()}
        gl = [tg[k] for k in ("rho", "B", "H", "ue", "ui")]
        T = table()
        p = cool.Params(n_sub=N_SUB)
        ms_f = _timed(torch, lambda: cool.step(T, p, *gl), steps * 5, warm, stream)
        _suite_line("forward, 128^3 uniform", "uniform_128c", m, ms_f, None, BYTES_PER_CELL, peak)
    if "adjoint" in want:
        g_ue = torch.ones_like(tg["ue"])
        g_ui = torch.full_like(tg["ui"], 0.5)
        nH, nB, nN, nT, nC = TABLE_N
        tgr = {"lb": torch.zeros(nT, device=dev), "ls": torch.zeros(nH * nB * nN * nT, device=dev),
               "lc": torch.zeros(nC * nC, device=dev)}
        ms_b = _timed(torch, lambda: cool.step_bwd(T, p, *gl, g_ue, g_ui), steps * 5, warm, stream)
        ms_bt = _timed(torch, lambda: cool.step_bwd(T, p, *gl, g_ue, g_ui, tgr), steps * 5, warm, stream)
        _suite_line("adjoint (inputs only), 128^3 uniform", "uniform_128c", m, ms_b, None, 48, peak)
        _suite_line("forward + adjoint (inputs only), 128^3 uniform", "uniform_128c", m, ms_f + ms_b, None, 76,
                    peak)
        _suite_line("forward + adjoint (inputs and table), 128^3 uniform", "uniform_128c", m, ms_f + ms_bt, None,
                    76, peak)
        # the autograd path: the forward keeps each cell's Jacobian, the
        # backward contracts it (explicit and implicit mode)
        uo, vo = torch.empty_like(gl[3]), torch.empty_like(gl[4])
        J = torch.empty((10, m), device=dev)
        for mode, label in ((cool.EXPLICIT, ""), (cool.IMPLICIT, ", implicit mode")):
            pm = cool.Params(n_sub=N_SUB, mode=mode)
            ms_fj = _timed(torch, lambda: cool.step_fwd_jac(T, pm, *gl, ue_out=uo, ui_out=vo, jac=J), steps * 5,
                           warm, stream)
            ms_bj = _timed(torch, lambda: cool.step_bwd_jac(J, g_ue, g_ui), steps * 5, warm, stream)
            _suite_line(f"forward with Jacobian + its contraction{label}, 128^3 uniform", "uniform_128c", m,
                        ms_fj + ms_bj, {"ms_fwd_jac": ms_fj, "ms_bwd_jac": ms_bj}, 76, peak)
        del g_ue, g_ui, tgr, uo, vo, J
    if "direct" in want:
        # the paper's analytic-versus-table comparison: every rate from the
        # formulas (FP64), on the first 2^18 of these cells
        k = 1 << 18
        d64 = [t[:k].double().contiguous() for t in gl]
        ms_d = _timed(torch, lambda: cool.step_direct(cool.TableSpec(n=TABLE_N), p, *d64), 1, 1, stream)
        _suite_line("direct formulas, no table (FP64), 2^18 of the 128^3 uniform cells", "uniform_128c", k, ms_d,
                    {"table_step_speedup": (m / (ms_f * 1e-3)) / (k / (ms_d * 1e-3))}, 56, peak)
        del d64
    if want & {"adjoint", "direct"}:
        del tg, gl
        torch.cuda.empty_cache()

    if "placement" in want:
        # where the table lives, one short run per choice (1 untimed + 2
        # timed launches each, so that one ncu capture of every k_step launch
        # of this section covers all of them): the L2 block layout (default),
        # the same with the persisting-L2 reservation, the two texture paths,
        # the TMA-staged fields, the block-scaled BF16 table; the paper-size
        # 100^4 table (beyond L2) on the block layout and both texture paths;
        # then, on the 448 x 192 x 192 shell (spatially coherent cells), the bound on
        # staging the table per tile: the same step with a 4-D channel of
        # 2x2x2 corners x 64 T_e nodes (L1-resident) against the
        # 128 x 128 x 64 x 64 table (302 MB).
        F = inputs.make(WORKLOAD)
        n = F["rho"].size
        fl = [torch.from_numpy(F[k]).to(dev) for k in ("rho", "B", "H", "ue", "ui")]
        uo, io = torch.empty_like(fl[3]), torch.empty_like(fl[4])
        del F
        p8 = cool.Params(n_sub=N_SUB)
        t32 = cool.Table(cool.TableSpec(n=TABLE_N))
        tbs = cool.Table(cool.TableSpec(n=TABLE_N, dtype=cool.BF16, row_scaled=1))
        runs = [("L2 block layout (default)", t32, p8, False),
                ("L2 block layout + persisting-L2 reservation", t32, p8, True),
                ("texture, point fetches + FP32 lerp", t32, cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_POINT),
                 False),
                ("texture, hardware trilinear filtering", t32,
                 cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_HWLERP), False),
                ("TMA-staged field tiles", t32, cool.Params(n_sub=N_SUB, path=cool.PATH_TMA_SMEM), False),
                ("BF16 block-scaled table", tbs, p8, False)]
        for name, t, p, persist in runs:
            t.l2_persist(persist)
            ms = _timed(torch, lambda: cool.step(t, p, *fl, ue_out=uo, ui_out=io), 2, 1, stream)
            t.l2_persist(False)
            _suite_line(f"placement: {name}", WORKLOAD, n, ms, {"table_packed_bytes": t.packed_bytes()},
                        BYTES_PER_CELL, peak)
        t32.free()
        tbs.free()
        # the paper's table size (100 nodes per axis; 457 MB packed, 3.6x L2):
        # the block layout against both texture paths beyond L2
        big = cool.Table(cool.TableSpec(n=(100,) * 5))
        for name, p in (("100^4 table, L2 block layout", p8),
                        ("100^4 table, texture, hardware trilinear filtering",
                         cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_HWLERP)),
                        ("100^4 table, texture, point fetches + FP32 lerp",
                         cool.Params(n_sub=N_SUB, path=cool.PATH_TEXTURE_POINT))):
            ms = _timed(torch, lambda: cool.step(big, p, *fl, ue_out=uo, ui_out=io), 2, 1, stream)
            _suite_line(f"placement: {name}", WORKLOAD, n, ms, {"table_packed_bytes": big.packed_bytes()},
                        BYTES_PER_CELL, peak)
        big.free()
        del fl, uo, io
        S = inputs.make("shell_448x192x192")
        sf = [torch.from_numpy(S[k]).to(dev) for k in ("rho", "B", "H", "ue", "ui")]
        ns = sf[0].numel()
        del S
        so = (torch.empty_like(sf[3]), torch.empty_like(sf[4]))
        for nn, label in (((128, 128, 64, 64, 64), "128x128x64x64 table (302 MB)"),
                          ((2, 2, 2, 64, 64), "2x2x2x64 4-D channel (L1-resident)")):
            tt = cool.Table(cool.TableSpec(n=nn))
            ms = _timed(torch, lambda: cool.step(tt, p8, *sf, ue_out=so[0], ui_out=so[1]), 2, 1, stream)
            _suite_line(f"placement: shell staging bound, {label}", "shell_448x192x192", ns, ms,
                        {"table_packed_bytes": tt.packed_bytes()}, BYTES_PER_CELL, peak)
            tt.free()
        del sf, so
        torch.cuda.empty_cache()

    if "surrogate" in want:
        # the surrogate step on the 512 x 256 x 256 shell (training untimed)
        S = inputs.make("shell_512x256x256")
        m = S["rho"].size
        ts = {k: torch.from_numpy(v).to(dev) for k, v in S.items()}
        del S
        sl = [ts[k] for k in ("rho", "B", "H", "ue", "ui")]
        so = [torch.empty_like(ts["ue"]), torch.empty_like(ts["ui"])]
        T = table()
        p = cool.Params(n_sub=N_SUB)
        t0 = time.time()
        sur = cool.Surrogate(T, cool.FitSpec(epochs=args.fit_epochs))
        torch.cuda.synchronize()
        fit_s = time.time() - t0
        info = sur.info()
        ms_t = _timed(torch, lambda: cool.step(T, p, *sl, ue_out=so[0], ui_out=so[1]), steps, warm, stream)
        _suite_line("table step, 512x256x256 shell", "shell_512x256x256", m, ms_t, None, BYTES_PER_CELL, peak)
        cells = info["mask_cells"]
        for name, bits in (("surrogate step, fitted fallback mask (tol 1e-3)", None),
                           ("surrogate step, network in every cell", np.zeros((cells + 31) // 32, np.uint32))):
            if bits is not None:
                sur.set_mask(bits)
            ms = _timed(torch, lambda: sur.step(p, *sl, ue_out=so[0], ui_out=so[1]), steps, warm, stream)
            c = cool.new_counters(dev)
            sur.step(p, *sl, ue_out=so[0], ui_out=so[1], counters=c)
            torch.cuda.synchronize()
            cd = cool.counters_dict(c)
            evals = N_SUB * (m - cd["fallback"])
            flops = 2.0 * 17024 * evals
            _suite_line(name, "shell_512x256x256", m, ms,
                        {"fallback_cells": cd["fallback"], "fit_seconds": fit_s, "fit": info,
                         "network_tflops": flops / (ms * 1e-3) / 1e12}, BYTES_PER_CELL, peak)
        sur.free()
    if "nsub" in want:
        # the step's time against the number of sub-cycles (the benchmark's
        # cells and table): the per-cell part and the cost of one sub-cycle
        F = inputs.make(WORKLOAD)
        n = F["rho"].size
        fl = [torch.from_numpy(F[k]).to(dev) for k in ("rho", "B", "H", "ue", "ui")]
        del F
        uo, io = torch.empty_like(fl[3]), torch.empty_like(fl[4])
        for ns in (1, 2, 4, 8, 16, 32):
            p = cool.Params(n_sub=ns)
            ms = _timed(torch, lambda: cool.step(table(), p, *fl, ue_out=uo, ui_out=io), steps, warm, stream)
            _suite_line(f"explicit, N_sub = {ns}", WORKLOAD, n, ms, None, BYTES_PER_CELL, peak)
        del fl, uo, io
    if "host_link" in want:
        # the end-to-end step's floor: the benchmark's 5 input fields host ->
        # device and its 2 outputs back, alone and at once, beside
        # cool_step_host (pinned host memory, 256^3 cells)
        F = inputs.make(WORKLOAD, seed=1002)
        n = F["rho"].size
        hin = {k: torch.from_numpy(v).pin_memory() for k, v in F.items()}
        del F
        hout = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
        din = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in hin}
        dout = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
        side = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

        def h2d():
            for k in hin:
                din[k].copy_(hin[k], non_blocking=True)

        def d2h():
            for a in range(2):
                hout[a].copy_(dout[a], non_blocking=True)

        def both():
            for st in side:
                st.wait_stream(stream)
            with torch.cuda.stream(side[0]):
                h2d()
            with torch.cuda.stream(side[1]):
                d2h()
            for st in side:
                stream.wait_stream(st)

        t = table()
        p = cool.Params(n_sub=N_SUB)
        res = {"h2d_ms": _timed(torch, h2d, steps, warm, stream), "d2h_ms": _timed(torch, d2h, steps, warm, stream),
               "both_at_once_ms": _timed(torch, both, steps, warm, stream),
               "step_host_ms": _timed(torch, lambda: cool.step_host(t, p, hin["rho"], hin["B"], hin["H"], hin["ue"],
                                                                    hin["ui"], hout[0], hout[1]), steps, warm, stream)}
        res["h2d_GBps"] = 20.0 * n / res["h2d_ms"] / 1e6
        res["d2h_GBps"] = 8.0 * n / res["d2h_ms"] / 1e6
        _suite_line("end to end through cool_step_host, and the host link alone", WORKLOAD, n, res["step_host_ms"],
                    res)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--suite", default=None, choices=["perf"],
                    help="secondary measurements, one JSON line per case, instead of the benchmark line")
    ap.add_argument("--section", default="all",
                    help="with --suite perf: comma-separated subset of " + ",".join(SECTIONS))
    ap.add_argument("--fit-epochs", type=int, default=16,
                    help="with --suite perf: training epochs of the surrogate (0: untrained network)")
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
    if args.suite is not None:
        if rank != 0:
            return 0
        return run_suite_perf(args, torch, cool, inputs, torch.device("cuda", local))
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
    ms, value = job_rate(dist, world, ms, n, dev)
    # each step on its own (events around every step, after the timed
    # region): the median and the spread of single steps beside the mean
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for s_i in range(args.steps):
        one()
        ev[s_i + 1].record(stream)
    torch.cuda.synchronize()
    singles = sorted(ev[s_i].elapsed_time(ev[s_i + 1]) for s_i in range(args.steps))
    per_step = {"median": singles[len(singles) // 2], "min": singles[0], "max": singles[-1],
                "total_ms": ms * args.steps}

    # end to end through the public API with host buffers (cool_step_host):
    # every step copies the five input fields from pinned host memory and
    # u_e, u_i back, in chunks that overlap copies and steps
    host_in = {k: torch.from_numpy(v).pin_memory() for k, v in F.items()}
    host_out = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out)

    def e2e_one():
        cool.step_host(table, params, host_in["rho"], host_in["B"], host_in["H"], host_in["ue"], host_in["ui"],
                       host_out[0], host_out[1])

    for _ in range(2):
        e2e_one()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.e2e_steps
    ms_e2e, e2e_value = job_rate(dist, world, ms_e2e, n, dev)

    # forward + adjoint (rank 0 only: a secondary measurement of this line)
    fb = None
    if rank == 0:
        fb_t, fb_grads, fb_G = fwd_bwd_gpu(torch, cool, inputs, dev, table, max(args.steps, 10))

    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_CELL * n / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_per_launch(), "peak_source": peak_kind,
            "kernel": "k_step_f32<true>", "bytes_per_cell": BYTES_PER_CELL,
            # what binds instead of HBM (ncu, fractions of each unit's peak)
            "ncu_utilisation": ncu_utilisation()}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = host_cores()
        sample = n   # every cell of the workload: about 2 s per step on 16 cores
        more = {}
        rate, t_build, times = cpu_oracle_rate(sample, cores, repeats=3, extra=more)
        o_ue, o_ui = more.pop("_outputs")
        ospec, otab = more.pop("_tables")
        max_err = {"u_e": rel_err_report(ue_o.cpu().numpy(), o_ue), "u_i": rel_err_report(ui_o.cpu().numpy(), o_ui),
                   "cells": int(o_ue.size), "against": "FP64 O2 oracle, same cells, same table spec",
                   "tolerance": 1e-5}
        fb_cpu, fb_err = fwd_bwd_oracle(fb_G, fb_grads, ospec, otab, cores)
        del o_ue, o_ui, otab
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all {sample} cells of the 256^3 workload, one 8-sub-cycle step, FP64 O2 "
                         f"oracle on {cores} threads (best of 3: {min(times):.1f} s, "
                         f"{sum(times):.1f} s in all); its 64^4 table built once untimed ({t_build:.0f} s)",
               "host": host_cpu_model(), **more}

    if rank == 0:
        # the library's autograd path (cool_step_fn): cool_step_fwd_jac, then
        # cool_step_bwd_jac; beside it cool_step + cool_step_bwd (the
        # sub-cycles recomputed in the backward), and with table adjoints
        ms_fb = fb_t["ms_fwd_jac"] + fb_t["ms_bwd_jac"]
        ms_fr = fb_t["ms_fwd"] + fb_t["ms_bwd"]
        m_fb = fb_t["cells"]
        a_fb = FWD_BWD_BYTES_PER_CELL * m_fb / (ms_fb * 1e-3) / 1e9
        ms_fbt = fb_t["ms_fwd"] + fb_t["ms_bwd_with_table_adjoints"]
        fb = {"value": m_fb / (ms_fb * 1e-3), "unit": UNIT, "ms_per_step": ms_fb,
              "workload": "128^3 uniform cells (synthetic, seeded), 64^4 FP32 table, 8 sub-cycles",
              "path": "cool_step_fwd_jac (outputs + each cell's 2x5 Jacobian, 40 B/cell kept) + "
                      "cool_step_bwd_jac (the contraction with the output adjoints)",
              "ms_fwd": fb_t["ms_fwd_jac"], "ms_bwd": fb_t["ms_bwd_jac"],
              "grads_equal_step_bwd": fb_t["jac_grads_equal_step_bwd"],
              "roofline": {"bound": "hbm", "achieved": a_fb, "peak": peak, "unit": "GB/s", "frac": a_fb / peak,
                           "bytes_per_cell": FWD_BWD_BYTES_PER_CELL, "peak_source": peak_kind},
              "recomputed": {"value": m_fb / (ms_fr * 1e-3), "ms_per_step": ms_fr, "ms_fwd": fb_t["ms_fwd"],
                             "ms_bwd": fb_t["ms_bwd"], "path": "cool_step + cool_step_bwd (sub-cycles recomputed)"},
              "with_table_adjoints": {"value": m_fb / (ms_fbt * 1e-3), "ms_per_step": ms_fbt,
                                      "ms_bwd": fb_t["ms_bwd_with_table_adjoints"]}}
        if cpu is not None:
            fb["cpu_baseline"] = fb_cpu
            fb["max_err"] = fb_err
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "per_step_ms": per_step,
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_dict(n, world), "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
                "gpu_launches": args.steps, "clocks": clk,
                "fwd_bwd": fb, "max_rel_err": max_err if cpu is not None else None,
                "issue_roofline": issue_roofline(ms, n, clk)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
