"""Precision of the reduced-storage tables on the 448 x 192 x 192 shell with
a 128 x 128 x 64 x 64 table (H, B, n_e, T_e; Coulomb 64^2): the report of
what each storage format and FP64 option costs and buys, with the bars it
must meet.

For each 4-D storage format (FP32, BF16, FP16, BF16 and FP16 row-scaled):
  * the storage error of the synchrotron channel (max |stored - exact| of
    its log2 values over a fixed subset of rows, through the oracle's
    packing mirror applied to the library's FP64 channel);
  * the step's relative error per field (u_e, u_i, q_cool) at 2048 sampled
    cells against the FP64 oracle on the FP64 table (O2) and on the direct
    formulas (O1);
  * cell-updates/s of the explicit step over the whole shell.
Then the FP64 options on the FP32 table: the fraction of cells that take
FP64 (equilibrium band, stiff implicit cells) and the step rate.  And the
interpolation error of each process (O2 vs O1 at the sampled cells' keys).

Bars: the FP32 table meets the FP32 parity bar (1e-5) at this size; a
16-bit format's step error stays within twice its channel's storage error
(the step is a contraction of rate errors: the limiter caps the removed
energy, the bridge is monotone); row scaling lowers the storage error.
Lines starting with REPORT are JSON.
"""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

N5 = (128, 128, 64, 64, 64)
SAMPLE = 2048
FORMATS = [("FP32", 0, 0, 0), ("BF16", 1, 0, 1), ("FP16", 2, 0, 2), ("BF16 row-scaled", 1, 1, 3),
           ("FP16 row-scaled", 2, 1, 4)]


def report(d):
    print("REPORT " + json.dumps(d), flush=True)


@pytest.fixture(scope="module")
def env(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    F = inputs.make("shell_448x192x192")
    n = F["rho"].size
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(n, SAMPLE, replace=False))
    sub = {k: v[idx].astype(np.float64) for k, v in F.items()}
    ospec = oracle.Spec(n=N5)
    prm = oracle.Params(n_sub=8)
    lazy = oracle.build_tables(ospec, syn=False)
    o2 = oracle.step(ospec, lazy, prm, sub["rho"], sub["B"], sub["H"], sub["ue"], sub["ui"], lazy=True)
    o1 = oracle.step(ospec, lazy, prm, sub["rho"], sub["B"], sub["H"], sub["ue"], sub["ui"], direct=True)
    return cool, F, idx, sub, ospec, lazy, o1, o2


def _errs(got, want, ue_in):
    out = {}
    for name, k in (("u_e", 0), ("u_i", 1)):
        r = np.abs(got[k] - want[k]) / np.abs(want[k])
        out[name] = {"max": float(r.max()), "median": float(np.median(r))}
    r = np.abs(got[2] - want[2]) / ue_in
    out["q_cool/u_e"] = {"max": float(r.max()), "median": float(np.median(r))}
    return out


def _gpu_step(cool, table, p, tf):
    fl = [tf[k] for k in ("rho", "B", "H", "ue", "ui")]
    qc = torch.empty_like(tf["ue"])
    cnt = cool.new_counters()
    ue, ui = cool.step(table, p, *fl, q_cool=qc, counters=cnt)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        cool.step(table, p, *fl)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5 if p.fp64_critical == 0 or p.mode == 0 else 1
    e0.record(stream)
    for _ in range(reps):
        cool.step(table, p, *fl)
    e1.record(stream)
    torch.cuda.synchronize()
    return ue, ui, qc, cool.counters_dict(cnt), e0.elapsed_time(e1) / reps


def test_formats_on_the_shell(env, oracle):
    from oracle import quant
    cool, F, idx, sub, ospec, lazy, o1, o2 = env
    n = F["rho"].size
    tf = {k: torch.from_numpy(v).cuda() for k, v in F.items()}
    p = cool.Params(n_sub=8)
    ti = torch.from_numpy(idx).cuda()
    storage = {}
    for name, dtype, scaled, fmt in FORMATS:
        t = cool.Table(cool.TableSpec(n=N5, dtype=dtype, row_scaled=scaled))
        ue, ui, qc, cnt, ms = _gpu_step(cool, t, p, tf)
        got = [a[ti].cpu().numpy().astype(np.float64) for a in (ue, ui, qc)]
        ls = t.export(1).reshape(-1, N5[3])[::16]
        st = quant.storage_error(ls, N5[3], fmt)
        storage[name] = st
        line = {"suite": "precision", "case": f"{name} table, explicit", "workload": "shell_448x192x192",
                "table": "128x128x64x64 syn + 64 brems + 64^2 Coulomb", "cells": n, "ms_per_step": ms,
                "cell_updates_per_s": n / (ms * 1e-3), "packed_bytes": t.packed_bytes(),
                "syn_storage_max_abs_dlog2": st, "syn_storage_max_rel": float(2.0 ** st - 1.0),
                "vs_O2": _errs(got, o2, sub["ue"]), "vs_O1": _errs(got, o1, sub["ue"]), "sample": SAMPLE,
                "counters": cnt}
        report(line)
        e = line["vs_O2"]
        if fmt == 0:
            assert e["u_e"]["max"] <= 1e-5 and e["u_i"]["max"] <= 1e-5
        else:
            bound = 2.0 * (2.0 ** st - 1.0) + 1e-5
            assert e["u_e"]["max"] <= bound and e["u_i"]["max"] <= bound, (name, e, bound)
        t.free()
    assert storage["BF16 row-scaled"] < storage["BF16"] and storage["FP16 row-scaled"] < storage["FP16"]


def test_paper_layout_on_the_shell(env, oracle):
    """The paper's table layout (one 4-D table of Q_total, the bridge folded
    in at the nodes) against the factored layout (brems, synchrotron, bridge
    at run time), both from the FP32 table, at the sampled cells against the
    direct formulas (O1): what interpolating the bridged rate costs."""
    cool, F, idx, sub, ospec, lazy, o1, o2 = env
    n = F["rho"].size
    tf = {k: torch.from_numpy(v).cuda() for k, v in F.items()}
    t = cool.Table(cool.TableSpec(n=N5))
    ti = torch.from_numpy(idx).cuda()
    res = {}
    for name, path in (("factored layout", cool.PATH_L2WINDOW), ("paper's layout (Q_total table)",
                                                                 cool.PATH_QTOTAL)):
        ue, ui, qc, cnt, ms = _gpu_step(cool, t, cool.Params(n_sub=8, path=path), tf)
        got = [a[ti].cpu().numpy().astype(np.float64) for a in (ue, ui, qc)]
        res[name] = _errs(got, o1, sub["ue"])
        report({"suite": "precision", "case": f"FP32 table, explicit, {name}", "workload": "shell_448x192x192",
                "cells": n, "ms_per_step": ms, "cell_updates_per_s": n / (ms * 1e-3), "vs_O1": res[name],
                "sample": SAMPLE})
    # both are the same method up to where the interpolation happens: their
    # errors against O1 are of the same order (the table's interpolation error)
    a, b = res["factored layout"]["u_e"], res["paper's layout (Q_total table)"]["u_e"]
    assert b["median"] <= 10 * a["median"] + 1e-5 and a["median"] <= 10 * b["median"] + 1e-5
    t.free()


def test_fp64_options_on_the_shell(env, oracle):
    cool, F, idx, sub, ospec, lazy, o1, o2 = env
    n = F["rho"].size
    tf = {k: torch.from_numpy(v).cuda() for k, v in F.items()}
    t = cool.Table(cool.TableSpec(n=N5))
    ti = torch.from_numpy(idx).cuda()
    prm_i = oracle.Params(n_sub=8, mode=1)
    o2i = oracle.step(ospec, lazy, prm_i, sub["rho"], sub["B"], sub["H"], sub["ue"], sub["ui"], lazy=True)
    for name, p, want in (("FP32 table, explicit, fp64_critical", cool.Params(n_sub=8, fp64_critical=1), o2),
                          ("FP32 table, implicit (FP32 Illinois)", cool.Params(n_sub=8, mode=cool.IMPLICIT), o2i),
                          ("FP32 table, implicit, fp64_critical",
                           cool.Params(n_sub=8, mode=cool.IMPLICIT, fp64_critical=1), o2i)):
        ue, ui, qc, cnt, ms = _gpu_step(cool, t, p, tf)
        got = [a[ti].cpu().numpy().astype(np.float64) for a in (ue, ui, qc)]
        fp64_cells = cnt["fp64_coulomb"] if p.fp64_critical else 0
        if p.fp64_critical and p.mode == cool.IMPLICIT:
            fp64_cells = cnt["fp64_coulomb"] + cnt["stiff"]   # upper bound (a cell may be both)
        line = {"suite": "precision", "case": name, "workload": "shell_448x192x192", "cells": n,
                "ms_per_step": ms, "cell_updates_per_s": n / (ms * 1e-3),
                "band_cells_frac": cnt["fp64_coulomb"] / n, "stiff_cells_frac": cnt["stiff"] / n,
                "fp64_cells_frac_upper": fp64_cells / n, "vs_O2": _errs(got, want, sub["ue"]),
                "sample": SAMPLE, "counters": cnt}
        report(line)
        assert 0.0 <= line["fp64_cells_frac_upper"] <= 2.0
        assert line["vs_O2"]["u_e"]["median"] <= 1e-5
    t.free()


def test_interpolation_error_per_process(env, oracle):
    """O2 vs O1 at the sampled cells' first-sub-cycle keys, per process
    (brems, eta Q_syn, Coulomb C): the table's own error, independent of the
    GPU.  The cell straddling the K2 switch (T_e = 1e8 K) is reported apart."""
    cool, F, idx, sub, ospec, lazy, o1, o2 = env
    prm = oracle.Params(n_sub=8)
    keys = oracle.keys_f32(prm, sub["rho"], sub["B"], sub["H"], sub["ue"], sub["ui"]).astype(np.float64)
    H, B, ne, Te, Ti = (keys[:, k] for k in range(5))
    x_t = oracle.nodes(ospec, 3)[0]
    j = np.clip(np.searchsorted(x_t, Te) - 1, 0, N5[3] - 2)
    straddle = (x_t[j] <= 1e8) & (x_t[j + 1] > 1e8)
    out = {}
    for proc in ("brems", "syn", "coulomb"):
        r = []
        for i in range(SAMPLE):
            if proc == "brems":
                a, b = oracle.interp_brems(ospec, lazy, Te[i]), np.log2(oracle.brems(Te[i]))
            elif proc == "syn":
                a = oracle.interp_syn(ospec, lazy, H[i], B[i], ne[i], Te[i], lazy=True)
                b = np.log2(oracle.eta_qsyn(H[i], B[i], ne[i], Te[i], spec=ospec))
            else:
                a = oracle.interp_coulomb(ospec, lazy, Ti[i], Te[i])
                b = np.log2(oracle.coulomb_C(Ti[i], Te[i], spec=ospec))
            r.append(abs(2.0 ** (a - b) - 1.0) if np.isfinite(a) and np.isfinite(b) else np.nan)
        r = np.array(r)
        ok = np.isfinite(r) & ~straddle
        out[proc] = {"max_rel": float(np.max(r[ok])), "median_rel": float(np.median(r[ok])),
                     "p99_rel": float(np.quantile(r[ok], 0.99))}
    out["straddling_K2_switch_cells"] = int(straddle.sum())
    report({"suite": "precision", "case": "table interpolation error per process (O2 vs O1)",
            "workload": "shell_448x192x192", "table": "128x128x64x64", "sample": SAMPLE, **out})
    assert out["brems"]["median_rel"] < 1e-2 and out["coulomb"]["median_rel"] < 1e-2
