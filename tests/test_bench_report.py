"""The bench line's reporting helpers (no GPU): the per-field error report,
the issue roofline and the ncu-derived fields keyed by the kernel sources."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_rel_err_report():
    want = np.array([1.0, 2.0, -4.0, 8.0])
    got = np.array([1.0, 2.0 * (1 + 2e-6), -4.0 * (1 - 3e-5), 8.0], np.float32)
    r = bench.rel_err_report(got, want)
    assert abs(r["max"] - 3e-5) < 1e-6             # float32 rounding of the inputs
    assert r["beyond_1e-5"] == 1
    assert r["p9999"] <= r["max"]


def test_issue_roofline_arithmetic():
    """148 SMs x 4 schedulers x 1 warp instruction per clock: a launch that
    issues exactly that many instructions in its time is at the roof."""
    r = bench.issue_roofline(1.0, 1 << 20, {"sm_mhz": 2000.0})
    if r is None:
        return   # the committed capture is of other kernel sources: nothing to report
    assert r["peak"] == 148 * 4 * 2000.0e6
    assert abs(r["frac"] - r["warp_instructions_per_launch"] / 1e-3 / r["peak"]) < 1e-12
    assert r["thread_instructions_per_cell"] > 0


def test_profile_fields_share_one_key():
    """traffic, utilisation and the issue line come from one capture: all
    present for the current kernel sources, or all absent."""
    got = [bench.traffic_per_launch() is not None, bench.ncu_utilisation() is not None,
           bench.issue_roofline(1.0, 1, None) is not None]
    assert all(got) or not any(got)


def test_kernel_source_sha_ignores_comments(tmp_path, monkeypatch):
    """The key changes with the device code, not with its comments."""
    csrc = tmp_path / "paper_2505_08855_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_text("int f() { return 1; }  // one\n/* block */\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.kernel_source_sha()
    for name in bench.KERNEL_SOURCES:
        (csrc / name).write_text("int f() { return 1; }  // another comment\n\n")
    assert bench.kernel_source_sha() == a
    (csrc / bench.KERNEL_SOURCES[0]).write_text("int f() { return 2; }\n")
    assert bench.kernel_source_sha() != a
