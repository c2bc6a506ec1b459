"""The C-ABI library without a GPU: it builds for sm_103a, loads, exports
every entry point include/cool.h declares, its structs have the header's
layout, and host-side argument validation answers without touching a GPU."""
import ctypes as C
import os
import re
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cool.h")


@pytest.fixture(scope="module")
def L():
    from paper_2505_08855_b300 import build, binding
    build.build()
    return binding.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cool_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    from paper_2505_08855_b300 import binding
    decl = declared_functions()
    assert len(decl) >= 13
    assert sorted(binding.EXPORTS) == decl
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2505_08855_b300", "libcool.so")],
                         capture_output=True, text=True, check=True).stdout
    syms = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in decl:
        assert name in syms, name


def test_build_targets_sm_103a_only():
    from paper_2505_08855_b300 import build
    flags = " ".join(build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags
    assert flags.count("-gencode") == 1


def test_struct_layout_matches_header(tmp_path):
    from paper_2505_08855_b300 import binding as b
    prog = tmp_path / "layout.c"
    fields = {
        "cool_table_spec": [f[0] for f in b.cool_table_spec._fields_],
        "cool_params": [f[0] for f in b.cool_params._fields_],
        "cool_counters": [f[0] for f in b.cool_counters._fields_],
        "cool_fit_spec": [f[0] for f in b.cool_fit_spec._fields_],
        "cool_surrogate_stats": [f[0] for f in b.cool_surrogate_stats._fields_],
        "cool_disk": [f[0] for f in b.cool_disk._fields_],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for st, fl in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fl:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(prog)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for st, fl in fields.items():
        cls = getattr(b, st)
        assert int(got[st]) == C.sizeof(cls), st
        for f in fl:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_host_validation_without_gpu(L):
    from paper_2505_08855_b300 import binding as b
    assert L.cool_strerror(b.COOL_EINVAL) == b"invalid argument"
    s = b.cool_table_spec()
    assert L.cool_table_spec_default(b.ref(s)) == b.COOL_OK
    assert (s.n_H, s.H_min, s.H_max, s.T_min, s.T_max) == (64, 1e3, 1e12, 1e2, 1e15)
    p = b.cool_params()
    assert L.cool_params_default(b.ref(p)) == b.COOL_OK
    assert p.limiter_frac == 0.3 and p.n_sub == 8
    h = C.c_void_p()
    # invalid specs are rejected before any CUDA call
    bad = b.cool_table_spec()
    L.cool_table_spec_default(b.ref(bad))
    bad.n_H = 1
    assert L.cool_build_table(b.ref(bad), None, b.ref(h)) == b.COOL_EINVAL
    bad.n_H = 64
    bad.T_max = bad.T_min
    assert L.cool_build_table(b.ref(bad), None, b.ref(h)) == b.COOL_EINVAL
    bad.T_max = 1e15
    bad.row_scaled = 1          # block scaling applies to 16-bit storage only
    assert L.cool_build_table(b.ref(bad), None, b.ref(h)) == b.COOL_EUNSUPPORTED
    bad.row_scaled = 0
    bad.dtype = b.COOL_F64      # FP64 storage of the 4-D channel is not a step format
    assert L.cool_build_table(b.ref(bad), None, b.ref(h)) == b.COOL_EUNSUPPORTED
    assert L.cool_build_table(None, None, b.ref(h)) == b.COOL_ENULL
    # a handle that was never created is rejected without being read
    fake = C.c_void_p(0x1234)
    assert L.cool_table_free(fake) == b.COOL_ESTATE
    assert L.cool_step(fake, b.ref(p), 0, 0, *([None] * 9), None, None) == b.COOL_ESTATE
    assert L.cool_step(None, b.ref(p), 0, 0, *([None] * 9), None, None) == b.COOL_ENULL
    assert L.cool_table_free(None) == b.COOL_OK


def test_product_path_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2505_08855_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "cool_oracle" not in src and "liboracle" not in src, f


def test_noalloc_wrapper_rejects_wrong_outputs_before_any_launch():
    """build_channels_noalloc writes through raw pointers: a float32 tensor or
    a short float64 tensor must be refused by the binding before the library
    is called (CPU tensors suffice: dtype and size are checked first)."""
    import torch
    import paper_2505_08855_b300 as cool
    spec = cool.TableSpec(n=(4, 5, 6, 7, 8))
    good = [torch.zeros(m, dtype=torch.float64) for m in (7, 4 * 5 * 6 * 7, 64)]
    bad32 = [good[0], good[1].float(), good[2]]
    with pytest.raises(ValueError, match="float64"):
        cool.build_channels_noalloc(spec, *bad32)
    short = [good[0], good[1], torch.zeros(63, dtype=torch.float64)]
    with pytest.raises(ValueError, match="exactly 64"):
        cool.build_channels_noalloc(spec, *short)
    with pytest.raises(ValueError, match="CUDA device"):
        cool.build_channels_noalloc(spec, *good)     # right sizes, but host tensors


def test_jacobian_wrappers_reject_wrong_tensors_before_any_launch():
    """step_fwd_jac and step_bwd_jac write through raw pointers: wrong dtypes,
    sizes (the Jacobian is 10 n floats) or host tensors are refused by the
    binding before the library is called."""
    import torch
    import paper_2505_08855_b300 as cool
    n = 16
    f = [torch.ones(n) for _ in range(5)]
    with pytest.raises(ValueError, match="step_fwd_jac"):
        cool.step_fwd_jac(None, cool.Params(), *f)                       # host tensors
    with pytest.raises(ValueError, match="step_fwd_jac"):
        cool.step_fwd_jac(None, cool.Params(), *[x.double() for x in f])  # float64
    g = torch.ones(n)
    with pytest.raises(ValueError, match="step_bwd_jac"):
        cool.step_bwd_jac(torch.ones(9 * n), g, g)                       # short Jacobian
    with pytest.raises(ValueError, match="step_bwd_jac"):
        cool.step_bwd_jac(torch.ones(10 * n), g, g)                      # host tensors
