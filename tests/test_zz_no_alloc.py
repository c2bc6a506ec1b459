"""The caller-allocated table build (cool_build_channels_noalloc).

Callers that reserve all device memory themselves cannot let the library
call cudaMalloc; this entry point writes the table's FP64 channels into
buffers the caller owns, with the builder's scratch in a fixed device array
inside the library.  Its channels must equal those of the allocating build
(cool_build_table, read back through cool_table_export) within the table
tolerance of the other GPU tests, on two calls in a row (the shared scratch
keeps the previous call's contents, so the second call checks that nothing
stale leaks through), and equal the FP64 oracle's tables of the same spec
within the same tolerance.  Collected last so that a failure here does not
hide the other tests.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12   # |dlog2| / max(1, |v|): the table tolerance of the GPU parity tests


def test_noalloc_build_matches_allocating_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import binding as b, build
    build.build()
    L = b.lib()
    import oracle as O
    for n in [(12, 10, 9, 17, 16), (16, 16, 16, 32, 24)]:
        spec = cool.TableSpec(n=n)
        ref = cool.Table(spec)
        want = [ref.export(ch) for ch in range(3)]
        ot = O.build_tables(O.Spec(n=n))
        orc = [ot["lb"], ot["ls"], np.asarray(ot["lc"]).reshape(-1)]
        sizes = [n[3], n[0] * n[1] * n[2] * n[3], n[4] * n[4]]
        for call in range(2):
            outs = [torch.full((m,), float("nan"), dtype=torch.float64, device="cuda") for m in sizes]
            cs = spec.c()
            st = L.cool_build_channels_noalloc(b.ref(cs), C.c_void_p(outs[0].data_ptr()),
                                               C.c_void_p(outs[1].data_ptr()), C.c_void_p(outs[2].data_ptr()),
                                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == b.COOL_OK, L.cool_strerror(st)
            torch.cuda.synchronize()
            for got, w, o in zip(outs, want, orc):
                g = got.cpu().numpy()
                assert np.all(np.abs(g - w) <= TOL * np.maximum(1.0, np.abs(w))), (n, call)
                assert np.all(np.abs(g - o) <= TOL * np.maximum(1.0, np.abs(o))), (n, call, "oracle")


def test_noalloc_rejects_axes_beyond_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import binding as b
    L = b.lib()
    spec = cool.TableSpec(n=(8, 8, 8, 257, 8))
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    cs = spec.c()
    st = L.cool_build_channels_noalloc(b.ref(cs), C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()),
                                       C.c_void_p(buf.data_ptr()), None)
    assert st == b.COOL_EINVAL
