"""The failure path of the kernels' bounded waits, made to happen without a
fault: a wait on a barrier that nothing completes runs out after its poll
limit, reports through its error word, and leaves the context usable (a
step and a tensor-core product run correctly afterwards)."""
import ctypes as C
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def cool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as c
    from paper_2505_08855_b300 import build
    build.build()
    return c


def test_wait_runs_out_and_reports(cool):
    t0 = time.perf_counter()
    assert cool.debug_wait_timeout(1000) == 1
    assert time.perf_counter() - t0 < 10.0


def test_bad_arguments(cool):
    from paper_2505_08855_b300 import binding as _b
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _b.lib().cool_debug_wait_timeout(1000, None, None) == _b.COOL_ENULL
    assert _b.lib().cool_debug_wait_timeout(0, err.data_ptr(), None) == _b.COOL_EINVAL
    assert _b.lib().cool_debug_wait_timeout((1 << 20) + 1, err.data_ptr(), None) == _b.COOL_EINVAL


def test_context_usable_after_the_timeout(cool, oracle):
    assert cool.debug_wait_timeout(100) == 1
    n = (12, 12, 12, 16, 16)
    tab = cool.Table(cool.TableSpec(n=n))
    ospec = oracle.Spec(n=n)
    otab = oracle.build_tables(ospec, nthreads=0)
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 16))
    tf = [torch.from_numpy(f[k].astype(np.float32)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    ue, ui = cool.step(tab, cool.Params(n_sub=4), *tf)
    torch.cuda.synchronize()
    want = oracle.step(ospec, otab, oracle.Params(n_sub=4),
                       *[f[k].astype(np.float32).astype(np.float64) for k in ("rho", "B", "H", "ue", "ui")])
    rel = np.abs(ue.cpu().numpy() - want[0]) / want[0]
    assert rel.max() <= 1e-5
    # a tensor-core product, which waits on its own completion signal
    from paper_2505_08855_b300 import binding as _b
    g = torch.Generator().manual_seed(5)
    a = torch.randn(128, 32, generator=g).to(torch.bfloat16).cuda()
    b = torch.randn(16, 32, generator=g).to(torch.bfloat16).cuda()
    c = torch.full((128, 16), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = _b.lib().cool_debug_gemm_bf16(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(c.data_ptr()),
                                       128, 16, 32, C.c_void_p(err.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    want_c = a.double().cpu() @ b.double().cpu().t()
    assert torch.allclose(c.double().cpu(), want_c, rtol=1e-5, atol=1e-4)
