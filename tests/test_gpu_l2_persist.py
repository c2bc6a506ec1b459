"""cool_table_l2_persist: the opt-in persisting-L2 reservation of the packed
4-D channel.

* The step's results do not depend on it (bit for bit).
* On raises the context's persisting-L2 limit to min(packed bytes, device
  maximum); off and freeing the table put back the value it had.
* Bad arguments are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

SMALL = (12, 12, 12, 16, 16)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 3))
    tf = [torch.from_numpy(f[k].astype(np.float32)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    return cool, tf


def _limit():
    rt = pytest.importorskip("cuda.bindings.runtime")
    err, v = rt.cudaDeviceGetLimit(rt.cudaLimit.cudaLimitPersistingL2CacheSize)
    assert int(err) == 0
    return v


def _max_persist():
    rt = pytest.importorskip("cuda.bindings.runtime")
    err, v = rt.cudaDeviceGetAttribute(rt.cudaDeviceAttr.cudaDevAttrMaxPersistingL2CacheSize, 0)
    assert int(err) == 0
    return v


def test_results_do_not_depend_on_the_reservation(env):
    cool, tf = env
    tab = cool.Table(cool.TableSpec(n=SMALL))
    p = cool.Params(n_sub=8)
    off = [t.clone() for t in cool.step(tab, p, *tf)]
    tab.l2_persist(True)
    on = [t.clone() for t in cool.step(tab, p, *tf)]
    tab.l2_persist(False)
    again = cool.step(tab, p, *tf)
    torch.cuda.synchronize()
    for a, b, c in zip(off, on, again):
        assert torch.equal(a, b) and torch.equal(a, c)
    tab.free()


def test_limit_raised_and_restored(env):
    cool, tf = env
    before = _limit()
    # a table whose packed channel (31.9 MB) exceeds the context's default
    # persisting-L2 limit, so that turning the reservation on raises it
    tab = cool.Table(cool.TableSpec(n=(48, 48, 48, 64, 16)))
    assert tab.packed_bytes() > before
    assert _limit() == before              # building a table leaves the context alone
    tab.l2_persist(True)
    raised = _limit()
    assert raised > before and raised >= min(tab.packed_bytes(), _max_persist())
    tab.l2_persist(True)                   # idempotent
    assert _limit() == raised
    tab.l2_persist(False)
    assert _limit() == before
    tab.l2_persist(True)
    tab.free()                             # freeing turns it off
    assert _limit() == before


def test_bad_arguments(env):
    cool, tf = env
    from paper_2505_08855_b300 import binding as _b
    assert _b.lib().cool_table_l2_persist(None, 1) == _b.COOL_ENULL
    tab = cool.Table(cool.TableSpec(n=SMALL))
    assert _b.lib().cool_table_l2_persist(tab.handle, 2) == _b.COOL_EINVAL
    h = tab.handle
    tab.free()
    assert _b.lib().cool_table_l2_persist(h, 1) == _b.COOL_ESTATE
