"""The step's dynamic tile order: each cell's result does not depend on
which warp steps it or when, so every schedule gives the same bits.

* Steps on two streams at once (each stream has its own tile counter)
  equal the same steps run one after the other.
* A step captured in a CUDA graph on a stream with no counter yet (the
  static order: nothing is allocated inside a capture) and replayed equals
  the plain step.
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
    tab = cool.Table(cool.TableSpec(n=SMALL))
    # enough cells for more tiles than resident warps (dynamic order in use)
    f = inputs.make("uniform_128c")
    tf = [torch.from_numpy(f[k].astype(np.float32)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    return cool, tab, tf


def test_concurrent_streams_equal_serial(env):
    cool, tab, tf = env
    p = cool.Params(n_sub=8)
    other = [t.flip(0).contiguous() for t in tf]
    want_a = [t.clone() for t in cool.step(tab, p, *tf)]
    want_b = [t.clone() for t in cool.step(tab, p, *other)]
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for _ in range(3):
        with torch.cuda.stream(s1):
            a = cool.step(tab, p, *tf, stream=s1)
        with torch.cuda.stream(s2):
            b = cool.step(tab, p, *other, stream=s2)
        outs.append((a, b))
    torch.cuda.synchronize()
    for a, b in outs:
        for x, y in zip(a, want_a):
            assert torch.equal(x, y)
        for x, y in zip(b, want_b):
            assert torch.equal(x, y)


def test_graph_capture_equals_plain_step(env):
    cool, tab, tf = env
    p = cool.Params(n_sub=8)
    want = [t.clone() for t in cool.step(tab, p, *tf)]
    ue_o, ui_o = torch.empty_like(tf[3]), torch.empty_like(tf[4])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cool.step(tab, p, *tf, ue_out=ue_o, ui_out=ui_o)
    ue_o.zero_()
    ui_o.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ue_o, want[0]) and torch.equal(ui_o, want[1])
