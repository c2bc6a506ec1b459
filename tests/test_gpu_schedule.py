"""The step's dynamic tile order: each cell's result does not depend on
which warp steps it or when, so every schedule gives the same bits.

* Steps on two streams at once (each stream has its own tile counter)
  equal the same steps run one after the other.
* A step captured in a CUDA graph on a stream with no counter yet (the
  static order: no tile counter is allocated inside a capture) and
  replayed equals the plain step, in every mode (implicit mode and
  fp64_critical allocate their list of flagged cells stream-ordered, which
  a graph holds as allocation nodes); so does the captured adjoint.
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


@pytest.mark.parametrize("mode,fp64", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_graph_capture_equals_plain_step(env, mode, fp64):
    """Implicit mode and fp64_critical also list their flagged cells in
    stream-ordered scratch: allocated and freed inside the graph."""
    cool, tab, tf = env
    p = cool.Params(n_sub=8, mode=mode, fp64_critical=fp64)
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


@pytest.mark.parametrize("mode", [0, 1])
def test_graph_capture_of_the_adjoint(env, mode):
    """The input gradients captured and replayed equal the plain call
    (implicit mode: the stiff cells' list in stream-ordered scratch)."""
    cool, tab, tf = env
    p = cool.Params(n_sub=8, mode=mode)
    n = tf[0].numel()
    a = torch.ones(n, device="cuda")
    b = torch.full((n,), -0.5, device="cuda")
    want = [t.clone() for t in cool.step_bwd(tab, p, *tf, a, b)]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        got = cool.step_bwd(tab, p, *tf, a, b)
    for t in got:
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip(got, want):
        assert torch.equal(x, y)


@pytest.mark.parametrize("mode", [0, 1])
def test_graph_capture_of_the_jacobian_pair(env, mode):
    """cool_step_fwd_jac + cool_step_bwd_jac captured in one graph and
    replayed equal the plain calls (implicit mode: the stiff cells' list in
    stream-ordered scratch inside the graph)."""
    cool, tab, tf = env
    p = cool.Params(n_sub=8, mode=mode)
    n = tf[0].numel()
    a = torch.ones(n, device="cuda")
    b = torch.full((n,), -0.5, device="cuda")
    ue, ui, jac = cool.step_fwd_jac(tab, p, *tf)
    want = [t.clone() for t in (ue, ui, *cool.step_bwd_jac(jac, a, b))]
    torch.cuda.synchronize()
    uo, vo, J = torch.empty_like(ue), torch.empty_like(ui), torch.empty_like(jac)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cool.step_fwd_jac(tab, p, *tf, ue_out=uo, ui_out=vo, jac=J)
        grads = cool.step_bwd_jac(J, a, b)
    for t in (uo, vo, J, *grads):
        t.zero_()
    g.replay()
    torch.cuda.synchronize()
    for x, y in zip((uo, vo, *grads), want):
        assert torch.equal(x, y)


def test_graph_replayed_on_another_stream_while_a_step_runs(env, oracle):
    """A step captured on stream s1 after s1 already owns a tile counter, and
    replayed on stream s2 while s1 runs a plain step: a capture never uses a
    counter (static order), so the two launches share nothing and both give
    the plain step's bits; a sample of cells also matches the FP64 oracle."""
    cool, tab, tf = env
    p = cool.Params(n_sub=8)
    other = [t.flip(0).contiguous() for t in tf]
    want_a = [t.clone() for t in cool.step(tab, p, *tf)]
    want_b = [t.clone() for t in cool.step(tab, p, *other)]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        cool.step(tab, p, *tf, stream=s1)          # s1 now owns a tile counter
    torch.cuda.synchronize()
    ue_g, ui_g = torch.empty_like(other[3]), torch.empty_like(other[4])
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s1):
        cool.step(tab, p, *other, ue_out=ue_g, ui_out=ui_g, stream=s1)
    torch.cuda.synchronize()
    for _ in range(3):
        ue_g.zero_()
        ui_g.zero_()
        torch.cuda.synchronize()
        with torch.cuda.stream(s1):
            a = cool.step(tab, p, *tf, stream=s1)
        with torch.cuda.stream(s2):
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(a[0], want_a[0]) and torch.equal(a[1], want_a[1])
        assert torch.equal(ue_g, want_b[0]) and torch.equal(ui_g, want_b[1])
    idx = np.random.default_rng(11).choice(tf[0].numel(), 2000, replace=False)
    ospec = oracle.Spec(n=SMALL)
    f = {k: other[i].cpu().numpy()[idx] for i, k in enumerate(("rho", "B", "H", "ue", "ui"))}
    ref = oracle.step(ospec, oracle.build_tables(ospec), oracle.Params(n_sub=8), **f)
    for got, r in ((ue_g, ref[0]), (ui_g, ref[1])):
        err = np.abs(got.cpu().double().numpy()[idx] - r) / np.abs(r)
        assert err.max() <= 1e-5


def test_list_scratch_grows_and_is_released(env):
    """Implicit steps keep their list of stiff cells in scratch kept per
    stream: a small call, a larger one (the scratch grows), the small one
    again, then after cool_release_scratch (allocated again): every result
    equals the first of its size, and the stiff counts agree."""
    cool, tab, tf = env
    p = cool.Params(n_sub=8, mode=1)
    small = [t[:5000] for t in tf]
    first_small = [x.clone() for x in cool.step(tab, p, *small)]
    first_big = [x.clone() for x in cool.step(tab, p, *tf)]
    again_small = cool.step(tab, p, *small)
    torch.cuda.synchronize()
    cool.release_scratch()
    c = cool.new_counters()
    after = cool.step(tab, p, *tf, counters=c)
    torch.cuda.synchronize()
    for x, y in zip(again_small, first_small):
        assert torch.equal(x, y)
    for x, y in zip(after, first_big):
        assert torch.equal(x, y)
    assert cool.counters_dict(c)["stiff"] > 0
