"""COOL_PATH_TMA_SMEM (the step with its field staging by bulk asynchronous
copies, double-buffered per warp) gives exactly the results of the default
path: the same per-cell arithmetic on the same cells, for every table
format, mode and FP64 option, on a cell count with a ragged tail.  (With
fp64_critical the default path steps the band and stiff cells in a second,
compacted pass and the TMA path per lane: the same bits.)"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

N5 = (12, 12, 12, 40, 24)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    f = inputs.make("uniform_128c")
    n = 300_037
    t = {k: torch.from_numpy(np.ascontiguousarray(v[:n])).cuda() for k, v in f.items()}
    return cool, t


@pytest.mark.parametrize("dtype,scaled", [(0, 0), (1, 0), (2, 1)])
@pytest.mark.parametrize("mode,fp64", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_tma_path_equals_default(env, dtype, scaled, mode, fp64):
    from paper_2505_08855_b300 import binding as _b
    cool, t = env
    tab = cool.Table(cool.TableSpec(n=N5, dtype=dtype, row_scaled=scaled))
    fl = [t[k] for k in ("rho", "B", "H", "ue", "ui")]
    outs = {}
    for path in (_b.COOL_PATH_L2WINDOW, _b.COOL_PATH_TMA_SMEM):
        p = cool.Params(n_sub=8, mode=mode, fp64_critical=fp64, path=path)
        qc = torch.empty_like(fl[0])
        qx = torch.empty_like(fl[0])
        c = cool.new_counters()
        ue, ui = cool.step(tab, p, *fl, q_cool=qc, q_cc=qx, counters=c)
        torch.cuda.synchronize()
        outs[path] = (ue, ui, qc, qx, c)
    a, b = outs[_b.COOL_PATH_L2WINDOW], outs[_b.COOL_PATH_TMA_SMEM]
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert cool.tma_error() == 0      # every bulk copy completed within its bounded wait


def test_tma_path_needs_aligned_fields(env):
    from paper_2505_08855_b300 import binding as _b
    cool, t = env
    tab = cool.Table(cool.TableSpec(n=N5))
    fl = [t[k][1:1001] for k in ("rho", "B", "H", "ue", "ui")]
    with pytest.raises(cool.CoolError) as e:
        cool.step(tab, cool.Params(path=_b.COOL_PATH_TMA_SMEM), *fl)
    assert e.value.status == _b.COOL_EALIGN
