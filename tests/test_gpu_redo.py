"""The fast index selection's extra work, per mode (GPU).

The step selects each interval from the lg2 guess and redoes a cell with
node compares (the exact rule) only when a key falls within ~1e-6 of a node
or the guess is in doubt: a few selections in a million.  The outputs are
the same either way, so only the redo counter shows a path that sends many
cells to the redo -- as the implicit solve's trial keys did while an
out-of-range key still counted as in doubt (every stiff cell redone).
Here the redo fraction of every mode stays far below the stiff and band
fractions, on 128^3 uniform cells with the 64^4 table.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    F = inputs.make("uniform_128c")
    tf = [torch.from_numpy(F[k]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    return cool, cool.Table(cool.TableSpec(n=(64,) * 5)), tf


@pytest.mark.parametrize("mode,fp64", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_exact_redo_is_rare(env, mode, fp64):
    cool, tab, tf = env
    n = tf[0].numel()
    cnt = cool.new_counters()
    cool.step(tab, cool.Params(n_sub=8, mode=mode, fp64_critical=fp64), *tf, counters=cnt)
    c = cool.counters_dict(cnt)
    print(f"\nmode {mode} fp64_critical {fp64}: exact redo {c['exact_redo']} of {n} cells "
          f"({c['exact_redo'] / n:.1e}); stiff {c['stiff']}, band {c['fp64_coulomb']}")
    assert c["exact_redo"] <= 1e-3 * n
    if mode == 1:
        assert c["stiff"] > 20 * c["exact_redo"]


def test_redo_counted_on_the_scalar_path(env):
    """Unaligned fields take the per-lane path: the same cells are redone."""
    cool, tab, tf = env
    m = 1 << 20
    counts = []
    for off in (0, 1):
        cnt = cool.new_counters()
        cool.step(tab, cool.Params(n_sub=8, mode=1), *[t[off:off + m] for t in tf], counters=cnt)
        counts.append(cool.counters_dict(cnt))
    a, b = counts
    print(f"\naligned: redo {a['exact_redo']}, stiff {a['stiff']}; shifted by one cell: redo {b['exact_redo']}, "
          f"stiff {b['stiff']}")
    assert b["exact_redo"] <= 1e-3 * m and b["stiff"] > 20 * b["exact_redo"]
