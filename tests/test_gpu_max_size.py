"""The step past 2^31 cells: 64-bit cell, tile and counter arithmetic.

The 32^3 uniform cells repeated on the device to 2^31 + 32765 cells (a
ragged tail for the scalar loop; 60 GB of fields and outputs).  Cells are
independent and the vector and scalar paths do the same per-cell
arithmetic, so every cell's result equals, bit for bit, the result of the
cell it repeats in a step over the 32^3 cells alone.  Checked on samples
spread over the whole range, around 2^31 and in the tail.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

SMALL = (12, 12, 12, 16, 16)


def test_step_beyond_2_31_cells():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    free, _ = torch.cuda.mem_get_info()
    base = inputs.make("uniform_32c")
    nb = base["rho"].size
    n = (1 << 31) + nb - 3
    if free < 8 * 4 * n + (4 << 30):
        pytest.skip("not enough device memory for 2^31 cells")
    tab = cool.Table(cool.TableSpec(n=SMALL))
    p = cool.Params(n_sub=4)
    small = [torch.from_numpy(base[k].astype(np.float32)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    want_e, want_i = [t.cpu().numpy() for t in cool.step(tab, p, *small)]
    reps = n // nb + 1
    big = [t.repeat(reps)[:n].contiguous() for t in small]
    ue, ui = cool.step(tab, p, *big)
    torch.cuda.synchronize()
    del big
    rng = np.random.default_rng(11)
    idx = np.concatenate([rng.integers(0, n, 20000), np.arange((1 << 31) - 300, (1 << 31) + 300),
                          np.arange(n - 500, n)])
    it = torch.from_numpy(idx).cuda()
    ge, gi = ue[it].cpu().numpy(), ui[it].cpu().numpy()
    assert np.array_equal(ge, want_e[idx % nb])
    assert np.array_equal(gi, want_i[idx % nb])
