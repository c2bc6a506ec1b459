"""cool_step_host (the step on host arrays, streamed through the device in
overlapping chunks) gives exactly the results of cool_step on device copies
of the same fields: every chunk runs the same kernel on the same cells."""
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
    tab = cool.Table(cool.TableSpec(n=(12, 12, 12, 16, 16)))
    f = inputs.make("uniform_128c")
    n = 300_001                                   # ragged against every chunk size below
    return cool, tab, {k: np.ascontiguousarray(v[:n]) for k, v in f.items()}


@pytest.mark.parametrize("pinned,chunk,mode,fp64", [(True, 0, 0, 0), (True, 65536, 0, 0), (False, 100_000, 0, 0),
                                                  (True, 65536, 1, 0), (True, 100_000, 1, 1)])
def test_host_step_equals_device_step(env, pinned, chunk, mode, fp64):
    """Implicit mode and fp64_critical: each chunk lists and steps its own
    flagged cells; the results and the counters are those of one step."""
    cool, tab, f = env
    n = f["rho"].size
    p = cool.Params(n_sub=8, mode=mode, fp64_critical=fp64)
    host = {k: torch.from_numpy(v) for k, v in f.items()}
    if pinned:
        host = {k: v.pin_memory() for k, v in host.items()}
    ue_h = torch.empty(n, dtype=torch.float32)
    ui_h = torch.empty(n, dtype=torch.float32)
    if pinned:
        ue_h, ui_h = ue_h.pin_memory(), ui_h.pin_memory()
    cnt = cool.new_counters()
    cool.step_host(tab, p, host["rho"], host["B"], host["H"], host["ue"], host["ui"], ue_h, ui_h,
                   chunk_cells=chunk, counters=cnt)
    torch.cuda.synchronize()
    dev = {k: v.cuda() for k, v in host.items()}
    c2 = cool.new_counters()
    ue_d, ui_d = cool.step(tab, p, dev["rho"], dev["B"], dev["H"], dev["ue"], dev["ui"], counters=c2)
    torch.cuda.synchronize()
    assert torch.equal(ue_h, ue_d.cpu()) and torch.equal(ui_h, ui_d.cpu())
    assert torch.equal(cnt.cpu(), c2.cpu())


def test_host_step_rejects_device_arrays(env):
    cool, tab, f = env
    t = [torch.from_numpy(f[k][:1000]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    with pytest.raises(ValueError):
        cool.step_host(tab, cool.Params(), *t, t[3].clone(), t[4].clone())
