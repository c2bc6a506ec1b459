"""The direct-formula step (cool_step_direct: every rate from the formulas
on the GPU in FP64, no table) against the oracle's direct step (O1), and
against the table step: the paper's analytic-versus-table comparison.

The two FP64 implementations evaluate the same formulas with different
algorithms (Bessel functions, root bracketing); the step's fields agree to
1e-11 relative (measured: 3e-15).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def env(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 61))
    f["rho"][3] = np.nan
    return cool, f


def _run(cool, p, f):
    tf = [torch.from_numpy(np.ascontiguousarray(f[k], np.float64)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    qc = torch.empty_like(tf[0])
    qx = torch.empty_like(tf[0])
    cnt = cool.new_counters()
    ue, ui = cool.step_direct(cool.TableSpec(), p, *tf, q_cool=qc, q_cc=qx, counters=cnt)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (ue, ui, qc, qx)], cool.counters_dict(cnt)


@pytest.mark.parametrize("mode,ncell", [(0, 538), (1, 160)])
def test_direct_step_matches_oracle_o1(env, oracle, mode, ncell):
    cool, f = env
    g = {k: v[:ncell] for k, v in f.items()}
    got, cnt = _run(cool, cool.Params(n_sub=4, mode=mode), g)
    spec = oracle.Spec(n=(4, 4, 4, 4, 4))
    tabs = oracle.build_tables(spec, syn=False)
    want = oracle.step(spec, tabs, oracle.Params(n_sub=4, mode=mode), *[g[k] for k in ("rho", "B", "H", "ue", "ui")],
                       direct=True)
    ok = np.isfinite(want[0])
    for k, name in ((0, "u_e"), (1, "u_i")):
        r = np.abs(got[k][ok] - want[k][ok]) / np.abs(want[k][ok])
        print(f"\nmode {mode}: {name} max rel {r.max():.2e}")
        assert r.max() <= 1e-11, name
    r = np.abs(got[2][ok] - want[2][ok]) / g["ue"][ok]
    assert r.max() <= 1e-11
    assert cnt["nonfinite"] == 1 and got[0][3] == g["ue"][3] and got[2][3] == 0.0
    if mode == 1:
        assert cnt["stiff"] == want[4]["stiff"]


def test_direct_refuses_other_options(env):
    from paper_2505_08855_b300 import binding as _b
    cool, f = env
    tf = [torch.from_numpy(np.ascontiguousarray(f[k][:64], np.float64)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    for p in (cool.Params(fp64_critical=1), cool.Params(path=_b.COOL_PATH_TEXTURE_POINT)):
        with pytest.raises(cool.CoolError) as e:
            cool.step_direct(cool.TableSpec(), p, *tf)
        assert e.value.status == _b.COOL_EUNSUPPORTED
    with pytest.raises(cool.CoolError) as e:
        cool.step_direct(cool.TableSpec(lnLambda=-1.0), cool.Params(), *tf)
    assert e.value.status == _b.COOL_EINVAL
