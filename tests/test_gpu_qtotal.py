"""The paper's table layout (COOL_PATH_QTOTAL, Sec. 3.1) against the FP64
oracle: the device-built log2 Q_total table, and the step that reads it.

* Table: the GPU's FP64 build from its own brems and synchrotron channels
  equals the oracle's to |dlog2| <= 1e-12 max(1, |v|).
* Step: FP32 bar, max relative error <= 1e-5 per field against the
  oracle's paper's-layout step (storage in FP32 included: the oracle reads
  the table's FP32 rounding), q_cool within 1e-5 of max(u_e, u_e'),
  counters equal.
* Combinations the layout does not cover are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

SMALL = (12, 12, 12, 16, 16)


@pytest.fixture(scope="module")
def env(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    tab = cool.Table(cool.TableSpec(n=SMALL))
    ospec = oracle.Spec(n=SMALL)
    otab = oracle.build_tables(ospec, nthreads=0)
    return cool, tab, ospec, otab


def test_table_matches_oracle(env, oracle):
    cool, tab, ospec, otab = env
    got = tab.export(3)
    want = oracle.build_qtotal(ospec, otab)
    assert np.all(np.abs(got - want) <= 1e-12 * np.maximum(1.0, np.abs(want)))


@pytest.mark.parametrize("n_sub", [1, 8])
def test_step_matches_oracle(env, oracle, n_sub):
    cool, tab, ospec, otab = env
    from paper_2505_08855_b300 import binding as _b
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 5))
    f = {k: v.astype(np.float32) for k, v in f.items()}
    tf = [torch.from_numpy(f[k]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    qc = torch.empty_like(tf[0])
    cnt = cool.new_counters()
    ue, ui = cool.step(tab, cool.Params(n_sub=n_sub, path=_b.COOL_PATH_QTOTAL), *tf, q_cool=qc, counters=cnt)
    torch.cuda.synchronize()
    # the oracle on the table as stored (FP32 log2 values)
    lt32 = tab.export(3).astype(np.float32).astype(np.float64)
    otab32 = dict(otab, lc=otab["lc"].astype(np.float32).astype(np.float64))
    want = oracle.step_qtotal(ospec, otab32, lt32, oracle.Params(n_sub=n_sub),
                              *[f[k].astype(np.float64) for k in ("rho", "B", "H", "ue", "ui")])
    g = [t.cpu().numpy().astype(np.float64) for t in (ue, ui, qc)]
    e_ue = np.abs(g[0] - want[0]) / want[0]
    e_ui = np.abs(g[1] - want[1]) / want[1]
    # q_cool = u_e + X - u_e': its error is measured on the scale of u_e
    # before and after the step (the exchange can multiply u_e)
    e_qc = np.abs(g[2] - want[2]) / np.maximum(f["ue"], want[0])
    print(f"\npaper's layout, N_sub={n_sub}: max rel u_e {e_ue.max():.2e}, u_i {e_ui.max():.2e}, "
          f"q_cool/u_e {e_qc.max():.2e}")
    assert e_ue.max() <= 1e-5 and e_ui.max() <= 1e-5 and e_qc.max() <= 1e-5
    c = cool.counters_dict(cnt)
    assert c["nonfinite"] == want[4]["invalid"]
    assert c["clamped"] == want[4]["clamped"]


def test_refused_combinations(env):
    cool, tab, ospec, otab = env
    from paper_2505_08855_b300 import binding as _b
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(256))
    tf = [torch.from_numpy(f[k].astype(np.float32)).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    P = _b.COOL_PATH_QTOTAL
    for p in (cool.Params(path=P, mode=cool.IMPLICIT), cool.Params(path=P, fp64_critical=1)):
        with pytest.raises(cool.CoolError) as e:
            cool.step(tab, p, *tf)
        assert e.value.status == _b.COOL_EUNSUPPORTED
    with pytest.raises(cool.CoolError) as e:
        cool.step(tab, cool.Params(path=P), *[t.double() for t in tf])
    assert e.value.status == _b.COOL_EUNSUPPORTED
    half = cool.Table(cool.TableSpec(n=SMALL, dtype=cool.BF16))
    with pytest.raises(cool.CoolError) as e:
        cool.step(half, cool.Params(path=P), *tf)
    assert e.value.status == _b.COOL_EUNSUPPORTED
    g = torch.ones_like(tf[0])
    with pytest.raises(cool.CoolError) as e:
        cool.step_bwd(tab, cool.Params(path=P), *tf, g, g)
    assert e.value.status == _b.COOL_EUNSUPPORTED


def test_layouts_against_direct_formulas_two_region(oracle):
    """Both layouts from the benchmark's 64^4 FP32 table on 1024 sampled
    256^3 two-region cells against the direct formulas (O1): the paper's
    layout interpolates the bridged rate, the factored one bridges
    interpolated rates; their errors against O1 are reported (REPORT) and
    are of the same order."""
    import json
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import binding as _b
    n5 = (64,) * 5
    tab = cool.Table(cool.TableSpec(n=n5))
    F = inputs.make("two_region_256c")
    tf = [torch.from_numpy(F[k]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    idx = np.sort(np.random.default_rng(9).choice(F["rho"].size, 1024, replace=False))
    sub = {k: v[idx].astype(np.float64) for k, v in F.items()}
    ospec = oracle.Spec(n=n5)
    lazy = oracle.build_tables(ospec, syn=False)
    o1 = oracle.step(ospec, lazy, oracle.Params(n_sub=8), sub["rho"], sub["B"], sub["H"], sub["ue"], sub["ui"],
                     direct=True)
    ti = torch.from_numpy(idx).cuda()
    med = {}
    for name, path in (("factored", _b.COOL_PATH_L2WINDOW), ("paper's layout", _b.COOL_PATH_QTOTAL)):
        ue, ui = cool.step(tab, cool.Params(n_sub=8, path=path), *tf)
        g = ue[ti].cpu().numpy().astype(np.float64)
        r = np.abs(g - o1[0]) / o1[0]
        med[name] = float(np.median(r))
        print("REPORT " + json.dumps({"suite": "precision", "case": f"two_region_256c, {name}",
                                      "vs_O1_u_e": {"median": med[name], "p99": float(np.quantile(r, 0.99)),
                                                    "max": float(r.max())}, "sample": 1024}))
    assert med["paper's layout"] <= 10 * med["factored"] + 1e-5 and med["factored"] <= 10 * med["paper's layout"] + 1e-5
    tab.free()
