"""The texture comparison paths (the paper's own design, Sec. 3.1) against
the FP64 oracle.

* COOL_PATH_TEXTURE_POINT: 16 point fetches and FP32 multilinear
  interpolation -- the same numbers as the table step, so the FP32 parity
  bar (1e-5 relative per field) applies.
* COOL_PATH_TEXTURE_HWLERP: the texture unit's trilinear filtering forms its
  weights in fixed point with 8 fractional bits, so each of the three
  filtered weights is off by up to 2^-8 and the interpolated log2 value by up
  to 2^-8 of the channel's node-to-node step per filtered axis.  The test
  bounds the error of the synchrotron value that way (through the step's
  cooled energy in one-sub-cycle cells where synchrotron dominates) and
  reports the step's error per field.
* Combinations the texture paths do not cover are refused.
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
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 8)[:4099])
    f = {k: v.astype(np.float32) for k, v in f.items()}
    return cool, tab, ospec, oracle.build_tables(ospec, nthreads=0), f


def _run(cool, tab, p, f):
    tf = [torch.from_numpy(f[k]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    qc = torch.empty_like(tf[0])
    qx = torch.empty_like(tf[0])
    cnt = cool.new_counters()
    ue, ui = cool.step(tab, p, *tf, q_cool=qc, q_cc=qx, counters=cnt)
    torch.cuda.synchronize()
    return [t.cpu().numpy().astype(np.float64) for t in (ue, ui, qc, qx)], cool.counters_dict(cnt)


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


@pytest.mark.parametrize("n_sub", [1, 8])
def test_point_path_matches_oracle(env, oracle, n_sub):
    from paper_2505_08855_b300 import binding as _b
    cool, tab, ospec, OT, f = env
    p = cool.Params(n_sub=n_sub, path=_b.COOL_PATH_TEXTURE_POINT)
    got, cnt = _run(cool, tab, p, f)
    want = oracle.step(ospec, OT, oracle.Params(n_sub=n_sub), *[f[k].astype(np.float64) for k in
                                                               ("rho", "B", "H", "ue", "ui")])
    e_ue, e_ui = _rel(got[0], want[0]).max(), _rel(got[1], want[1]).max()
    print(f"\ntexture point, N_sub={n_sub}: max rel u_e {e_ue:.2e}, u_i {e_ui:.2e}")
    assert e_ue <= 1e-5 and e_ui <= 1e-5
    assert cnt["nonfinite"] == want[4]["invalid"]


def test_hw_lerp_error_within_fixed_point_bound(env, oracle):
    from paper_2505_08855_b300 import binding as _b
    cool, tab, ospec, OT, f = env
    fields = [f[k].astype(np.float64) for k in ("rho", "B", "H", "ue", "ui")]
    for n_sub in (1, 8):
        got, _ = _run(cool, tab, cool.Params(n_sub=n_sub, path=_b.COOL_PATH_TEXTURE_HWLERP), f)
        want = oracle.step(ospec, OT, oracle.Params(n_sub=n_sub), *fields)
        r = _rel(got[0], want[0])
        print(f"\ntexture hw lerp, N_sub={n_sub}: rel err u_e median {np.median(r):.2e}, "
              f"99% {np.quantile(r, 0.99):.2e}, max {r.max():.2e}; u_i max {_rel(got[1], want[1]).max():.2e}")
    # the bound, in cells whose one-sub-cycle cooling is unlimited and
    # synchrotron-dominated in the optically thin regime: there q_cool is
    # proportional to 2^(l_syn), so log2 of the ratio of the cooled energies
    # is the error of the interpolated log2 value
    ls = OT["ls"].reshape(SMALL[:4])
    step = max(np.abs(np.diff(ls, axis=a)).max() for a in (1, 2, 3))   # B, n_e, T_e: filtered axes
    bound = 3 * step * 2.0 ** -8 + 1e-4
    got, _ = _run(cool, tab, cool.Params(n_sub=1, path=_b.COOL_PATH_TEXTURE_HWLERP), f)
    pt, _ = _run(cool, tab, cool.Params(n_sub=1, path=_b.COOL_PATH_TEXTURE_POINT), f)
    qa, qb = got[2], pt[2]
    ok = (qb > 0) & (qb < 0.25 * f["ue"]) & (qa > 0)
    dl = np.abs(np.log2(qa[ok] / qb[ok]))
    print(f"log2 error of the cooled energy (unlimited cells): max {dl.max():.3e}, bound {bound:.3e} "
          f"(max node step {step:.1f})")
    assert ok.sum() > 100
    assert dl.max() <= bound


def test_texture_paths_refuse_what_they_do_not_cover(env):
    from paper_2505_08855_b300 import binding as _b
    cool, tab, ospec, OT, f = env
    tf = [torch.from_numpy(f[k][:256]).cuda() for k in ("rho", "B", "H", "ue", "ui")]
    for path in (_b.COOL_PATH_TEXTURE_POINT, _b.COOL_PATH_TEXTURE_HWLERP):
        for p in (cool.Params(path=path, mode=cool.IMPLICIT), cool.Params(path=path, fp64_critical=1)):
            with pytest.raises(cool.CoolError) as e:
                cool.step(tab, p, *tf)
            assert e.value.status == _b.COOL_EUNSUPPORTED
        with pytest.raises(cool.CoolError) as e:
            cool.step(tab, cool.Params(path=path), *[t.double() for t in tf])
        assert e.value.status == _b.COOL_EUNSUPPORTED
        half = cool.Table(cool.TableSpec(n=SMALL, dtype=cool.BF16))
        with pytest.raises(cool.CoolError) as e:
            cool.step(half, cool.Params(path=path), *tf)
        assert e.value.status == _b.COOL_EUNSUPPORTED
        g = torch.ones_like(tf[0])
        with pytest.raises(cool.CoolError) as e:
            cool.step_bwd(tab, cool.Params(path=path), *tf, g, g)
        assert e.value.status == _b.COOL_EUNSUPPORTED
