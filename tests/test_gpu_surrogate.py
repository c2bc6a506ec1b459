"""The surrogate network's GPU kernels against the numpy reference
(oracle.mlp, pinned by finite differences), its training, and the step
that uses it (cool_surrogate_infer) against the oracle's surrogate step.

* gradients of one batch (all five tcgen05 products of the training tile):
  each parameter group within 2e-3 of its largest entry -- both sides round
  the same operands to bf16; a value within rounding of a bf16 boundary may
  round the other way (one bf16 ulp, 0.4 %, of that element);
* forward evaluation within 1e-3 standard deviations;
* training on the GPU lowers the loss and fits the channel.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N5 = (12, 12, 12, 24, 16)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    tab = cool.Table(cool.TableSpec(n=N5))
    return cool, tab


def _groups():
    from oracle import mlp
    return {"W1": (mlp.P_W1, mlp.P_b1), "b1": (mlp.P_b1, mlp.P_W2), "W2": (mlp.P_W2, mlp.P_b2),
            "b2": (mlp.P_b2, mlp.P_w3), "w3": (mlp.P_w3, mlp.P_b3), "b3": (mlp.P_b3, mlp.P_N)}


def test_grads_match_reference(env):
    from oracle import mlp
    cool, tab = env
    s = cool.Surrogate(tab, cool.FitSpec(n_samples=1 << 14, batch=1 << 14, epochs=0))
    p = s.params().astype(np.float64)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (2048, 4)).astype(np.float32)
    y = rng.normal(0, 1, 2048).astype(np.float32)
    g, loss = s.grads(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    want, wloss = mlp.grads(p, x.astype(np.float64), y.astype(np.float64), s.info()["x_switch"])
    assert abs(loss - wloss) <= 1e-4 * wloss
    for name, (a, b) in _groups().items():
        scale = np.abs(want[a:b]).max()
        err = np.abs(g[a:b] - want[a:b]).max() / scale
        print(f"\ngrad {name}: max |diff| / max |g| = {err:.2e}")
        assert err <= 2e-3, name


def test_eval_matches_reference(env):
    from oracle import mlp
    cool, tab = env
    s = cool.Surrogate(tab, cool.FitSpec(n_samples=1 << 14, batch=1 << 14, epochs=0))
    p = s.params().astype(np.float64)
    info = s.info()
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (5000, 4)).astype(np.float32)
    got = s.eval(torch.from_numpy(x).cuda()).cpu().numpy()
    want = info["mean"] + info["std"] * mlp.forward(p, x.astype(np.float64), info["x_switch"])
    assert np.abs(got - want).max() <= 1e-3 * info["std"]


def test_training_fits_the_channel(env, oracle):
    cool, tab = env
    s = cool.Surrogate(tab, cool.FitSpec(n_samples=1 << 20, batch=8192, epochs=6, lr=3e-3))
    info = s.info()
    print(f"\ntrained: loss {info['final_loss']:.3e} (standardised), steps {info['steps']}, "
          f"fallback cells {info['fallback_cells']} / {info['mask_cells']}, std {info['std']:.1f} log2")
    assert info["steps"] == (1 << 20) // 8192 * 6
    assert info["final_loss"] < 0.02
    # the network follows the channel over its ~270 log2 units of range (a
    # coarse fit: the fallback mask, not this test, decides where it is used)
    ospec = oracle.Spec(n=N5)
    rng = np.random.default_rng(5)
    idx = [rng.integers(0, k, 400) for k in N5[:4]]
    x = np.stack([2 * idx[d] / (N5[d] - 1) - 1 for d in range(4)], axis=1).astype(np.float32)
    flat = ((idx[0] * N5[1] + idx[1]) * N5[2] + idx[2]) * N5[3] + idx[3]
    want = oracle.syn_at(ospec, flat)
    got = s.eval(torch.from_numpy(x).cuda()).cpu().numpy()
    print(f"node error: median {np.median(np.abs(got - want)):.2f}, max {np.abs(got - want).max():.1f} log2")
    assert np.median(np.abs(got - want)) < 5.0
    assert np.corrcoef(got, want)[0, 1] > 0.99


# ---- the step with the network (cool_surrogate_infer) ------------------------

@pytest.fixture(scope="module")
def infer_env(env, oracle):
    from paper_2505_08855_b300 import inputs
    cool, tab = env
    s = cool.Surrogate(tab, cool.FitSpec(n_samples=1 << 18, batch=8192, epochs=2, lr=3e-3))
    spec = oracle.Spec(n=N5)
    otab = oracle.build_tables(spec, nthreads=8)
    f = inputs.make("uniform_32c")
    f = inputs.subsample(f, np.arange(0, 32 ** 3, 8)[:4099])        # 32 tiles of 128 + 3
    f = {k: v.astype(np.float32) for k, v in f.items()}
    return cool, tab, s, spec, otab, f


def _gpu_fields(f):
    return [torch.from_numpy(f[k]).cuda() for k in ("rho", "B", "H", "ue", "ui")]


def _run_infer(cool, s, prm, f):
    fl = _gpu_fields(f)
    qc = torch.empty_like(fl[0])
    qx = torch.empty_like(fl[0])
    cnt = cool.new_counters()
    ue, ui = s.step(prm, *fl, q_cool=qc, q_cc=qx, counters=cnt)
    torch.cuda.synchronize()
    return [t.cpu().numpy().astype(np.float64) for t in (ue, ui, qc, qx)], cool.counters_dict(cnt)


def _oracle_fields(f):
    return [f[k].astype(np.float64) for k in ("rho", "B", "H", "ue", "ui")]


def test_infer_all_fallback_is_the_table_step(infer_env):
    """Every fallback bit set: the network is never used and the step equals
    cool_step on the same table (the same FP32 arithmetic)."""
    cool, tab, s, spec, otab, f = infer_env
    cells = s.info()["mask_cells"]
    s.set_mask(np.full((cells + 31) // 32, 0xFFFFFFFF, np.uint32))
    prm = cool.Params(n_sub=4)
    got, cnt = _run_infer(cool, s, prm, f)
    fl = _gpu_fields(f)
    qc = torch.empty_like(fl[0])
    qx = torch.empty_like(fl[0])
    ue, ui = cool.step(tab, prm, *fl, q_cool=qc, q_cc=qx)
    want = [t.cpu().numpy().astype(np.float64) for t in (ue, ui, qc, qx)]
    for k in range(4):
        err = np.max(np.abs(got[k] - want[k]) / np.maximum(np.abs(want[k]), 1e-30))
        print(f"\nfield {k}: max rel diff vs cool_step {err:.1e}")
        assert err <= 1e-6, k
    assert cnt["fallback"] == f["rho"].size - cnt["nonfinite"]


def _compare_net_step(got, want, n):
    """GPU vs oracle with the network in use.  Both sides round the network
    input to two bf16 parts, but the kernel forms it from FP32 keys and the
    oracle from FP64 ones: the low part resolves 2^-16 of the coordinate, so
    in about one evaluation in a hundred the two round it differently and
    the network output moves by (its slope) x 2^-16 x 2, a few 1e-4 relative
    in Q_syn.  A hidden activation within rounding of a bf16 tie flips the
    same way, rarely.  So: the median cell within 1e-5, 99 % of cells within
    1e-3, every cell within 3e-2 (relative, u_e and u_i; q_cool relative to
    u_e)."""
    ue_g, ui_g, qc_g = got[:3]
    ue_o, ui_o, qc_o = want[:3]
    rel = np.maximum(np.abs(ue_g - ue_o) / ue_o, np.abs(ui_g - ui_o) / ui_o)
    rel = np.maximum(rel, np.abs(qc_g - qc_o) / ue_o)
    q50, q99, qmax = np.median(rel), np.quantile(rel, 0.99), rel.max()
    print(f"\nnetwork step vs oracle: median {q50:.1e}, 99% {q99:.1e}, max {qmax:.1e} (n={n})")
    assert q50 <= 1e-5 and q99 <= 1e-3 and qmax <= 3e-2


def test_infer_network_matches_oracle(infer_env, oracle):
    cool, tab, s, spec, otab, f = infer_env
    cells = s.info()["mask_cells"]
    s.set_mask(np.zeros((cells + 31) // 32, np.uint32))
    info = s.info()
    prm = cool.Params(n_sub=4)
    got, cnt = _run_infer(cool, s, prm, f)
    want = oracle.step_surrogate(spec, otab, s.params(), info["mean"], info["std"], None,
                                 oracle.Params(n_sub=4), *_oracle_fields(f))
    _compare_net_step(got, want, f["rho"].size)
    assert cnt["fallback"] == 0 and want[4]["fallback"] == 0
    # the network is not a bystander: its channel changes the step
    tabstep = oracle.step(spec, otab, oracle.Params(n_sub=4), *_oracle_fields(f))
    assert np.mean(np.abs(tabstep[2] - want[2]) > 1e-3 * np.abs(tabstep[2]) + 1e-30) > 0.05


def test_infer_mixed_mask_matches_oracle(infer_env, oracle):
    cool, tab, s, spec, otab, f = infer_env
    cells = s.info()["mask_cells"]
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, (cells + 31) // 32, dtype=np.uint64).astype(np.uint32)
    s.set_mask(bits)
    info = s.info()
    assert 0.4 * cells < info["fallback_cells"] < 0.6 * cells
    prm = cool.Params(n_sub=4)
    got, cnt = _run_infer(cool, s, prm, f)
    want = oracle.step_surrogate(spec, otab, s.params(), info["mean"], info["std"], s.mask(),
                                 oracle.Params(n_sub=4), *_oracle_fields(f))
    _compare_net_step(got, want, f["rho"].size)
    print(f"fallback cells: GPU {cnt['fallback']}, oracle {want[4]['fallback']}")
    assert abs(cnt["fallback"] - want[4]["fallback"]) <= 0.01 * f["rho"].size
    assert 0 < want[4]["fallback"] < f["rho"].size


def test_infer_invalid_cells_and_errors(infer_env):
    from paper_2505_08855_b300 import binding as _b
    cool, tab, s, spec, otab, f = infer_env
    g = {k: v[:300].copy() for k, v in f.items()}
    g["rho"][5] = -1.0
    g["ue"][7] = np.nan
    g["B"][9] = -2.0
    prm = cool.Params(n_sub=4)
    got, cnt = _run_infer(cool, s, prm, g)
    for i in (5, 7, 9):
        assert (np.isnan(got[0][i]) and np.isnan(g["ue"][i])) or got[0][i] == g["ue"][i]
        assert got[1][i] == g["ui"][i] and got[2][i] == 0.0
    assert cnt["nonfinite"] == 3
    fl = _gpu_fields(g)
    with pytest.raises(cool.CoolError) as e:
        s.step(cool.Params(n_sub=4, mode=1), *fl)
    assert e.value.status == _b.COOL_EUNSUPPORTED
    other = cool.Table(cool.TableSpec(n=(12, 12, 12, 16, 16)))
    with pytest.raises(cool.CoolError) as e:
        s.step(prm, *fl, table=other)
    assert e.value.status == _b.COOL_EINVAL
    half = cool.Table(cool.TableSpec(n=N5, dtype=cool.BF16))
    with pytest.raises(cool.CoolError) as e:
        s.step(prm, *fl, table=half)
    assert e.value.status == _b.COOL_EUNSUPPORTED
    empty = [t[:0] for t in fl]
    s.step(prm, *empty)


# ---- what the surrogate buys -----------------------------------------------------

def test_surrogate_gain_vs_equal_bytes_table(oracle):
    """The surrogate's gain is storage, not speed: against the direct
    formulas (O1) at random off-node points of the box, compare the network
    (about 35 KB as stored for inference, 16384 Adam steps on 2^22 samples)
    with a table of the same byte budget (9^4 FP32 nodes, 26 KB) and with
    the table it was fitted to (512 KB).  The
    network is also smooth: its log2 output has a continuous first
    derivative, where the multilinear table's slope jumps at every node."""
    import paper_2505_08855_b300 as cool
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n_fit = (16, 16, 16, 32, 16)
    tab = cool.Table(cool.TableSpec(n=n_fit))
    s = cool.Surrogate(tab, cool.FitSpec(n_samples=1 << 22, batch=16384, epochs=64, lr=2e-3))
    info = s.info()
    spec = oracle.Spec(n=n_fit)
    l0, span, xs = oracle.net_box(spec)
    rng = np.random.default_rng(21)
    npts = 1500
    x = rng.uniform(-0.98, 0.98, (npts, 4))
    lv = l0 + (x + 1) * span / 2
    pts = np.exp2(lv)
    o1 = np.array([np.log2(oracle.eta_qsyn(*p, spec=spec)) for p in pts])
    net = s.eval(torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy().astype(np.float64)
    small = oracle.Spec(n=(9, 9, 9, 9, 16))
    st = oracle.build_tables(small, nthreads=8)
    t9 = np.array([oracle.interp_syn(small, st, *p) for p in pts])
    ft = oracle.build_tables(spec, nthreads=8)
    tf = np.array([oracle.interp_syn(spec, ft, *p) for p in pts])
    ok = np.isfinite(o1)
    e_net, e_9, e_f = (np.abs(a[ok] - o1[ok]) for a in (net, t9, tf))
    table_bytes_9 = 9 ** 4 * 4
    print(f"\nnetwork: {info['param_bytes_bf16']} B, loss {info['final_loss']:.2e}, "
          f"fallback {info['fallback_cells']}/{info['mask_cells']}")
    for name, e in (("network", e_net), (f"9^4 table ({table_bytes_9} B)", e_9),
                    (f"fitted table ({16 ** 3 * 32 * 4} B)", e_f)):
        print(f"  |l - l_O1| {name}: median {np.median(e):.3f}, 90% {np.quantile(e, 0.9):.3f}, "
              f"max {e.max():.2f} log2")
    # smoothness along T_e: first differences of the network (rounding off,
    # C restatement) vary continuously; the table's jump at nodes
    p = s.params()
    t = np.linspace(-0.9, 0.9, 3601)
    base = rng.uniform(-0.8, 0.8, 3)
    line = np.column_stack([np.full_like(t, base[0]), np.full_like(t, base[1]), np.full_like(t, base[2]), t])
    yn = oracle.net_eval(p, info["mean"], info["std"], xs, line, rounding=False)
    dt = t[1] - t[0]
    sl = np.diff(yn) / dt
    jump_net = np.abs(np.diff(sl))
    lt = l0[3] + (t + 1) * span[3] / 2
    yt = np.array([oracle.interp_syn(spec, ft, *np.exp2(l0[:3] + (base + 1) * span[:3] / 2), np.exp2(v))
                   for v in lt])
    jump_tab = np.abs(np.diff(np.diff(yt) / dt))
    far = np.abs(t[1:-1] - xs) > 3 * dt          # away from the switch
    print(f"  slope change per step along T_e away from the switch: network max {jump_net[far].max():.3f}, "
          f"fitted table max {jump_tab[far].max():.1f} (log2 per unit of x)")
    # why the network cannot replace the table at the fallback tolerance
    # (|2^(l_net - l_table) - 1| <= 1e-3, i.e. 0.00144 log2): at table nodes,
    # the error of the exact network (FP64, no rounding: what training
    # reached) and the error added by the bf16 operands of the tensor-core
    # products (rounded minus exact network), against the table's values
    tol = np.log2(1.0 + 1e-3)
    nodes = rng.integers(0, np.array(n_fit[:4]), size=(20000, 4))
    xn = 2.0 * nodes / (np.array(n_fit[:4]) - 1.0) - 1.0
    l_tab = np.asarray(ft["ls"]).reshape(n_fit[:4])[nodes[:, 0], nodes[:, 1], nodes[:, 2], nodes[:, 3]]
    y64 = oracle.net_eval(p, info["mean"], info["std"], xs, xn, rounding=False)
    y16 = oracle.net_eval(p, info["mean"], info["std"], xs, xn, rounding=True)
    e_apx, e_rnd, e_tot = np.abs(y64 - l_tab), np.abs(y16 - y64), np.abs(y16 - l_tab)
    print(f"  at 20000 table nodes (output std {info['std']:.1f} log2): exact-network error median "
          f"{np.median(e_apx):.3f}, 10 % {np.quantile(e_apx, 0.1):.4f}; bf16-operand rounding median "
          f"{np.median(e_rnd):.4f}, 10 % {np.quantile(e_rnd, 0.1):.5f}; nodes within the 1e-3 tolerance: "
          f"exact network {np.mean(e_apx <= tol):.4f}, as run {np.mean(e_tot <= tol):.4f}")
    # with 16384 Adam steps (measured: median 0.21, 90 % 0.77, max 12.4 log2
    # against 0.41, 3.96, 25.3 for the equal-bytes table) the network is the
    # better use of 35 KB on all three; it stays far from the fitted table
    # (0.026 median), which is why the fallback mask exists
    assert info["param_bytes_bf16"] * 14 < 16 ** 3 * 32 * 4
    assert jump_net[far].max() < 0.05 * jump_tab[far].max()
    assert np.median(e_net) < 0.75 * np.median(e_9)
    assert np.quantile(e_net, 0.9) < 0.5 * np.quantile(e_9, 0.9)
    assert e_net.max() < e_9.max()
