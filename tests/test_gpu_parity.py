"""GPU parity of libcool against the FP64 CPU oracle (through the C ABI).

Tolerances:
  * table build (FP64 on the GPU vs FP64 oracle): |dlog2| <= 1e-12 max(1, |v|)
  * node arrays and index selection: bit-exact; weights within 2e-7
    (lg2.approx on [1, 2^dl]: ~2^-22 absolute)
  * FP64 step: max relative error <= 1e-12 per field
  * FP32 step: max relative error <= 1e-5 per field (u_e, u_i), the bar
    set for the FP32 path (FP32 log2 table storage alone contributes up to
    ln2 * 2^-17 ~ 5e-6 at |log2 Q| ~ 100)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

SMALL = (12, 12, 12, 16, 16)
CFG1 = (32, 32, 32, 32, 32)
TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module")
def cool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as c
    from paper_2505_08855_b300 import build
    build.build()
    return c


@pytest.fixture(scope="module")
def small(cool, oracle):
    tab = cool.Table(cool.TableSpec(n=SMALL))
    ospec = oracle.Spec(n=SMALL)
    return tab, ospec, oracle.build_tables(ospec, nthreads=0)


@pytest.fixture(scope="module")
def cfg1(cool, oracle):
    tab = cool.Table(cool.TableSpec(n=CFG1))
    ospec = oracle.Spec(n=CFG1)
    return tab, ospec, oracle.build_tables(ospec, nthreads=0)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def to_dev(f, dtype):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to("cuda", dtype) for k, v in f.items()}


def run_gpu(cool, tab, params, tf, **kw):
    qc = torch.empty_like(tf["ue"])
    qx = torch.empty_like(tf["ue"])
    cnt = cool.new_counters()
    ue, ui = cool.step(tab, params, tf["rho"], tf["B"], tf["H"], tf["ue"], tf["ui"],
                       q_cool=qc, q_cc=qx, counters=cnt, **kw)
    torch.cuda.synchronize()
    return (ue.cpu().double().numpy(), ui.cpu().double().numpy(), qc.cpu().double().numpy(),
            qx.cpu().double().numpy(), cool.counters_dict(cnt))


# ---- table -----------------------------------------------------------------------

def test_table_matches_oracle(small):
    tab, ospec, OT = small
    for ch, key in ((0, "lb"), (1, "ls"), (2, "lc")):
        g = tab.export(ch)
        o = np.asarray(OT[key]).reshape(-1)
        assert np.all(np.abs(g - o) <= 1e-12 * np.maximum(1.0, np.abs(o))), key


def test_nodes_bit_equal(small, oracle):
    tab, ospec, _ = small
    for a in range(5):
        assert np.array_equal(tab.nodes(a), oracle.nodes(ospec, a)[2])


def test_table_64_sampled_nodes(cool, oracle):
    """The full-size 64^4 table (bench workload): 3000 random nodes of the
    4-D channel and every node of the 1-D / 2-D channels."""
    n = (64,) * 5
    tab = cool.Table(cool.TableSpec(n=n))
    ospec = oracle.Spec(n=n)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, 64 ** 4, 3000)
    want = oracle.syn_at(ospec, idx)
    got = tab.export(1)[idx]
    assert np.all(np.abs(got - want) <= 1e-12 * np.maximum(1.0, np.abs(want)))
    OT = oracle.build_tables(ospec, syn=False)
    assert np.all(np.abs(tab.export(0) - OT["lb"]) <= 1e-12 * np.abs(OT["lb"]))
    assert np.all(np.abs(tab.export(2) - OT["lc"].reshape(-1)) <= 1e-12 * np.abs(OT["lc"].reshape(-1)))


def test_debug_lookup_bit_exact(cool, small, oracle):
    tab, ospec, _ = small
    rng = np.random.default_rng(0)
    for a in range(5):
        x32 = oracle.nodes(ospec, a)[2]
        keys = np.exp(rng.uniform(np.log(ospec.lo[a]) - 1, np.log(ospec.hi[a]) + 1, 1_000_000))
        near = np.concatenate([x32, np.nextafter(x32, 0), np.nextafter(x32, np.inf),
                               (x32 * (1 + rng.uniform(-1e-6, 1e-6, (200, x32.size)))).reshape(-1)])
        keys = np.concatenate([keys, near]).astype(np.float32)
        gi, gw = cool.debug_lookup(tab, a, torch.from_numpy(keys).cuda())
        oi, ow = oracle.select_f32(ospec, a, keys)
        assert np.array_equal(gi.cpu().numpy(), oi), a
        assert np.abs(gw.cpu().numpy() - ow).max() < 2e-7, a


def test_debug_lookup_step_rule(cool, small, oracle):
    """The step's selection (lookup axes 5..9 = table axes 0..4: the lg2
    guess, the weight band, exact node compares near a node) gives the exact
    rule's index bit for bit, on random keys, keys on the nodes, one ulp off
    them, within 1e-5 of them, and outside the axis; weights within 2e-7."""
    tab, ospec, _ = small
    rng = np.random.default_rng(1)
    for a in range(5):
        x32 = oracle.nodes(ospec, a)[2]
        keys = np.exp(rng.uniform(np.log(ospec.lo[a]) - 1, np.log(ospec.hi[a]) + 1, 1_000_000))
        near = np.concatenate([x32, np.nextafter(x32, 0), np.nextafter(x32, np.inf),
                               (x32 * (1 + rng.uniform(-1e-5, 1e-5, (400, x32.size)))).reshape(-1),
                               (x32 * (1 + rng.uniform(-1e-7, 1e-7, (400, x32.size)))).reshape(-1)])
        keys = np.concatenate([keys, near]).astype(np.float32)
        gi, gw = cool.debug_lookup(tab, a + 5, torch.from_numpy(keys).cuda())
        oi, ow = oracle.select_f32(ospec, a, keys)
        assert np.array_equal(gi.cpu().numpy(), oi), a
        assert np.abs(gw.cpu().numpy() - ow).max() < 2e-7, a


MIXED = (6, 40, 9, 33, 24)   # every axis a different size (and n_Tc != n_Te)


@pytest.fixture(scope="module")
def mixed(cool, oracle):
    tab = cool.Table(cool.TableSpec(n=MIXED))
    ospec = oracle.Spec(n=MIXED)
    return tab, ospec, oracle.build_tables(ospec, nthreads=0)


def test_mixed_axis_sizes_lookup(cool, mixed, oracle):
    """Both selection rules (exact node compares, axes 0..4; the step's lg2
    guess with its redo near a node, axes 5..9) on a table whose axes all
    differ in size: each axis uses its own guess constants and arrays.
    Indices bit-exact.  The weight is w = r / dl, r = log2(key * (1/x_j))
    by lg2.approx: r carries 2^-22 max(1, r) from lg2.approx plus the two
    FP32 roundings (1/x_j and the product, 2^-24 / ln 2 each in log2
    units), so |dw| <= (2^-22 max(1, r) + 2^-23 / ln 2) / dl + 2^-24
    <= 4.7e-7 max(1, 1/dl), 1/dl the nodes per octave (1.17 on the 40-node
    B axis, where 2e-7 no longer bounds it)."""
    tab, ospec, _ = mixed
    rng = np.random.default_rng(11)
    for a in range(5):
        x32 = oracle.nodes(ospec, a)[2]
        inv_dl = (MIXED[a] - 1) / np.log2(ospec.hi[a] / ospec.lo[a])
        w_tol = 4.7e-7 * max(1.0, inv_dl)
        keys = np.exp(rng.uniform(np.log(ospec.lo[a]) - 2, np.log(ospec.hi[a]) + 2, 200_000))
        near = np.concatenate([x32, np.nextafter(x32, 0), np.nextafter(x32, np.inf),
                               (x32 * (1 + rng.uniform(-1e-5, 1e-5, (200, x32.size)))).reshape(-1)])
        keys = np.concatenate([keys, near]).astype(np.float32)
        oi, ow = oracle.select_f32(ospec, a, keys)
        for axis in (a, a + 5):
            gi, gw = cool.debug_lookup(tab, axis, torch.from_numpy(keys).cuda())
            assert np.array_equal(gi.cpu().numpy(), oi), axis
            assert np.abs(gw.cpu().numpy() - ow).max() < w_tol, axis


@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_axis_sizes_step(cool, mixed, oracle, mode):
    tab, ospec, OT = mixed
    f = inputs.subsample(inputs.make("uniform_32c", dtype=np.float32), np.arange(0, 32 ** 3, 7)[:4099])
    want = oracle.step(ospec, OT, oracle.Params(n_sub=8, mode=mode), **f)
    got = run_gpu(cool, tab, cool.Params(n_sub=8, mode=mode), to_dev(f, torch.float32))
    for k in range(2):
        assert rel(got[k], want[k]).max() <= TOL32, k


# ---- step --------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n_sub", [4, 8])
def test_step_fp64_parity(cool, oracle, cfg1, mode, n_sub):
    tab, ospec, OT = cfg1
    f = inputs.make("uniform_32c")
    want = oracle.step(ospec, OT, oracle.Params(n_sub=n_sub, mode=mode), **f)
    got = run_gpu(cool, tab, cool.Params(n_sub=n_sub, mode=mode), to_dev(f, torch.float64))
    for k in range(2):
        assert rel(got[k], want[k]).max() <= TOL64
    scale = np.maximum(f["ue"], np.abs(want[2]))
    assert np.all(np.abs(got[2] - want[2]) <= TOL64 * scale)
    assert np.all(np.abs(got[3] - want[3]) <= TOL64 * np.maximum(f["ue"] + f["ui"], 0))
    assert got[4]["stiff"] == want[4]["stiff"]
    assert got[4]["nonfinite"] == 0


@pytest.mark.parametrize("fp64_critical", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n_sub", [4, 8])
def test_step_fp32_parity(cool, oracle, cfg1, mode, n_sub, fp64_critical):
    tab, ospec, OT = cfg1
    f = inputs.make("uniform_32c", dtype=np.float32)
    want = oracle.step(ospec, OT, oracle.Params(n_sub=n_sub, mode=mode), **f)
    got = run_gpu(cool, tab, cool.Params(n_sub=n_sub, mode=mode, fp64_critical=fp64_critical),
                  to_dev(f, torch.float32))
    eu, ei = rel(got[0], want[0]), rel(got[1], want[1])
    print(f"\nFP32 mode {mode} n_sub {n_sub} fp64_critical {fp64_critical}: "
          f"max rel u_e {eu.max():.2e}, u_i {ei.max():.2e}")
    assert eu.max() <= TOL32 and ei.max() <= TOL32
    # diagnostics: conservation identities hold on the GPU outputs
    ue0 = f["ue"].astype(np.float64)
    slack = 4e-6 * np.maximum(ue0, got[0]) + 1e-6 * (np.abs(got[3]) + np.abs(got[2]))
    assert np.all(np.abs(got[0] - (ue0 + got[3] - got[2])) <= slack)
    # stiff decisions may differ only where q is within rounding of the limiter
    assert abs(got[4]["stiff"] - want[4]["stiff"]) <= 2 + want[4]["stiff"] // 1000


@pytest.mark.parametrize("mode,fp64", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_ragged_unaligned_inplace_bitwise(cool, cfg1, mode, fp64):
    """The 128-bit path, the scalar tail and the unaligned scalar path give
    bit-identical cells; in-place output equals out-of-place.  In implicit
    mode and with fp64_critical the aligned call lists its flagged cells
    (from its tiles and its ragged tail) for the list kernel, the unaligned
    one steps every cell on its own lane: the same bits."""
    tab, _, _ = cfg1
    n = 4 * 1000 + 3
    f = inputs.uniform(n + 1, seed=21, dtype=np.float32)
    tf = to_dev(f, torch.float32)
    p = cool.Params(n_sub=8, mode=mode, fp64_critical=fp64)
    full = {k: v[:n].contiguous() for k, v in tf.items()}
    ue_a, ui_a = cool.step(tab, p, full["rho"], full["B"], full["H"], full["ue"], full["ui"])
    off = {k: v[1:n + 1] for k, v in {k: torch.cat([v[:1], v[:n]]) for k, v in tf.items()}.items()}
    assert off["rho"].data_ptr() % 16 != 0
    ue_b, ui_b = cool.step(tab, p, off["rho"], off["B"], off["H"], off["ue"], off["ui"])
    ue_c = full["ue"].clone()
    ui_c = full["ui"].clone()
    cool.step(tab, p, full["rho"], full["B"], full["H"], ue_c, ui_c, ue_out=ue_c, ui_out=ui_c)
    torch.cuda.synchronize()
    assert torch.equal(ue_a, ue_b) and torch.equal(ui_a, ui_b)
    assert torch.equal(ue_a, ue_c) and torch.equal(ui_a, ui_c)
    for m in (1, 2, 3, 5):
        part = {k: v[:m].contiguous() for k, v in tf.items()}
        ue_m, _ = cool.step(tab, p, part["rho"], part["B"], part["H"], part["ue"], part["ui"])
        assert torch.equal(ue_m, ue_a[:m])


def test_empty_and_invalid_cells(cool, cfg1):
    tab, _, _ = cfg1
    p = cool.Params()
    e = torch.empty(0, device="cuda")
    ue, ui = cool.step(tab, p, e, e, e, e, e)
    assert ue.numel() == 0
    f = inputs.uniform(64, seed=22, dtype=np.float32)
    f["rho"][0] = np.nan
    f["ue"][1] = -1.0
    f["ui"][2] = np.inf
    f["rho"][3] = 0.0
    f["B"][4] = -2.0
    f["H"][5] = np.nan
    tf = to_dev(f, torch.float32)
    got = run_gpu(cool, tab, p, tf)
    assert got[4]["nonfinite"] == 6
    for i in range(6):
        assert np.array_equal(got[0][i], f["ue"][i], equal_nan=True)
        assert np.array_equal(got[1][i], f["ui"][i], equal_nan=True)
    assert np.all(np.isfinite(got[0][6:])) and np.all(got[0][6:] > 0)


def test_out_of_range_keys_clamp(cool, oracle, cfg1):
    tab, ospec, OT = cfg1
    f = inputs.uniform(4096, seed=23, dtype=np.float32)
    f["H"][:100] *= 1e8       # H_cm beyond 1e12 cm
    f["rho"][100:200] = 1e-20  # n_e below 1e2
    f["ue"][200:300] *= 1e-12  # T_e below 1e2 K
    want = oracle.step(ospec, OT, oracle.Params(n_sub=4), **f)
    got = run_gpu(cool, tab, cool.Params(n_sub=4), to_dev(f, torch.float32))
    assert rel(got[0], want[0]).max() <= TOL32
    assert rel(got[1], want[1]).max() <= TOL32
    assert got[4]["clamped"] == want[4]["clamped"] >= 300


def test_bad_arguments(cool, cfg1):
    tab, _, _ = cfg1
    t = torch.ones(8, device="cuda")
    with pytest.raises(cool.CoolError):
        cool.step(tab, cool.Params(n_sub=0), t, t, t, t, t)
    with pytest.raises(cool.CoolError):
        cool.step(tab, cool.Params(limiter_frac=0.0), t, t, t, t, t)
    for path in (4, 99):   # the surrogate path is cool_surrogate_infer's; 99 is no path
        with pytest.raises(cool.CoolError):
            cool.step(tab, cool.Params(path=path), t, t, t, t, t)


def test_save_load_roundtrip(cool, cfg1, tmp_path):
    tab, _, _ = cfg1
    path = str(tmp_path / "t.cooltab")
    tab.save(path)
    t2 = cool.Table.load(path)
    for ch in range(3):
        assert np.array_equal(t2.export(ch), tab.export(ch))
    f = to_dev(inputs.uniform(1000, seed=24, dtype=np.float32), torch.float32)
    p = cool.Params()
    a = cool.step(tab, p, f["rho"], f["B"], f["H"], f["ue"], f["ui"])
    b = cool.step(t2, p, f["rho"], f["B"], f["H"], f["ue"], f["ui"])
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    with pytest.raises(cool.CoolError):
        cool.Table.load(path)
    t2.free()
    with pytest.raises(cool.CoolError):
        t2.export(0)


def test_full_size_sampled_parity(cool, oracle):
    """256^3 two-region cells, 64^4 table, 8 sub-cycles, launched as the
    benchmark launches it; 1500 sampled cells against the oracle (lazy
    table: only the nodes those cells visit are evaluated)."""
    n = (64,) * 5
    tab = cool.Table(cool.TableSpec(n=n))
    F = inputs.make("two_region_256c")
    tf = to_dev(F, torch.float32)
    p = cool.Params(n_sub=8)
    ue, ui = cool.step(tab, p, tf["rho"], tf["B"], tf["H"], tf["ue"], tf["ui"])
    torch.cuda.synchronize()
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(F["rho"].size, 1500, replace=False))
    sub = inputs.subsample(F, idx)
    ospec = oracle.Spec(n=n)
    OT = oracle.build_tables(ospec, syn=False)
    want = oracle.step(ospec, OT, oracle.Params(n_sub=8), **sub, lazy=True)
    eu = rel(ue.cpu().numpy()[idx], want[0])
    ei = rel(ui.cpu().numpy()[idx], want[1])
    print(f"\nfull-size sample: max rel u_e {eu.max():.2e}, u_i {ei.max():.2e}")
    assert eu.max() <= TOL32 and ei.max() <= TOL32


@pytest.mark.parametrize("mode", [0, 1])
def test_paper_size_table_sampled_parity(cool, oracle, mode):
    """The paper's table size (100 nodes per axis, Sec. 2.6; 457 MB packed,
    beyond L2) on the 256^3 two-region cells, 8 sub-cycles, explicit and
    implicit, launched as the benchmark launches its step; 1024 sampled
    cells against the oracle (lazy 100^4 table)."""
    n = (100,) * 5
    tab = cool.Table(cool.TableSpec(n=n))
    F = inputs.make("two_region_256c")
    tf = to_dev(F, torch.float32)
    p = cool.Params(n_sub=8, mode=mode)
    ue, ui = cool.step(tab, p, tf["rho"], tf["B"], tf["H"], tf["ue"], tf["ui"])
    torch.cuda.synchronize()
    tab.free()
    idx = np.sort(np.random.default_rng(100 + mode).choice(F["rho"].size, 1024, replace=False))
    sub = inputs.subsample(F, idx)
    ospec = oracle.Spec(n=n)
    OT = oracle.build_tables(ospec, syn=False)
    want = oracle.step(ospec, OT, oracle.Params(n_sub=8, mode=mode), **sub, lazy=True)
    eu = rel(ue.cpu().numpy()[idx], want[0])
    ei = rel(ui.cpu().numpy()[idx], want[1])
    print(f"\n100^4 table, mode {mode}: max rel u_e {eu.max():.2e}, u_i {ei.max():.2e}")
    assert eu.max() <= TOL32 and ei.max() <= TOL32
