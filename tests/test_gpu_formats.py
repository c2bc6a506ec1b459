"""Reduced-precision table storage on the GPU (BF16 / FP16, plain and
block-scaled) against the oracle's storage mirror (oracle.quant).

* packing: the GPU's packed words equal the mirror's words computed from the
  oracle's FP64 table; a word may differ only where the two FP64 tables
  (equal to ~1e-14) straddle a rounding boundary, and then by one code;
* step: the GPU step on the packed table equals the oracle step reading the
  same stored values (oracle.step_pairs) within the FP32 bar, 1e-5, so the
  precision experiment isolates storage error from arithmetic error;
* the storage error of each process is printed (brems and Coulomb stay
  FP32; the synchrotron channel takes the 16-bit formats).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402

N5 = (12, 12, 12, 40, 24)
FORMATS = [("f32", 0, 0), ("bf16", 1, 0), ("f16", 2, 0), ("bf16_scaled", 1, 1), ("f16_scaled", 2, 1)]


@pytest.fixture(scope="module")
def env(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_08855_b300 as cool
    from paper_2505_08855_b300 import build
    build.build()
    ospec = oracle.Spec(n=N5)
    return cool, ospec, oracle.build_tables(ospec, nthreads=0)


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - b) / np.abs(b)


@pytest.mark.parametrize("name,dtype,scaled", FORMATS)
def test_packed_words_match_mirror(env, name, dtype, scaled):
    from oracle import quant
    cool, ospec, OT = env
    tab = cool.Table(cool.TableSpec(n=N5, dtype=dtype, row_scaled=scaled))
    fmt = quant.FMT[name]
    want, _ = quant.pack(OT["ls"], N5[3], fmt)
    got = tab.export_packed().reshape(want.shape)
    diff = got != want
    assert diff.mean() < 1e-3, name
    if diff.any():
        # only single-code rounding-boundary differences are allowed
        if fmt == 0:
            d = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
            assert d[diff].max() <= 1
        else:
            for sh in (0, 16):
                a = ((got >> sh) & 0xFFFF).astype(np.int64)
                b = ((want >> sh) & 0xFFFF).astype(np.int64)
                if fmt in (3, 4):
                    a[..., :2] = b[..., :2]   # off/scale words compared below
                assert np.abs(a - b).max() <= 1
            if fmt in (3, 4):
                for w in (0, 1):
                    x = got[..., w].view(np.float32).astype(np.float64)
                    y = want[..., w].view(np.float32).astype(np.float64)
                    assert np.all(np.abs(x - y) <= 2.0 ** -23 * np.abs(y) + 1e-30)


@pytest.mark.parametrize("name,dtype,scaled", FORMATS)
@pytest.mark.parametrize("mode", [0, 1])
def test_step_parity_on_stored_values(env, oracle, name, dtype, scaled, mode):
    from oracle import quant
    cool, ospec, OT = env
    tab = cool.Table(cool.TableSpec(n=N5, dtype=dtype, row_scaled=scaled))
    _, pairs = quant.pack(OT["ls"], N5[3], quant.FMT[name])
    lb32 = OT["lb"].astype(np.float32).astype(np.float64)
    lc32 = OT["lc"].astype(np.float32).astype(np.float64)
    f = inputs.uniform(20000 + 3, seed=50, dtype=np.float32)
    p = oracle.Params(n_sub=8, mode=mode)
    want = oracle.step_pairs(ospec, lb32, pairs, lc32, p, **f)
    tf = {k: torch.from_numpy(v).cuda() for k, v in f.items()}
    ue, ui = cool.step(tab, cool.Params(n_sub=8, mode=mode), tf["rho"], tf["B"], tf["H"], tf["ue"], tf["ui"])
    torch.cuda.synchronize()
    eu = rel(ue.cpu().numpy(), want[0])
    ei = rel(ui.cpu().numpy(), want[1])
    # the storage error itself, for the record: against the FP64 table
    full = oracle.step(ospec, OT, p, **f)
    su = rel(ue.cpu().numpy(), full[0]).max()
    print(f"\n{name} mode {mode}: vs stored values u_e {eu.max():.2e} u_i {ei.max():.2e}; "
          f"vs FP64 table u_e {su:.2e}; syn storage error {quant.storage_error(OT['ls'], N5[3], quant.FMT[name]):.2e} log2")
    assert eu.max() <= 1e-5 and ei.max() <= 1e-5
