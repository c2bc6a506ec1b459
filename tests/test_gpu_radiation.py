"""cool_radiation_te (the radiation-pressure correction of T_e, Sec. 5.2)
against the oracle's closed-form quartic root: FP32 within 1e-5 relative
(the scaled Newton iteration converges to FP32 precision; FP32 logarithms
and the FP32 key T_e,sim = s_Te u_e / rho add a few ulp); the thick flags
equal except where tau_sca lies within FP32 rounding of tau_crit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2505_08855_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def fields():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_08855_b300 import build
    build.build()
    f = inputs.make("uniform_128c")
    n = 1_000_003
    rng = np.random.default_rng(8)
    scale = np.exp(rng.uniform(0, 28, n)).astype(np.float32)     # densities reaching the thick regime
    rho = (f["rho"][:n] * scale).astype(np.float32)
    ue = (f["ue"][:n] * scale).astype(np.float32)
    H = f["H"][:n].copy()
    rho[5], ue[6], H[7] = -1.0, np.nan, -3.0
    return rho, H, ue


@pytest.mark.parametrize("offset", [0, 1])
def test_matches_oracle(fields, oracle, offset):
    import paper_2505_08855_b300 as cool
    rho, H, ue = (a[offset:] for a in fields)
    p = cool.Params()
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rho, H, ue)]
    thick = torch.zeros(rho.size, dtype=torch.uint8, device="cuda")
    te, _ = cool.radiation_te(p, *t, thick_out=thick)
    torch.cuda.synchronize()
    got = te.cpu().numpy().astype(np.float64)
    gth = thick.cpu().numpy().astype(bool)
    want, wth = oracle.radiation_te(oracle.Params(), rho, H, ue, tau_crit=4.6, a_rad=cool.A_RAD_PAPER)
    bad = ~np.isfinite(want)
    assert np.array_equal(bad, ~np.isfinite(got)) and bad.sum() == 3
    rs = 1.67262192369e-24
    tau = rho.astype(np.float64) * (3e-7 / rs) * 6.6524587321e-25 * H * (6.6743e-8 * 10 * 1.98847e33 /
                                                                        2.99792458e10 ** 2)
    edge = np.abs(tau / 4.6 - 1) < 1e-5
    ok = ~bad & ~edge
    assert np.array_equal(gth[ok], wth[ok])
    assert wth[ok].mean() > 0.1 and (~wth[ok]).mean() > 0.1
    r = np.abs(got[ok] - want[ok]) / want[ok]
    print(f"\nradiation T_e: max rel {r.max():.2e}, thick cells {wth[ok].sum()} of {ok.sum()}")
    assert r.max() <= 1e-5
