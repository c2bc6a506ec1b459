"""Pins of the oracle's paper's-layout table and step (Sec. 3.1: one 4-D
table of the total cooling rate, the bridge of Eqs. 11-12 folded in), no
GPU.

* The table at its nodes equals the total rate from the direct formulas
  (O1: bremsstrahlung + eta Q_syn, then the bridge): a wrong node index, a
  dropped n_e^2 or a transposed axis fails it.
* On keys at the nodes the interpolation returns node values, so one
  sub-cycle of the paper's-layout step cools exactly as the factored step
  (which bridges the node values at run time).
* Away from nodes the two readings differ by the interpolation of a
  nonlinear bridge: both are within the table's interpolation error of O1.
"""
import numpy as np
import pytest

N5 = (6, 7, 8, 12, 9)


@pytest.fixture(scope="module")
def env(oracle):
    spec = oracle.Spec(n=N5)
    tab = oracle.build_tables(spec, nthreads=8)
    return spec, tab, oracle.build_qtotal(spec, tab)


def _node(oracle, spec, a, j):
    x64, l64, _ = oracle.nodes(spec, a)
    return x64[j]


def test_table_equals_direct_total_rate_at_nodes(oracle, env):
    spec, tab, lt = env
    rng = np.random.default_rng(5)
    nH, nB, nN, nT, _ = N5
    for _ in range(60):
        h, b, n, t = (int(rng.integers(0, m)) for m in (nH, nB, nN, nT))
        H, B, ne, T = (_node(oracle, spec, a, j) for a, j in ((0, h), (1, b), (2, n), (3, t)))
        want = np.log2(oracle.qtotal_direct(H, B, ne, T, spec))
        got = lt[((h * nB + b) * nN + n) * nT + t]
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (h, b, n, t)


def _cells_on_nodes(oracle, spec, p, rng, m):
    """Fields whose (H_cm, B_G, n_e, T_e) keys are nodes of the table and
    T_i = T_e (no exchange)."""
    G, MSUN, C, MP, KB = (oracle.const(k) for k in ("G", "M_sun", "c", "m_p", "k_B"))
    rg = G * p.M_bh_msun * MSUN / C ** 2
    s_n = p.rho_scale / MP
    s_B = np.sqrt(4 * np.pi * p.rho_scale) * C
    s_T = (p.gamma_e - 1) * MP * C ** 2 / KB
    out = {k: np.zeros(m) for k in ("rho", "B", "H", "ue", "ui")}
    for i in range(m):
        h, b, n = (int(rng.integers(1, N5[a] - 1)) for a in range(3))
        t = int(rng.integers(1, N5[3] - 1))
        ne = _node(oracle, spec, 2, n)
        rho = ne / s_n
        out["rho"][i] = rho
        out["B"][i] = _node(oracle, spec, 1, b) / s_B
        out["H"][i] = _node(oracle, spec, 0, h) / rg
        out["ue"][i] = out["ui"][i] = _node(oracle, spec, 3, t) * rho / s_T
    return out


def test_step_on_node_keys_equals_factored_step(oracle, env):
    spec, tab, lt = env
    p = oracle.Params(n_sub=1)
    f = _cells_on_nodes(oracle, spec, p, np.random.default_rng(6), 400)
    args = [f[k] for k in ("rho", "B", "H", "ue", "ui")]
    a = oracle.step(spec, tab, p, *args)
    b = oracle.step_qtotal(spec, tab, lt, p, *args)
    # q_cool relative to u_e: the keys are nodes up to one rounding of the
    # unit conversions (~1e-16 of a node spacing)
    assert np.allclose(b[2], a[2], rtol=1e-9, atol=1e-12 * f["ue"].max())
    assert np.allclose(b[0], a[0], rtol=1e-12)


def test_both_layouts_near_the_direct_formulas(oracle, env):
    """Off the nodes both table readings stay within the table's
    interpolation error of O1 (a few per cent on this coarse grid)."""
    spec, tab, lt = env
    from paper_2505_08855_b300 import inputs
    f = inputs.subsample(inputs.make("uniform_32c"), np.arange(0, 32 ** 3, 97))
    p = oracle.Params(n_sub=1)
    args = [f[k] for k in ("rho", "B", "H", "ue", "ui")]
    o1 = oracle.step(spec, tab, p, *args, direct=True)
    fa = oracle.step(spec, tab, p, *args)
    qt = oracle.step_qtotal(spec, tab, lt, p, *args)
    e_fa = np.abs(fa[0] - o1[0]) / o1[0]
    e_qt = np.abs(qt[0] - o1[0]) / o1[0]
    assert np.median(e_fa) < 0.05 and np.median(e_qt) < 0.05
