"""Pins of the oracle's table, interpolation and sub-cycled step (no GPU).

Interpolation is pinned by exactness at nodes and on log-affine tables, by
numpy's searchsorted for the index rule and by its second-order convergence
to the direct formulas; the step by conservation laws, closed forms of the
limiter / Coulomb clamp, and the implicit residual.
"""
import math

import numpy as np
import pytest

from paper_2505_08855_b300 import inputs

C_LIGHT = 2.99792458e10
K_B = 1.380649e-16
M_P = 1.67262192369e-24


@pytest.fixture(scope="module")
def small(oracle):
    spec = oracle.Spec(n=(12, 12, 12, 16, 16))
    return spec, oracle.build_tables(spec, nthreads=8)


def test_nodes_log_spaced_inclusive(oracle):
    spec = oracle.Spec(n=(7, 9, 11, 13, 5))
    for a in range(5):
        x64, l64, x32 = oracle.nodes(spec, a)
        assert abs(x64[0] / spec.lo[a] - 1) < 1e-15
        assert abs(x64[-1] / spec.hi[a] - 1) < 1e-14
        r = x64[1:] / x64[:-1]
        assert np.allclose(r, (spec.hi[a] / spec.lo[a]) ** (1 / (spec.n[a] - 1)), rtol=1e-13)
        assert np.all(x32 == x64.astype(np.float32))


def test_select_matches_searchsorted(oracle):
    spec = oracle.Spec(n=(8, 16, 32, 64, 128))
    rng = np.random.default_rng(5)
    for a in range(5):
        x64, l64, x32 = oracle.nodes(spec, a)
        N = x32.size
        keys = np.exp(rng.uniform(np.log(spec.lo[a]) - 2, np.log(spec.hi[a]) + 2, 20000)).astype(np.float32)
        # keys exactly on nodes and one ulp either side
        on = np.concatenate([x32, np.nextafter(x32, 0), np.nextafter(x32, np.inf)])
        keys = np.concatenate([keys, on.astype(np.float32)])
        idx, w = oracle.select_f32(spec, a, keys)
        ref = np.clip(np.searchsorted(x32, keys, side="right") - 1, 0, N - 2)
        assert np.array_equal(idx, ref)
        wref = np.clip((np.log2(keys.astype(np.float64)) - l64[ref]) / (l64[1] - l64[0]), 0, 1)
        assert np.allclose(w, wref, rtol=0, atol=1e-13)
        # last node -> cell N-2 with w = 1; first node -> cell 0, w = 0
        i2, w2 = oracle.select_f32(spec, a, np.array([x32[-1], x32[0]], np.float32))
        assert i2[0] == N - 2 and abs(w2[0] - 1) < 1e-6   # FP32 node rounding
        assert i2[1] == 0 and w2[1] < 1e-6


def test_interp_exact_at_nodes(oracle, small):
    spec, T = small
    xs = [oracle.nodes(spec, a)[0] for a in range(5)]
    rng = np.random.default_rng(1)
    nH, nB, nN, nT, nC = spec.n
    ls = T["ls"].reshape(nH, nB, nN, nT)
    for _ in range(200):
        h, b, n, t = (rng.integers(0, k) for k in (nH, nB, nN, nT))
        v = oracle.interp_syn(spec, T, xs[0][h], xs[1][b], xs[2][n], xs[3][t])
        assert abs(v - ls[h, b, n, t]) <= 1e-13 * max(1.0, abs(v))
        vb = oracle.interp_brems(spec, T, xs[3][t])
        assert abs(vb - T["lb"][t]) <= 1e-13 * abs(vb)
    for i in range(nC):
        for e in range(nC):
            v = oracle.interp_coulomb(spec, T, xs[4][i], xs[4][e])
            assert abs(v - T["lc"][i, e]) <= 1e-13 * abs(v)


def test_interp_exact_on_log_affine_table(oracle):
    """A table whose log2 values are affine in the log2 coordinates is
    reproduced exactly everywhere inside the grid (pins index and weights)."""
    spec = oracle.Spec(n=(5, 6, 7, 9, 11))
    ls_axes = [oracle.nodes(spec, a)[1] for a in range(5)]
    c = [0.7, -1.3, 0.25, 2.0]
    g = np.meshgrid(*ls_axes[:4], indexing="ij")
    ls = (3.0 + sum(ci * gi for ci, gi in zip(c, g))).reshape(-1)
    lb = 1.5 - 0.5 * ls_axes[3]
    li, le = np.meshgrid(ls_axes[4], ls_axes[4], indexing="ij")
    lc = -2.0 + 0.3 * li - 0.9 * le
    T = dict(ls=np.ascontiguousarray(ls), lb=lb, lc=lc)
    rng = np.random.default_rng(2)
    for _ in range(300):
        p = [math.exp(rng.uniform(math.log(spec.lo[a]), math.log(spec.hi[a]))) for a in range(5)]
        lp = [math.log2(x) for x in p]
        want = 3.0 + sum(ci * li_ for ci, li_ in zip(c, lp[:4]))
        assert abs(oracle.interp_syn(spec, T, *p[:4]) - want) < 1e-11
        assert abs(oracle.interp_brems(spec, T, p[3]) - (1.5 - 0.5 * lp[3])) < 1e-11
        assert abs(oracle.interp_coulomb(spec, T, p[4], p[3]) - (-2.0 + 0.3 * lp[4] - 0.9 * lp[3])) < 1e-11
    # outside the grid: constant extrapolation (clamped weights)
    v_out = oracle.interp_brems(spec, T, spec.hi[3] * 10)
    v_edge = oracle.interp_brems(spec, T, spec.hi[3])
    assert abs(v_out - v_edge) < 1e-12


def test_table_nodes_equal_direct_formulas(oracle, small):
    spec, T = small
    xs = [oracle.nodes(spec, a)[0] for a in range(5)]
    nH, nB, nN, nT, nC = spec.n
    ls = T["ls"].reshape(nH, nB, nN, nT)
    rng = np.random.default_rng(3)
    for _ in range(20):
        h, b, n, t = (int(rng.integers(0, k)) for k in (nH, nB, nN, nT))
        want = math.log2(oracle.eta_qsyn(xs[0][h], xs[1][b], xs[2][n], xs[3][t], spec))
        assert ls[h, b, n, t] == want
    for t in range(nT):
        assert T["lb"][t] == math.log2(oracle.brems(xs[3][t]))
    assert T["lc"][3, 5] == math.log2(oracle.coulomb_C(xs[4][3], xs[4][5], spec))


def test_interp_converges_second_order(oracle):
    """O2 -> O1 at off-node points as the grid is refined (nested grids on a
    narrow box away from the K2 switch): error ratio ~4 per halving."""
    lo = (1e6, 1e3, 1e14, 2e9, 1e6)
    hi = (1e7, 1e4, 1e15, 2e10, 1e9)
    rng = np.random.default_rng(4)
    pts = [[math.exp(rng.uniform(math.log(lo[a]), math.log(hi[a]))) for a in range(4)] for _ in range(40)]
    errs = []
    for N in (5, 9, 17):
        spec = oracle.Spec(n=(N, N, N, N, N), lo=lo, hi=hi)
        T = oracle.build_tables(spec, nthreads=8)
        errs.append(np.array([abs(oracle.interp_syn(spec, T, *p) - math.log2(oracle.eta_qsyn(*p, spec)))
                              for p in pts]))
    r1 = np.median(errs[0] / errs[1])
    r2 = np.median(errs[1] / errs[2])
    assert r1 > 2.8 and r2 > 2.8, (r1, r2)   # first order would give ~2
    assert errs[2].max() < 0.25 * errs[0].max()


# ---- step ----------------------------------------------------------------------

def _const_tables(spec, ls=-2000.0, lb=-2000.0, lc=-2000.0):
    nH, nB, nN, nT, nC = spec.n
    return dict(ls=np.full(nH * nB * nN * nT, float(ls)), lb=np.full(nT, float(lb)),
                lc=np.full((nC, nC), float(lc)))


def _units(p):
    G, MSUN = 6.6743e-8, 1.98847e33
    rg = G * (p.M_bh_msun * MSUN) / C_LIGHT ** 2
    tg = rg / C_LIGHT
    return dict(rg=rg, tg=tg, hs=p.dt * tg / p.n_sub, escale=p.rho_scale * C_LIGHT ** 2,
                sT=(p.gamma_e - 1) * M_P * C_LIGHT ** 2 / K_B)


def test_exchange_conserves_energy(oracle, small):
    spec, T = small
    Tx = dict(T)
    Tx["ls"] = np.full_like(T["ls"], -2000.0)
    Tx["lb"] = np.full_like(T["lb"], -2000.0)
    f = inputs.uniform(4096, seed=11)
    p = oracle.Params(n_sub=8)
    ue, ui, qc, qx, cnt = oracle.step(spec, Tx, p, **f)
    tot0 = f["ue"] + f["ui"]
    assert np.all(np.abs((ue + ui) / tot0 - 1) <= 2 * p.n_sub * 2.0 ** -53)   # rounding of 2 adds per sub-cycle
    assert np.all(qc == 0.0)
    assert np.allclose(ue, f["ue"] + qx, rtol=1e-15)
    assert np.allclose(ui, f["ui"] - qx, rtol=1e-15)
    # energy flows from the hotter to the colder species, never past T_e = T_i
    Te0, Ti0 = f["ue"] / f["rho"], f["ui"] / f["rho"]
    Te1, Ti1 = ue / f["rho"], ui / f["rho"]
    assert np.all(np.sign(Ti1 - Te1) * np.sign(Ti0 - Te0) >= 0)
    assert np.all(np.sign(qx) == np.sign(Ti0 - Te0))


def test_strong_coupling_reaches_equilibrium(oracle):
    spec = oracle.Spec(n=(4, 4, 4, 4, 4))
    T = _const_tables(spec, lc=200.0)
    f = inputs.uniform(512, seed=12)
    p = oracle.Params(n_sub=1, gamma_i=1.4)
    ue, ui, _, _, _ = oracle.step(spec, T, p, **f)
    # (gamma_e - 1) u_e = (gamma_i - 1) u_i after the clamped exchange
    assert np.allclose((p.gamma_e - 1) * ue, (p.gamma_i - 1) * ui, rtol=1e-13)


def test_coulomb_single_subcycle_closed_form(oracle):
    spec = oracle.Spec(n=(4, 4, 4, 4, 4))
    lc = -110.0
    T = _const_tables(spec, lc=lc)
    f = inputs.uniform(512, seed=13)
    p = oracle.Params(n_sub=1)
    u = _units(p)
    ue, ui, _, qx, _ = oracle.step(spec, T, p, **f)
    ne = f["rho"] * p.rho_scale / M_P
    Te = u["sT"] * f["ue"] / f["rho"]
    Ti = u["sT"] * f["ui"] / f["rho"]
    X = u["hs"] * ne * ne * 2.0 ** lc * (Ti - Te) / u["escale"]
    Xeq = (f["ui"] - f["ue"]) / 2
    X = np.where(np.abs(X) > np.abs(Xeq), Xeq, X)
    assert np.allclose(qx, X, rtol=1e-13, atol=0)


def test_explicit_cooling_recurrence_and_limiter(oracle):
    """Constant thin rate Q: each sub-cycle removes min(h Q_tot(T)/e, 0.3 u)
    with the bridge of Eq. 11; with a huge rate in an optically thin cell
    the limiter gives u (0.7)^N exactly."""
    spec = oracle.Spec(n=(4, 4, 4, 4, 4))
    f = inputs.uniform(256, seed=14)
    for ls in (60.0, 90.0, 120.0):
        T = _const_tables(spec, ls=ls)
        p = oracle.Params(n_sub=6)
        u = _units(p)
        ue, _, qc, _, _ = oracle.step(spec, T, p, **f)
        ne = f["rho"] * p.rho_scale / M_P
        want = f["ue"].copy()
        for k in range(p.n_sub):
            for i in range(want.size):
                Te = u["sT"] * want[i] / f["rho"][i]
                q = u["hs"] * oracle.bridge(2.0 ** ls, Te, f["H"][i] * u["rg"], ne[i]) / u["escale"]
                want[i] -= min(q, 0.3 * want[i])
        assert np.allclose(ue, want, rtol=1e-13)
        assert np.allclose(qc, f["ue"] - ue, rtol=1e-12)
    # limiter: optically thin cell (tiny H, tiny density) with a huge rate
    g = dict(rho=np.array([1e-4]), B=np.array([1e-3]), H=np.array([1e-3]),
             ue=np.array([1e-5]), ui=np.array([1e-5]))
    T = _const_tables(spec, ls=80.0)
    ue, _, _, _, _ = oracle.step(spec, T, oracle.Params(n_sub=5), **g)
    assert ue[0] == pytest.approx(1e-5 * 0.7 ** 5, rel=1e-14)


def test_implicit_residual(oracle, small):
    spec, T = small
    f = inputs.uniform(4096, seed=15)
    p = oracle.Params(n_sub=1, mode=1)
    ue, ui, qc, qx, cnt = oracle.step(spec, T, p, **f)
    assert cnt["stiff"] > 50
    q0 = np.array([oracle.cool_q_cell(spec, T, p, f["rho"][i], f["B"][i], f["H"][i],
                                      f["ue"][i] + qx[i]) for i in range(f["rho"].size)])
    u_pre = f["ue"] + qx
    stiff = q0 > 0.3 * u_pre
    assert stiff.sum() == cnt["stiff"]
    checked = 0
    for i in np.flatnonzero(stiff)[:200]:
        qn = oracle.cool_q_cell(spec, T, p, f["rho"][i], f["B"][i], f["H"][i], ue[i])
        # backward Euler: u' = u - q(u'), to the bisection's resolution
        assert abs(ue[i] + qn - u_pre[i]) <= 1e-9 * u_pre[i]
        checked += 1
    assert checked > 50
    # non-stiff cells take the same explicit step as mode 0
    ue0, _, _, _, _ = oracle.step(spec, T, oracle.Params(n_sub=1, mode=0), **f)
    assert np.array_equal(ue[~stiff], ue0[~stiff])


def test_invalid_cells_pass_through(oracle, small):
    spec, T = small
    f = inputs.uniform(8, seed=16)
    f["rho"][0] = np.nan
    f["ue"][1] = -1.0
    f["ui"][2] = np.inf
    f["rho"][3] = 0.0
    f["B"][4] = -1.0
    ue, ui, qc, qx, cnt = oracle.step(spec, T, oracle.Params(), **f)
    assert cnt["invalid"] == 5
    for i in range(5):
        assert (ue[i] == f["ue"][i] or (np.isnan(ue[i]) and np.isnan(f["ue"][i])))
        assert (ui[i] == f["ui"][i] or (np.isnan(ui[i]) and np.isnan(f["ui"][i])))
        assert qc[i] == 0 and qx[i] == 0


def test_keys_f32_sequence(oracle):
    """FP32 keys: fixed IEEE op sequence, replayed here with numpy float32
    arithmetic; T = 7.2588e12 K x u/rho for gamma = 5/3 (m_p c^2/k = 1.0888e13 K)."""
    f = inputs.uniform(1000, seed=17, dtype=np.float32)
    p = oracle.Params()
    k = oracle.keys_f32(p, **f)
    sT = np.float32((p.gamma_e - 1) * M_P * C_LIGHT ** 2 / K_B)
    assert abs(float(sT) / 7.2588e12 - 1) < 1e-4
    inv = (sT / f["rho"]).astype(np.float32)
    assert np.array_equal(k[:, 3], (f["ue"] * inv).astype(np.float32))
    s_n = np.float32(p.rho_scale / M_P)
    assert np.array_equal(k[:, 2], (f["rho"] * s_n).astype(np.float32))
    s_B = np.float32(math.sqrt(4 * math.pi * p.rho_scale) * C_LIGHT)
    assert np.array_equal(k[:, 1], (f["B"] * s_B).astype(np.float32))


# ---- reduced-precision storage mirror (oracle.quant) -----------------------------

def test_quant_roundings_match_torch():
    """bf16 / f16 codes are round-to-nearest-even of the FP32 value: checked
    against torch's CPU conversions (an independent implementation)."""
    import torch
    from oracle import quant
    rng = np.random.default_rng(40)
    x = np.concatenate([rng.uniform(-200, 200, 100000), rng.uniform(-1, 1, 100000)]).astype(np.float32)
    tb = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16).astype(np.uint32)
    assert np.array_equal(quant.bf16_bits(x), tb)
    th = torch.from_numpy(x).to(torch.float16).view(torch.int16).numpy().view(np.uint16).astype(np.uint32)
    assert np.array_equal(quant.f16_bits(x), th)


def test_quant_pack_layout_and_error(oracle):
    from oracle import quant
    rng = np.random.default_rng(41)
    nT = 40
    ls = np.cumsum(rng.normal(0, 1.0, (30, nT)), axis=1) - 80.0
    for fmt in range(5):
        words, pairs = quant.pack(ls, nT, fmt)
        W, S = quant.WS[fmt]
        assert words.shape == (30, (nT - 1 + S - 1) // S, 8)
        # pairs reproduce the exact values within the format's resolution
        exact = np.stack([ls[:, :-1], ls[:, 1:]], axis=2)
        err = np.abs(pairs - exact).max()
        bound = {0: 2 ** -24 * 128, 1: 2 ** -8 * 128, 2: 2 ** -11 * 128, 3: None, 4: None}[fmt]
        if bound is not None:
            assert err <= bound
        else:
            half = 0.5 * (ls.max() - ls.min())
            assert err <= (2 ** -8 if fmt == 3 else 2 ** -11) * half
        if fmt in (0, 1, 2):
            # plain formats: the pair values do not depend on the block
            assert np.array_equal(pairs[:, 1:, 0], pairs[:, :-1, 1])
    # block scaling is more accurate than plain 16-bit storage of large log2 values
    assert quant.storage_error(ls, nT, 3) < quant.storage_error(ls, nT, 1)
    assert quant.storage_error(ls, nT, 4) < quant.storage_error(ls, nT, 2)


def test_step_pairs_equals_step_for_exact_pairs(oracle, small):
    """The paired-table step with exact (unrounded) pairs equals the step."""
    spec, T = small
    nT = spec.n[3]
    ls = T["ls"].reshape(-1, nT)
    pairs = np.stack([ls[:, :-1], ls[:, 1:]], axis=2)
    f = inputs.uniform(2000, seed=42)
    p = oracle.Params(n_sub=4)
    a = oracle.step(spec, T, p, **f)
    b = oracle.step_pairs(spec, T["lb"], pairs, T["lc"], p, **f)
    assert np.allclose(a[0], b[0], rtol=1e-14) and np.allclose(a[1], b[1], rtol=1e-14)
