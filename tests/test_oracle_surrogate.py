"""Pins of the oracle's surrogate step (no GPU): the step of Sec. 3.2 with
the 4-D synchrotron channel read from the surrogate network, except in table
cells whose fallback bit is set.

* The C network equals the numpy network of oracle.mlp (itself pinned by
  finite differences) with and without the bf16 operand roundings.
* With every bit set it is the table step, bit for bit.
* A network that outputs a constant c is the table step on a table whose
  4-D channel is c everywhere (multilinear interpolation of a constant).
* With one sub-cycle each cell reads exactly one table cell: under a mask
  that mixes all four indices, every cell equals the table step when its
  cell's bit is set and the network step otherwise; the counter counts the
  former.
"""
import numpy as np
import pytest

from paper_2505_08855_b300 import inputs

N5 = (6, 7, 6, 10, 8)


@pytest.fixture(scope="module")
def env(oracle):
    spec = oracle.Spec(n=N5)
    tab = oracle.build_tables(spec, nthreads=8)
    f = inputs.make("uniform_32c")
    f = inputs.subsample(f, np.arange(0, 32 ** 3, 23))
    return spec, tab, f


def _params(seed, scale=1.0):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    p = np.zeros(mlp.P_N, np.float32)
    W1 = rng.uniform(-1, 1, (128, 16)) * np.sqrt(6 / 5) * scale
    W1[:, 5:] = 0
    p[mlp.P_W1:mlp.P_b1] = W1.reshape(-1)
    p[mlp.P_b1:mlp.P_W2] = rng.normal(0, 0.1, 128)
    p[mlp.P_W2:mlp.P_b2] = rng.uniform(-1, 1, 128 * 128) * np.sqrt(6 / 128)
    p[mlp.P_b2:mlp.P_w3] = rng.normal(0, 0.1, 128)
    p[mlp.P_w3:mlp.P_b3] = rng.normal(0, 0.3, 128)
    p[mlp.P_b3] = 0.2
    return p


def _fields(f):
    return [f[k] for k in ("rho", "B", "H", "ue", "ui")]


def test_c_network_equals_numpy(oracle):
    from oracle import mlp
    p = _params(1)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (3000, 4)).astype(np.float32).astype(np.float64)
    xs = -0.2
    for rounding in (False, True):
        got = oracle.net_eval(p, -40.0, 25.0, xs, x, rounding=rounding)
        want = -40.0 + 25.0 * mlp.forward(p.astype(np.float64), x, xs, rounding=rounding)
        err = np.abs(got - want)
        if not rounding:
            assert err.max() <= 1e-11 * 25.0
        else:
            # a hidden activation within a rounding error of a bf16 tie may
            # round the other way in the two summation orders
            assert np.quantile(err, 0.999) <= 1e-11 * 25.0
            assert err.max() <= 1e-2 * 25.0


def test_all_bits_set_is_the_table_step(oracle, env):
    spec, tab, f = env
    prm = oracle.Params(n_sub=4)
    cells = (N5[0] - 1) * (N5[1] - 1) * (N5[2] - 1) * (N5[3] - 1)
    mask = np.full((cells + 31) // 32, 0xFFFFFFFF, np.uint32)
    got = oracle.step_surrogate(spec, tab, _params(3), 0.0, 1.0, mask, prm, *_fields(f))
    want = oracle.step(spec, tab, prm, *_fields(f))
    for a, b in zip(got[:4], want[:4]):
        assert np.array_equal(a, b)
    valid = f["rho"].size - want[4]["invalid"]
    assert got[4]["fallback"] == valid
    assert want[4]["fallback"] == 0


def test_constant_network_is_a_constant_table(oracle, env):
    from oracle import mlp
    spec, tab, f = env
    prm = oracle.Params(n_sub=4)
    p = np.zeros(mlp.P_N, np.float32)
    p[mlp.P_b3] = 0.75
    mean, std = -60.0, 8.0
    got = oracle.step_surrogate(spec, tab, p, mean, std, None, prm, *_fields(f))
    flat = dict(tab)
    flat["ls"] = np.full_like(tab["ls"], mean + std * 0.75)
    want = oracle.step(spec, flat, prm, *_fields(f))
    for a, b in zip(got[:4], want[:4]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)
    assert got[4]["fallback"] == 0
    # the constant is in the regime where it matters: cooling is not limited
    # everywhere and not negligible everywhere
    q = want[2] / f["ue"]
    assert np.mean(q > 1e-6) > 0.05 and np.mean(q < 0.3 * 4 * 0.99) > 0.05


def test_mixed_mask_selects_per_table_cell(oracle, env):
    spec, tab, f = env
    prm = oracle.Params(n_sub=1)
    p = _params(4)
    mean, std = -50.0, 20.0
    nH, nB, nN, nT = (k - 1 for k in N5[:4])
    h, b, n, t = np.meshgrid(np.arange(nH), np.arange(nB), np.arange(nN), np.arange(nT), indexing="ij")
    flag = ((h + 2 * b + 3 * n + t) % 3 == 0).reshape(-1)
    cells = flag.size
    bits = np.zeros((cells + 31) // 32, np.uint32)
    for c in np.flatnonzero(flag):
        bits[c >> 5] |= np.uint32(1 << (c & 31))
    fl = _fields(f)
    mixed = oracle.step_surrogate(spec, tab, p, mean, std, bits, prm, *fl)
    net = oracle.step_surrogate(spec, tab, p, mean, std, None, prm, *fl)
    table = oracle.step(spec, tab, prm, *fl)
    # the table cell each cell reads: H, B, n_e from the input keys, T_e
    # after the Coulomb exchange (ue + q_cc)
    ue1 = f["ue"] + table[3]
    ui1 = f["ui"] - table[3]
    keys = oracle.keys_f32(prm, f["rho"], f["B"], f["H"], ue1, ui1).astype(np.float64)
    j = [oracle.select_f32(spec, a, keys[:, a].astype(np.float32))[0] for a in range(4)]
    cell = ((j[0] * nB + j[1]) * nN + j[2]) * nT + j[3]
    want_table = flag[cell]
    # skip keys within FP32 rounding of a T_e node (the oracle selects on
    # the FP64 key, keys_f32 gives its FP32 rounding)
    x32 = oracle.nodes(spec, 3)[2].astype(np.float64)
    near = np.min(np.abs(keys[:, 3:4] / x32[None, :] - 1.0), axis=1) < 1e-6
    ok = ~near & np.isfinite(keys).all(axis=1) & (f["rho"] > 0)
    assert ok.sum() > 0.9 * ok.size
    for k in range(4):
        exp = np.where(want_table, table[k], net[k])
        assert np.array_equal(mixed[k][ok], exp[ok]), k
    assert want_table[ok].any() and (~want_table[ok]).any()
    valid = np.isfinite(keys).all(axis=1) & (f["rho"] > 0)
    assert abs(mixed[4]["fallback"] - int(want_table[valid].sum())) <= int((near & valid).sum())
