"""Pins of the oracle's adjoint (no GPU): central finite differences.

Kink-aware: a cell is skipped when a perturbation changes any discrete
decision (table cell, clamp, limiter branch, stiff branch), detected by the
hash the oracle returns; the skip count is printed and bounded.  The implicit
branch's gradient comes from the implicit-function theorem, so agreement with
FD of the bisection result also pins that reading.
"""
import numpy as np
import pytest

from paper_2505_08855_b300 import inputs

EPS = 1e-3


@pytest.fixture(scope="module")
def tab(oracle):
    spec = oracle.Spec(n=(16, 16, 16, 24, 24))
    return spec, oracle.build_tables(spec, nthreads=8)


def _loss(oracle, spec, T, p, f, a, b, i, k, scale):
    g = {kk: v.copy() for kk, v in f.items()}
    name = ["rho", "B", "H", "ue", "ui"][k]
    g[name][i] = g[name][i] * scale
    r = oracle.step_bwd(spec, T, p, **g, g_ue=a, g_ui=b)
    return a * r["ue"] + b * r["ui"], r["sig"]


@pytest.mark.parametrize("mode", [0, 1])
def test_adjoint_matches_central_fd(oracle, tab, mode):
    spec, T = tab
    n = 1024
    f = inputs.make("uniform_128c", dtype=np.float64)
    rng = np.random.default_rng(1003)
    idx = rng.choice(f["rho"].size, n, replace=False)
    f = inputs.subsample(f, idx)
    a = rng.uniform(0.5, 1.5, n)
    b = rng.uniform(-1.0, 1.0, n)
    p = oracle.Params(n_sub=8, mode=mode)
    base = oracle.step_bwd(spec, T, p, **f, g_ue=a, g_ui=b)
    names = ["g_rho", "g_B", "g_H", "g_ue", "g_ui"]
    fields = ["rho", "B", "H", "ue", "ui"]
    checked = skipped = 0
    worst = 0.0
    for k in range(5):
        fds = []
        ok = np.ones(n, bool)
        for eps in (EPS, EPS / 2):
            gp = {kk: v.copy() for kk, v in f.items()}
            gm = {kk: v.copy() for kk, v in f.items()}
            gp[fields[k]] *= 1 + eps
            gm[fields[k]] *= 1 - eps
            rp = oracle.step_bwd(spec, T, p, **gp, g_ue=a, g_ui=b)
            rm = oracle.step_bwd(spec, T, p, **gm, g_ue=a, g_ui=b)
            ok &= (rp["sig"] == base["sig"]) & (rm["sig"] == base["sig"])
            fds.append((a * rp["ue"] + b * rp["ui"] - a * rm["ue"] - b * rm["ui"]) / (2 * eps * f[fields[k]]))
        # central differences at eps and eps/2 combined (Richardson): O(eps^4)
        fd = (4 * fds[1] - fds[0]) / 3
        g = base[names[k]]
        L0 = a * base["ue"] + b * base["ui"]
        # compare the change of L: |fd - g| x / |L|, a scale-free measure
        err = np.abs(fd - g) * np.abs(f[fields[k]]) / np.maximum(np.abs(L0), 1e-300)
        checked += ok.sum()
        skipped += (~ok).sum()
        worst = max(worst, err[ok].max())
        assert np.all(err[ok] < 1e-6), (fields[k], err[ok].max())
    print(f"\nmode {mode}: checked {checked}, skipped {skipped} (kinks), worst {worst:.2e}")
    assert skipped < 0.25 * (checked + skipped)


def test_adjoint_table_entries_fd(oracle, tab):
    spec, T = tab
    n = 512
    f = inputs.uniform(n, seed=1004)
    rng = np.random.default_rng(5)
    a = rng.uniform(0.5, 1.5, n)
    b = rng.uniform(-1.0, 1.0, n)
    p = oracle.Params(n_sub=8)
    base = oracle.step_bwd(spec, T, p, **f, g_ue=a, g_ui=b, table_grads=True)
    delta = 1e-3
    for key, gkey in (("ls", "g_ls"), ("lb", "g_lb"), ("lc", "g_lc")):
        g = base[gkey].reshape(-1)
        for e in np.argsort(-np.abs(g))[:3]:
            vals = []
            sigs = []
            for sgn in (1, -1):
                T2 = {kk: v.copy() for kk, v in T.items()}
                flat = T2[key].reshape(-1)
                flat[e] += sgn * delta
                r = oracle.step_bwd(spec, T2, p, **f, g_ue=a, g_ui=b)
                vals.append(a * r["ue"] + b * r["ui"])
                sigs.append(r["sig"])
            ok = (sigs[0] == base["sig"]) & (sigs[1] == base["sig"])
            fd = ((vals[0] - vals[1])[ok]).sum() / (2 * delta)
            sub = inputs.subsample(f, np.flatnonzero(ok))
            g_ok = oracle.step_bwd(spec, T, p, **sub, g_ue=a[ok], g_ui=b[ok], table_grads=True)[gkey].reshape(-1)[e]
            assert abs(fd - g_ok) <= 1e-4 * max(abs(g_ok), 1e-30) + 1e-12, (key, e, fd, g_ok)


def test_mlp_reference_gradient_fd():
    """The numpy network's reverse-mode gradient (without the bf16 operand
    roundings) against central differences of its own loss."""
    from oracle import mlp
    rng = np.random.default_rng(9)
    p = np.zeros(mlp.P_N)
    W1 = rng.uniform(-1, 1, (128, 16)) * np.sqrt(6 / 5)
    W1[:, 5:] = 0
    p[mlp.P_W1:mlp.P_b1] = W1.reshape(-1)
    p[mlp.P_b1:mlp.P_W2] = rng.normal(0, 0.1, 128)
    p[mlp.P_W2:mlp.P_b2] = rng.uniform(-1, 1, 128 * 128) * np.sqrt(6 / 128)
    p[mlp.P_b2:mlp.P_w3] = rng.normal(0, 0.1, 128)
    p[mlp.P_w3:mlp.P_b3] = rng.normal(0, 0.1, 128)
    p[mlp.P_b3] = 0.3
    x = rng.uniform(-1, 1, (64, 4))
    y = rng.normal(0, 1, 64)
    xs = 0.1   # both sides of the switch occur among the points
    g, _ = mlp.grads(p, x, y, xs, rounding=False)
    assert np.all(g[mlp.P_W1:mlp.P_b1].reshape(128, 16)[:, 5:] == 0)
    idx = np.concatenate([rng.choice(np.flatnonzero(np.arange(mlp.P_b1) % 16 < 5), 8),
                          np.arange(4, mlp.P_b1, 16)[:3],
                          rng.integers(mlp.P_b1, mlp.P_N, 30), [mlp.P_b3]])
    h = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.grads(pp, x, y, xs, rounding=False)[1] - mlp.grads(pm, x, y, xs, rounding=False)[1]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_mlp_input_parts():
    """The two bf16 parts of each input carry 16 significant bits (|x - hi -
    lo| <= 2^-16 |x|, against 2^-8 |x| for hi alone), and the switch side is
    +1 strictly above xs and -1 at or below it."""
    from oracle import mlp
    rng = np.random.default_rng(10)
    x = rng.uniform(-1, 1, (4000, 4)).astype(np.float32).astype(np.float64)
    x[0, 3] = np.float32(0.25)
    X = mlp.features(x, 0.25)
    err = np.abs(x - X[:, :4] - X[:, 4:8])
    assert np.all(err <= 2.0 ** -16 * np.abs(x))
    assert np.max(np.abs(x - X[:, :4]) / np.abs(x)) > 2.0 ** -10
    assert np.array_equal(X[:, 8], np.where(x[:, 3] > 0.25, 1.0, -1.0))
    assert X[0, 8] == -1.0
