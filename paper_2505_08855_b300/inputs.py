"""Seeded synthetic cell fields ("MAD-like" accretion-flow cells).

Shared by the tests, the benchmark and the oracle's callers.  This module
holds no cooling arithmetic: it only draws code-unit fields (G = c = M = 1,
the 4 pi absorbed in b, as in the paper's Sec. 3.2) from the recipes below,
which stand in for H-AMR snapshot data (the paper's simulations, Sec. 3.3,
are not available).

Fields, all code units, structure of arrays:
    rho  rest-mass density (the paper's rho_scale maps rho = 1 to g cm^-3)
    B    magnetic-field magnitude |b|
    H    thermal scale height, in r_g
    ue   electron internal energy density
    ui   ion internal energy density
    r    radius in r_g (only with ``with_r=True``: the disk-geometry step)

Recipes (seed fixed per workload):
  * ``uniform``  -- rho ~ logU[1e-4, 1]; u_i/rho, u_e/rho ~ logU[1e-6, 1e-1]
    independently; plasma beta ~ logU[0.1, 100] with
    |b| = sqrt(2 (gamma-1)(u_i + u_e) / beta); H/r ~ U[0.05, 0.5] and
    r ~ logU[2, 1000] r_g, H = (H/r) r.
  * ``two_region`` -- as ``uniform`` on a 3-D grid split by a smooth seeded
    mask (sum of 8 random periodic sinusoids > 0) into a cold-thin region
    (u_i/rho, u_e/rho ~ logU[1e-6, 1e-5], rho x 10: T ~ 1e7 K) and a
    hot-thick region (u_e/rho ~ logU[3e-4, 3e-3]: T_e ~ 2e9-2e10 K,
    T_i/T_e ~ logU[1, 100]).
  * ``shell`` -- spherical-like shell on an (r, theta, phi) grid: r
    log-spaced on [2, 1000] r_g, theta in (0, pi), phi uniform;
    rho = (r/2)^-1.5 exp(0.1 N(0,1)); u_i/rho = (0.1/r) exp(0.1 N(0,1));
    T_i/T_e = 1 for r > 50 r_g rising log-linearly to 30 at r = 2 r_g;
    H/r from 0.35 at r = 2 to 0.1 at r = 1000 (log-linear) x exp(0.05 N);
    beta ~ logU[0.1, 100].
"""
import numpy as np

GAMMA = 5.0 / 3.0


def _logu(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def _b_from_beta(ue, ui, beta, gamma=GAMMA):
    return np.sqrt(2.0 * (gamma - 1.0) * (ui + ue) / beta)


def _out(d, r, with_r, dtype):
    if with_r:
        d = dict(d, r=r)
    return {k: np.ascontiguousarray(v.astype(dtype)) for k, v in d.items()}


def uniform(n, seed=1001, dtype=np.float64, with_r=False):
    rng = np.random.default_rng(seed)
    rho = _logu(rng, 1e-4, 1.0, n)
    ui = rho * _logu(rng, 1e-6, 1e-1, n)
    ue = rho * _logu(rng, 1e-6, 1e-1, n)
    beta = _logu(rng, 0.1, 100.0, n)
    B = _b_from_beta(ue, ui, beta)
    r = _logu(rng, 2.0, 1000.0, n)
    H = rng.uniform(0.05, 0.5, n) * r
    return _out(dict(rho=rho, B=B, H=H, ue=ue, ui=ui), r, with_r, dtype)


def _mask(shape, rng):
    """Smooth periodic mask: sum of 8 sinusoids with small integer wave
    vectors; True where positive.  Evaluated plane by plane (low memory)."""
    nx, ny, nz = shape
    ks = rng.integers(1, 4, size=(8, 3)) * rng.choice([-1, 1], size=(8, 3))
    ph = rng.uniform(0, 2 * np.pi, 8)
    amp = rng.uniform(0.5, 1.0, 8)
    y = np.arange(ny)[:, None] * (2 * np.pi / ny)
    z = np.arange(nz)[None, :] * (2 * np.pi / nz)
    out = np.empty(shape, bool)
    for i in range(nx):
        x = i * (2 * np.pi / nx)
        acc = np.zeros((ny, nz))
        for k in range(8):
            acc += amp[k] * np.sin(ks[k, 0] * x + ks[k, 1] * y + ks[k, 2] * z + ph[k])
        out[i] = acc > 0
    return out.reshape(-1)


def two_region(shape=(256, 256, 256), seed=1002, dtype=np.float32, with_r=False):
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed)
    hot = _mask(shape, rng)
    base = uniform(n, seed=seed + 7, dtype=np.float64, with_r=True)
    rho = base["rho"]
    nh = int(hot.sum())
    nc = n - nh
    # cold-thin region
    rho_c = rho[~hot] * 10.0
    ui_c = rho_c * _logu(rng, 1e-6, 1e-5, nc)
    ue_c = rho_c * _logu(rng, 1e-6, 1e-5, nc)
    # hot-thick region
    rho_h = rho[hot]
    ue_h = rho_h * _logu(rng, 3e-4, 3e-3, nh)
    ui_h = ue_h * _logu(rng, 1.0, 100.0, nh)
    rho = rho.copy()
    ue = np.empty(n)
    ui = np.empty(n)
    rho[~hot] = rho_c
    ue[~hot], ui[~hot] = ue_c, ui_c
    ue[hot], ui[hot] = ue_h, ui_h
    beta = _logu(rng, 0.1, 100.0, n)
    B = _b_from_beta(ue, ui, beta)
    out = dict(rho=rho, B=B, H=base["H"], ue=ue, ui=ui)
    return _out(out, base["r"], with_r, dtype)


def shell(shape=(448, 192, 192), seed=1004, dtype=np.float32, with_r=False):
    nr, nth, nph = shape
    n = nr * nth * nph
    rng = np.random.default_rng(seed)
    r1 = np.exp(np.linspace(np.log(2.0), np.log(1000.0), nr))
    r = np.repeat(r1, nth * nph)
    rho = (r / 2.0) ** -1.5 * np.exp(0.1 * rng.standard_normal(n))
    ui = rho * (0.1 / r) * np.exp(0.1 * rng.standard_normal(n))
    # T_i/T_e: 1 beyond 50 r_g, log-linear up to 30 at 2 r_g
    f = np.clip((np.log(50.0) - np.log(r)) / (np.log(50.0) - np.log(2.0)), 0.0, 1.0)
    tratio = np.exp(f * np.log(30.0))
    ue = ui / tratio
    hr = np.exp(np.log(0.35) + (np.log(0.1) - np.log(0.35))
                * (np.log(r) - np.log(2.0)) / (np.log(1000.0) - np.log(2.0)))
    H = hr * r * np.exp(0.05 * rng.standard_normal(n))
    beta = _logu(rng, 0.1, 100.0, n)
    B = _b_from_beta(ue, ui, beta)
    out = dict(rho=rho, B=B, H=H, ue=ue, ui=ui)
    return _out(out, r, with_r, dtype)


# The workloads by name: (recipe, keyword arguments).
WORKLOADS = {
    "uniform_32c": (uniform, dict(n=32 ** 3, seed=1001)),
    "two_region_256c": (two_region, dict(shape=(256, 256, 256), seed=1002)),
    "uniform_128c": (uniform, dict(n=128 ** 3, seed=1003, dtype=np.float32)),
    "shell_448x192x192": (shell, dict(shape=(448, 192, 192), seed=1004)),
    "shell_512x256x256": (shell, dict(shape=(512, 256, 256), seed=1005)),
}


def make(name, **over):
    fn, kw = WORKLOADS[name]
    kw = dict(kw)
    kw.update(over)
    return fn(**kw)


def subsample(fields, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in fields.items()}
