"""Pins of the oracle's disk-geometry step (Sec. 2.7 scale height H_th =
c_s/Omega_K, Sec. 3.2.3 temperature floor), no GPU.

* With the geometry switched off the disk step is the plain step, and with
  H_th from the state it is the plain step fed H_th per cell (bit for bit).
* The sound speed's relativistic enthalpy: c_s^2 -> gamma P / rho for a cold
  gas (P << rho) and -> gamma - 1 for an ultra-relativistic one (u >> rho),
  the textbook limits; Omega_K r -> r^-1/2 (Kepler) without spin.
* The floor: a cell whose gas temperature P/rho starts below T_floor is not
  cooled at all (q_cool = 0; only the energy-conserving exchange acts, so
  P/rho is unchanged with gamma_e = gamma_i); a cell starting above ends at
  or above (1 - limiter) T_floor; the counter counts floored cells.
"""
import numpy as np
import pytest

from paper_2505_08855_b300 import inputs

N5 = (8, 8, 8, 12, 12)


@pytest.fixture(scope="module")
def env(oracle):
    spec = oracle.Spec(n=N5)
    tab = oracle.build_tables(spec, nthreads=8)
    f = inputs.subsample(inputs.make("uniform_32c", with_r=True), np.arange(0, 32 ** 3, 11))
    return spec, tab, f


def _fl(f):
    return [f[k] for k in ("rho", "B", "H", "ue", "ui")]


def test_geometry_off_and_h_from_state_reduce_to_plain_step(oracle, env):
    spec, tab, f = env
    p = oracle.Params(n_sub=4)
    plain = oracle.step(spec, tab, p, *_fl(f))
    got = oracle.step_disk(spec, tab, p, *_fl(f), f["r"], spin=0.9375)
    for a, b in zip(got[:4], plain[:4]):
        assert np.array_equal(a, b)
    assert got[4]["floor"] == 0
    hth = np.array([oracle.h_thermal(p, *x, spin=0.9375) for x in zip(f["rho"], f["ue"], f["ui"], f["r"])])
    plain2 = oracle.step(spec, tab, p, f["rho"], f["B"], hth, f["ue"], f["ui"])
    got2 = oracle.step_disk(spec, tab, p, f["rho"], f["B"], None, f["ue"], f["ui"], f["r"], spin=0.9375,
                            h_from_state=True)
    for a, b in zip(got2[:4], plain2[:4]):
        assert np.array_equal(a, b)
    assert not np.array_equal(got2[0], plain[0])     # H_th differs from the H field


def test_sound_speed_and_kepler_limits(oracle):
    p = oracle.Params()
    g = 5.0 / 3.0
    r = 100.0
    # cold gas: c_s^2 -> gamma P / rho, P = (gamma - 1) u
    rho, ue, ui = 1.0, 1e-9, 2e-9
    cs2 = (oracle.h_thermal(p, rho, ue, ui, r) / r ** 1.5) ** 2
    assert abs(cs2 / (g * (g - 1) * (ue + ui) / rho) - 1) < 1e-8
    # ultra-relativistic gas: c_s^2 -> gamma - 1
    cs2 = (oracle.h_thermal(p, 1e-12, 1.0, 2.0, r) / r ** 1.5) ** 2
    assert abs(cs2 / (g - 1) - 1) < 1e-10
    # spin enters Omega_K = 1/(r^1.5 + a): H grows by (r^1.5 + a)/r^1.5
    h0 = oracle.h_thermal(p, 1.0, 1e-4, 1e-4, 4.0, 0.0)
    h1 = oracle.h_thermal(p, 1.0, 1e-4, 1e-4, 4.0, 0.9375)
    assert abs(h1 / h0 - (8.0 + 0.9375) / 8.0) < 1e-14


def test_temperature_floor(oracle, env):
    spec, tab, f = env
    p = oracle.Params(n_sub=8)
    hf = 0.05
    ue, ui, qc, qx, cnt = oracle.step_disk(spec, tab, p, *_fl(f), f["r"], h_floor=hf)
    g = 5.0 / 3.0
    theta0 = (g - 1) * (f["ue"] + f["ui"]) / f["rho"]
    theta1 = (g - 1) * (ue + ui) / f["rho"]
    tfl = 0.5 * np.pi * (hf * f["r"] / (f["r"] ** 1.5)) ** 2
    below = theta0 < tfl
    assert below.any() and (~below).any()
    assert np.all(qc[below] == 0.0)
    assert np.allclose(theta1[below], theta0[below], rtol=1e-14, atol=0)
    assert np.all(theta1[~below] >= (1 - p.limiter_frac) * tfl[~below] * (1 - 1e-12))
    assert cnt["floor"] >= below.sum()
    # some cells cross the floor during the step, and are then left alone
    crossed = ~below & (theta1 < tfl)
    assert crossed.any()
    plain = oracle.step(spec, tab, p, *_fl(f))
    never = ~below & (((g - 1) * (plain[0] + plain[1]) / f["rho"]) >= tfl)
    assert np.array_equal(ue[never], plain[0][never])
