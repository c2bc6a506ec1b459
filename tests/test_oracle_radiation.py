"""Pins of the oracle's radiation-pressure correction (Sec. 5.2): the
closed-form root of the total-pressure quartic a T^4 + n k T = n k T_e,sim.

* the closed form against numpy's companion-matrix roots (a library
  routine of its own) on moderate coefficients;
* the residual relative to the largest term over 60 decades of each
  coefficient, and the two limits (radiation-dominated T -> (c/a)^(1/4),
  gas-dominated T -> c/b);
* per cell: thin cells keep T_e,sim, thick cells satisfy the pressure
  balance, and the corrected T_e never exceeds T_e,sim.
"""
import numpy as np

from paper_2505_08855_b300 import inputs


def test_quartic_matches_numpy_roots(oracle):
    rng = np.random.default_rng(1)
    for _ in range(300):
        a, b, c = np.exp(rng.uniform(-5, 5, 3))
        r = np.roots([a, 0.0, 0.0, b, -c])
        pos = r[(np.abs(r.imag) < 1e-9 * np.abs(r)) & (r.real > 0)].real
        assert pos.size == 1
        x = oracle.quartic_root(a, b, c)
        assert abs(x - pos[0]) <= 1e-12 * pos[0]


def test_quartic_residual_and_limits(oracle):
    rng = np.random.default_rng(2)
    for _ in range(3000):
        la, lb, lc = rng.uniform(-70, 70, 3)
        a, b, c = 10.0 ** la, 10.0 ** lb, 10.0 ** lc
        x = oracle.quartic_root(a, b, c)
        assert x > 0
        res = abs(a * x ** 4 + b * x - c) / max(a * x ** 4, b * x, c)
        assert res <= 1e-13, (a, b, c, x, res)
    a, c = 2.0, 3.0
    assert abs(oracle.quartic_root(a, 1e-30, c) / (c / a) ** 0.25 - 1) < 1e-14
    assert abs(oracle.quartic_root(1e-30, a, c) / (c / a) - 1) < 1e-14


def test_cells_thin_kept_thick_balanced(oracle):
    f = inputs.make("uniform_32c")
    p = oracle.Params()
    rho = f["rho"] * np.exp(np.random.default_rng(3).uniform(0, 25, f["rho"].size))   # reach thick cells
    te, thick = oracle.radiation_te(p, rho, f["H"], f["ue"] * rho / f["rho"], tau_crit=4.6)
    mp, c, kb = 1.67262192369e-24, 2.99792458e10, 1.380649e-16
    ne = rho * p.rho_scale / mp
    te_sim = (p.gamma_e - 1) * mp * c * c / kb * (f["ue"] * rho / f["rho"]) / rho
    assert thick.any() and (~thick).any()
    assert np.array_equal(te[~thick], te_sim[~thick])
    lhs = oracle.A_RAD * te[thick] ** 4 + ne[thick] * kb * te[thick]
    rhs = ne[thick] * kb * te_sim[thick]
    assert np.max(np.abs(lhs - rhs) / rhs) <= 1e-12
    assert np.all(te[thick] <= te_sim[thick])
