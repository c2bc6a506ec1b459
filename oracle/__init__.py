"""FP64 CPU oracle of the two-temperature cooling step (arXiv 2505.08855).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this package.  The
product path (paper_2505_08855_b300) never imports it.  It shares no code
with the CUDA library; see cool_oracle.c for the formulas and the readings of
the paper it follows.

Python side: ctypes marshalling of numpy arrays only; every computation is
in cool_oracle.c.
"""
import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


class _Spec(C.Structure):
    _fields_ = [("n", C.c_int * 5), ("lo", C.c_double * 5), ("hi", C.c_double * 5),
                ("k2_switch_T", C.c_double), ("lnLambda", C.c_double),
                ("theta_i_uses_mp", C.c_int), ("compton_literal", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("rho_scale", C.c_double), ("M_bh_msun", C.c_double),
                ("gamma_e", C.c_double), ("gamma_i", C.c_double), ("dt", C.c_double),
                ("n_sub", C.c_int), ("mode", C.c_int),
                ("limiter_frac", C.c_double), ("eq_band", C.c_double),
                ("coulomb_clamp", C.c_double), ("implicit_iters", C.c_int)]


class _Disk(C.Structure):
    _fields_ = [("spin", C.c_double), ("h_floor", C.c_double), ("h_from_state", C.c_int)]


# Axis order: 0 H_th [cm], 1 |B| [G], 2 n_e [cm^-3], 3 T_e [K] (cooling),
# 4 T [K] (Coulomb, both T_i and T_e).  Ranges of Sec. 2.6 / 2.8.
PAPER_LO = (1e3, 1.0, 1e2, 1e2, 1e2)
PAPER_HI = (1e12, 1e10, 1e25, 1e15, 1e15)


@dataclasses.dataclass
class Spec:
    n: tuple = (32, 32, 32, 32, 32)
    lo: tuple = PAPER_LO
    hi: tuple = PAPER_HI
    k2_switch_T: float = 1e8
    lnLambda: float = 20.0
    theta_i_uses_mp: int = 1
    compton_literal: int = 0

    def c(self):
        return _Spec((C.c_int * 5)(*self.n), (C.c_double * 5)(*self.lo),
                     (C.c_double * 5)(*self.hi), self.k2_switch_T, self.lnLambda,
                     self.theta_i_uses_mp, self.compton_literal)


@dataclasses.dataclass
class Params:
    rho_scale: float = 3e-7
    M_bh_msun: float = 10.0
    gamma_e: float = 5.0 / 3.0
    gamma_i: float = 5.0 / 3.0
    dt: float = 1e-2
    n_sub: int = 4
    mode: int = 0
    limiter_frac: float = 0.3
    eq_band: float = 0.1
    coulomb_clamp: float = 1.0
    implicit_iters: int = 60

    def c(self):
        return _Params(self.rho_scale, self.M_bh_msun, self.gamma_e, self.gamma_i, self.dt,
                       self.n_sub, self.mode, self.limiter_frac, self.eq_band,
                       self.coulomb_clamp, self.implicit_iters)


_d, _i, _ll, _f = C.c_double, C.c_int, C.c_longlong, C.c_float
_P = C.c_void_p


def _declare(L):
    sig = {
        "orc_const": (_d, [_i]),
        "orc_kve": (_d, [_i, _d]),
        "orc_theta_e": (_d, [_d]),
        "orc_brems_ee": (_d, [_d]),
        "orc_brems_ei": (_d, [_d]),
        "orc_brems": (_d, [_d]),
        "orc_log_Iprime": (_d, [_d]),
        "orc_Iprime": (_d, [_d]),
        "orc_k2_factor": (_d, [_d, _d]),
        "orc_nu0": (_d, [_d, _d]),
        "orc_eps_syn": (_d, [_d, _d, _d, _d, _d]),
        "orc_nu_c": (_d, [_d, _d, _d, _d, _d, _P]),
        "orc_J": (_d, [_d, _i]),
        "orc_qsyn_nu": (_d, [_d, _d, _d, _d, _d, _d, _i]),
        "orc_eta": (_d, [_d, _d, _d, _d, _i]),
        "orc_eta_qsyn": (_d, [_d, _d, _d, _d, _P, _P]),
        "orc_bridge": (_d, [_d, _d, _d, _d]),
        "orc_qtotal_direct": (_d, [_d, _d, _d, _d, _P]),
        "orc_coulomb_C": (_d, [_d, _d, _P]),
        "orc_gl16": (None, [_P, _P]),
        "orc_nodes": (None, [_P, _i, _P, _P, _P]),
        "orc_build_brems": (None, [_P, _P]),
        "orc_syn_node": (_d, [_P, _i, _i, _i, _i]),
        "orc_build_syn": (None, [_P, _P, _i]),
        "orc_build_syn_at": (None, [_P, _ll, _P, _P, _i]),
        "orc_build_coulomb": (None, [_P, _P]),
        "orc_select": (_i, [_P, _i, _d, _P, _P]),
        "orc_select_f32": (None, [_P, _i, _ll, _P, _P, _P]),
        "orc_interp_syn": (_d, [_P, _P, _i, _d, _d, _d, _d]),
        "orc_interp_brems": (_d, [_P, _P, _d]),
        "orc_interp_coulomb": (_d, [_P, _P, _d, _d]),
        "orc_step": (_i, [_P, _P, _P, _P, _i, _i, _P, _ll, _P, _P, _P, _P, _P,
                          _P, _P, _P, _P, _P, _i]),
        "orc_keys_f32": (None, [_P, _ll, _P, _P, _P, _P, _P, _P]),
        "orc_cool_q_cell": (_d, [_P, _P, _P, _P, _i, _P, _d, _d, _d, _d]),
        "orc_step_pairs": (_i, [_P, _P, _P, _P, _P, _ll, _P, _P, _P, _P, _P,
                                _P, _P, _P, _P, _P, _i]),
        "orc_build_qtotal": (None, [_P, _P, _P, _P]),
        "orc_step_qtotal": (_i, [_P, _P, _P, _P, _ll, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _i]),
        "orc_step_bwd": (_i, [_P, _P, _P, _P, _P, _ll, _P, _P, _P, _P, _P, _P, _P, _P,
                              _P, _P, _P, _P, _P, _P, _i, _i]),
        "orc_step_surrogate": (_i, [_P, _P, _P, _P, _P, _d, _d, _P, _P, _d, _P, _i, _P, _ll,
                                    _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _i]),
        "orc_net_eval": (_i, [_P, _d, _d, _d, _i, _ll, _P, _P]),
        "orc_quartic_root": (_d, [_d, _d, _d]),
        "orc_h_thermal": (_d, [_P, _d, _d, _d, _d, _d]),
        "orc_step_disk": (_i, [_P, _P, _P, _P, _i, _P, _P, _ll, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                               _i]),
        "orc_radiation_te": (None, [_P, _d, _d, _ll, _P, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _ref(x):
    return C.cast(C.pointer(x), C.c_void_p)


# ---- scalar physics ---------------------------------------------------------

def const(name):
    idx = dict(c=0, k_B=1, m_e=2, m_p=3, e=4, h=5, sigma_T=6, sigma_SB=7, G=8, M_sun=9)[name]
    return lib().orc_const(idx)


def kve(nu, z):
    return lib().orc_kve(int(nu), float(z))


def theta_e(T):
    return lib().orc_theta_e(float(T))


def brems_ee(T):
    return lib().orc_brems_ee(float(T))


def brems_ei(T):
    return lib().orc_brems_ei(float(T))


def brems(T):
    return lib().orc_brems(float(T))


def Iprime(x):
    return lib().orc_Iprime(float(x))


def k2_factor(T, k2_switch_T=1e8):
    return lib().orc_k2_factor(float(T), float(k2_switch_T))


def nu0(B, T):
    return lib().orc_nu0(float(B), float(T))


def eps_syn(nu, ne, B, T, k2_switch_T=1e8):
    return lib().orc_eps_syn(float(nu), float(ne), float(B), float(T), float(k2_switch_T))


def nu_c(H, B, ne, T, k2_switch_T=1e8):
    flag = C.c_int(0)
    v = lib().orc_nu_c(float(H), float(B), float(ne), float(T), float(k2_switch_T), _ref(flag))
    return v, flag.value


def J(xc, panels=64):
    return lib().orc_J(float(xc), int(panels))


def qsyn_nu(H, B, ne, T, nuc, k2_switch_T=1e8, panels=64):
    return lib().orc_qsyn_nu(float(H), float(B), float(ne), float(T), float(k2_switch_T),
                             float(nuc), int(panels))


def eta(nuc, T, ne, H, literal=0):
    return lib().orc_eta(float(nuc), float(T), float(ne), float(H), int(literal))


def eta_qsyn(H, B, ne, T, spec=None):
    s = (spec or Spec()).c()
    return lib().orc_eta_qsyn(float(H), float(B), float(ne), float(T), _ref(s), None)


def bridge(qthin, T, H, ne):
    return lib().orc_bridge(float(qthin), float(T), float(H), float(ne))


def qtotal_direct(H, B, ne, T, spec=None):
    s = (spec or Spec()).c()
    return lib().orc_qtotal_direct(float(H), float(B), float(ne), float(T), _ref(s))


def coulomb_C(Ti, Te, spec=None):
    s = (spec or Spec()).c()
    return lib().orc_coulomb_C(float(Ti), float(Te), _ref(s))


def gl16():
    x = np.zeros(16)
    w = np.zeros(16)
    lib().orc_gl16(_ptr(x), _ptr(w))
    return x, w


# ---- tables ----------------------------------------------------------------

def nodes(spec, axis):
    n = spec.n[axis]
    x64 = np.zeros(n)
    l64 = np.zeros(n)
    x32 = np.zeros(n, np.float32)
    s = spec.c()
    lib().orc_nodes(_ref(s), int(axis), _ptr(x64), _ptr(l64), _ptr(x32))
    return x64, l64, x32


def build_tables(spec, nthreads=0, syn=True):
    """Full O2 tables (log2 values).  syn=False leaves the 4-D channel NaN
    (lazy: nodes are computed on first use by a single-threaded step)."""
    s = spec.c()
    nH, nB, nN, nT, nC = spec.n
    lb = np.zeros(nT)
    lc = np.zeros(nC * nC)
    ls = np.full(nH * nB * nN * nT, np.nan)
    lib().orc_build_brems(_ref(s), _ptr(lb))
    lib().orc_build_coulomb(_ref(s), _ptr(lc))
    if syn:
        lib().orc_build_syn(_ref(s), _ptr(ls), int(nthreads))
    return dict(lb=lb, ls=ls, lc=lc.reshape(nC, nC))


def syn_at(spec, flat_idx, nthreads=0):
    """4-D channel values at the given flat indices (computed pointwise)."""
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.zeros(idx.size)
    s = spec.c()
    lib().orc_build_syn_at(_ref(s), idx.size, _ptr(idx), _ptr(out), int(nthreads))
    return out


def syn_node(spec, h, b, n, t):
    s = spec.c()
    return lib().orc_syn_node(_ref(s), int(h), int(b), int(n), int(t))


def select_f32(spec, axis, keys):
    k = np.ascontiguousarray(keys, dtype=np.float32)
    idx = np.zeros(k.size, np.int32)
    w = np.zeros(k.size)
    s = spec.c()
    lib().orc_select_f32(_ref(s), int(axis), k.size, _ptr(k), _ptr(idx), _ptr(w))
    return idx, w


def interp_syn(spec, tables, H, B, ne, T, lazy=False):
    s = spec.c()
    return lib().orc_interp_syn(_ref(s), _ptr(tables["ls"]), int(lazy), float(H), float(B),
                                float(ne), float(T))


def interp_brems(spec, tables, T):
    s = spec.c()
    return lib().orc_interp_brems(_ref(s), _ptr(tables["lb"]), float(T))


def interp_coulomb(spec, tables, Ti, Te):
    s = spec.c()
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    return lib().orc_interp_coulomb(_ref(s), _ptr(lc), float(Ti), float(Te))


def round_tables(tables, dtype=np.float32):
    """The tables with their log2 values rounded to `dtype` (the packed
    storage precision of the GPU path), returned as FP64 arrays."""
    return {k: v.astype(dtype).astype(np.float64) for k, v in tables.items()}


# ---- step ------------------------------------------------------------------

COUNTER_NAMES = ("clamped", "invalid", "stiff", "eq_band", "implicit_fail", "fallback", "floor")


def step(spec, tables, params, rho, B, H, ue, ui, lazy=False, direct=False, nthreads=0):
    """One cool_step of the O2 (table) or O1 (direct) oracle on FP64 copies of
    the fields.  Returns (ue_out, ui_out, q_cool, q_cc, counters dict)."""
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (rho, B, H, ue, ui)]
    n = f[0].size
    ue_o = np.zeros(n)
    ui_o = np.zeros(n)
    qc = np.zeros(n)
    qx = np.zeros(n)
    cnt = np.zeros(7, np.int64)
    s = spec.c()
    p = params.c()
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    ls = tables["ls"]
    assert ls.flags.c_contiguous and ls.dtype == np.float64
    rc = lib().orc_step(_ref(s), _ptr(tables["lb"]), _ptr(ls), _ptr(lc), int(lazy), int(direct),
                        _ref(p), n, *[_ptr(a) for a in f], _ptr(ue_o), _ptr(ui_o), _ptr(qc),
                        _ptr(qx), _ptr(cnt), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_step failed: {rc}")
    return ue_o, ui_o, qc, qx, dict(zip(COUNTER_NAMES, cnt.tolist()))


def cool_q_cell(spec, tables, params, rho, B, H, ue, direct=False):
    """Energy removed by cooling in one sub-cycle at electron energy ue."""
    s = spec.c()
    p = params.c()
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    return lib().orc_cool_q_cell(_ref(s), _ptr(tables["lb"]), _ptr(tables["ls"]), _ptr(lc),
                                 int(direct), _ref(p), float(rho), float(B), float(H), float(ue))


def step_pairs(spec, lb, lsp, lc, params, rho, B, H, ue, ui, nthreads=0):
    """The O2 step reading the 4-D channel as per-interval node pairs
    lsp[row, t, 0/1] (see oracle.quant) and the given brems/Coulomb
    channels.  Returns the same tuple as step()."""
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (rho, B, H, ue, ui)]
    n = f[0].size
    outs = [np.zeros(n) for _ in range(4)]
    cnt = np.zeros(7, np.int64)
    s = spec.c()
    p = params.c()
    lsp = np.ascontiguousarray(lsp, dtype=np.float64)
    lb = np.ascontiguousarray(lb, dtype=np.float64)
    lc = np.ascontiguousarray(lc, dtype=np.float64).reshape(-1)
    rc = lib().orc_step_pairs(_ref(s), _ptr(lb), _ptr(lsp), _ptr(lc), _ref(p), n, *[_ptr(a) for a in f],
                              *[_ptr(a) for a in outs], _ptr(cnt), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_step_pairs failed: {rc}")
    return outs[0], outs[1], outs[2], outs[3], dict(zip(COUNTER_NAMES, cnt.tolist()))


def build_qtotal(spec, tables):
    """The paper's table layout (Sec. 3.1): log2 Q_total on the 4-D grid,
    the bridge of Eqs. 11-12 applied at each node to the table's brems and
    synchrotron values (flat, the layout of tables['ls'])."""
    s = spec.c()
    ls = tables["ls"]
    assert ls.flags.c_contiguous and ls.dtype == np.float64 and not np.isnan(ls).any()
    ltot = np.zeros_like(ls)
    lib().orc_build_qtotal(_ref(s), _ptr(tables["lb"]), _ptr(ls), _ptr(ltot))
    return ltot


def step_qtotal(spec, tables, ltot, params, rho, B, H, ue, ui, nthreads=0):
    """The O2 step on the paper's layout: the cooling rate interpolated from
    ltot (build_qtotal) instead of brems + synchrotron + run-time bridge;
    the Coulomb exchange as step().  Returns the same tuple as step()."""
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (rho, B, H, ue, ui)]
    n = f[0].size
    outs = [np.zeros(n) for _ in range(4)]
    cnt = np.zeros(7, np.int64)
    s = spec.c()
    p = params.c()
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    ltot = np.ascontiguousarray(ltot, dtype=np.float64)
    rc = lib().orc_step_qtotal(_ref(s), _ptr(lc), _ptr(ltot), _ref(p), n, *[_ptr(a) for a in f],
                               *[_ptr(a) for a in outs], _ptr(cnt), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_step_qtotal failed: {rc}")
    return outs[0], outs[1], outs[2], outs[3], dict(zip(COUNTER_NAMES, cnt.tolist()))


def step_bwd(spec, tables, params, rho, B, H, ue, ui, g_ue, g_ui, table_grads=False, nthreads=0, lazy=False):
    """Adjoint of step(): returns dict with g_rho, g_B, g_H, g_ue, g_ui (per
    cell), the table adjoints g_lb, g_ls, g_lc (natural layouts) when asked,
    sig (hash of each cell's discrete decisions) and the forward outputs.
    lazy: tables from build_tables(..., syn=False); the 4-D channel's nodes
    are computed on first use (one thread)."""
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (rho, B, H, ue, ui, g_ue, g_ui)]
    n = f[0].size
    grads = np.zeros((n, 5))
    sig = np.zeros(n, np.uint64)
    ue_o = np.zeros(n)
    ui_o = np.zeros(n)
    nH, nB, nN, nT, nC = spec.n
    g_lb = np.zeros(nT) if table_grads else None
    g_ls = np.zeros(nH * nB * nN * nT) if table_grads else None
    g_lc = np.zeros(nC * nC) if table_grads else None
    s = spec.c()
    p = params.c()
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    rc = lib().orc_step_bwd(_ref(s), _ptr(tables["lb"]), _ptr(tables["ls"]), _ptr(lc), _ref(p), n,
                            *[_ptr(a) for a in f], _ptr(grads), _ptr(g_lb), _ptr(g_ls), _ptr(g_lc),
                            _ptr(sig), _ptr(ue_o), _ptr(ui_o), int(nthreads), 1 if lazy else 0)
    if rc != 0:
        raise RuntimeError(f"orc_step_bwd failed: {rc}")
    out = dict(g_rho=grads[:, 0], g_B=grads[:, 1], g_H=grads[:, 2], g_ue=grads[:, 3], g_ui=grads[:, 4],
               sig=sig, ue=ue_o, ui=ui_o)
    if table_grads:
        out.update(g_lb=g_lb, g_ls=g_ls, g_lc=g_lc.reshape(nC, nC))
    return out


def net_box(spec):
    """(l0[4], span[4], xs): the surrogate's input normalisation over the
    table box (log2 of the H, B, n_e, T_e ranges) and the normalised log2 of
    the K2 switch temperature."""
    l0 = np.log2(np.asarray(spec.lo[:4], np.float64))
    span = np.log2(np.asarray(spec.hi[:4], np.float64)) - l0
    xs = 2.0 * (np.log2(spec.k2_switch_T) - l0[3]) / span[3] - 1.0
    return l0, span, float(xs)


def net_eval(params, mean, std, xs, x, rounding=True):
    """The surrogate network (C restatement) at normalised points x [n][4]."""
    p = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros(x.shape[0])
    lib().orc_net_eval(_ptr(p), float(mean), float(std), float(xs), int(rounding), x.shape[0], _ptr(x),
                       _ptr(out))
    return out


def step_surrogate(spec, tables, params, mean, std, mask, prm, rho, B, H, ue, ui, rounding=True,
                   nthreads=0):
    """The O2 step with the surrogate network in place of the 4-D channel
    (table where the uint32 fallback bits `mask` are set; None: nowhere).
    Returns the same tuple as step(); counters['fallback'] counts cells that
    read the table in some sub-cycle."""
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in (rho, B, H, ue, ui)]
    n = f[0].size
    outs = [np.zeros(n) for _ in range(4)]
    cnt = np.zeros(7, np.int64)
    s = spec.c()
    pc = prm.c()
    l0, span, xs = net_box(spec)
    pv = np.ascontiguousarray(params, np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint32)
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    rc = lib().orc_step_surrogate(_ref(s), _ptr(tables["lb"]), _ptr(tables["ls"]), _ptr(lc), _ptr(pv),
                                  float(mean), float(std), _ptr(l0), _ptr(span), xs, _ptr(m), int(rounding),
                                  _ref(pc), n, *[_ptr(a) for a in f], *[_ptr(a) for a in outs], _ptr(cnt),
                                  int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_step_surrogate failed: {rc}")
    return outs[0], outs[1], outs[2], outs[3], dict(zip(COUNTER_NAMES, cnt.tolist()))


def h_thermal(params, rho, ue, ui, r, spin=0.0):
    """H_th = c_s / Omega_K [r_g] of one cell (Sec. 2.7)."""
    p = params.c()
    return lib().orc_h_thermal(_ref(p), float(rho), float(ue), float(ui), float(r), float(spin))


def step_disk(spec, tables, params, rho, B, H, ue, ui, r, spin=0.0, h_floor=0.0, h_from_state=False,
              direct=False, nthreads=0):
    """The O2 (or O1) step with the disk geometry of each cell: H_th from the
    state when h_from_state (H may be None), the temperature floor when
    h_floor > 0.  Returns the same tuple as step(); counters['floor']."""
    f = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))
         for a in (rho, B, H, ue, ui, r)]
    n = f[0].size
    outs = [np.zeros(n) for _ in range(4)]
    cnt = np.zeros(7, np.int64)
    s = spec.c()
    p = params.c()
    d = _Disk(float(spin), float(h_floor), int(bool(h_from_state)))
    lc = np.ascontiguousarray(tables["lc"]).reshape(-1)
    rc = lib().orc_step_disk(_ref(s), _ptr(tables["lb"]), _ptr(tables["ls"]), _ptr(lc), int(direct), _ref(p),
                             _ref(d), n, *[_ptr(a) for a in f[:5]], _ptr(f[5]), *[_ptr(a) for a in outs],
                             _ptr(cnt), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"orc_step_disk failed: {rc}")
    return outs[0], outs[1], outs[2], outs[3], dict(zip(COUNTER_NAMES, cnt.tolist()))


A_RAD = 7.5646e-15   # radiation constant as printed with the total-pressure equation (Sec. 5.2)


def quartic_root(a, b, c):
    """Positive root of a x^4 + b x - c = 0 (closed form, a, b, c > 0)."""
    return lib().orc_quartic_root(float(a), float(b), float(c))


def radiation_te(params, rho, H, ue, tau_crit=4.6, a_rad=A_RAD):
    """(T_e [K], thick flag) of the radiation-pressure correction per cell."""
    f = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (rho, H, ue)]
    n = f[0].size
    te = np.zeros(n)
    thick = np.zeros(n, np.int32)
    p = params.c()
    lib().orc_radiation_te(_ref(p), float(tau_crit), float(a_rad), n, *[_ptr(x) for x in f], _ptr(te),
                           _ptr(thick))
    return te, thick.astype(bool)


def keys_f32(params, rho, B, H, ue, ui):
    f = [np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (rho, B, H, ue, ui)]
    n = f[0].size
    keys = np.zeros((n, 5), np.float32)
    p = params.c()
    lib().orc_keys_f32(_ref(p), n, *[_ptr(a) for a in f], _ptr(keys))
    return keys
