"""B300-native two-temperature cooling step (arXiv 2505.08855).

Python front end of libcool (include/cool.h):

    import paper_2505_08855_b300 as cool
    tab = cool.Table(cool.TableSpec(n=(64, 64, 64, 64, 64)))     # built on the GPU in FP64
    ue, ui = cool.step(tab, cool.Params(n_sub=8), rho, B, H, ue, ui)

Fields are CUDA torch tensors (float32 or float64, contiguous).  Every
computation runs in the library's CUDA kernels on the tensors' device and
the current torch stream; this module only marshals arguments.
"""
import ctypes as C
import dataclasses

from . import binding as _b

F32, BF16, F16, F64 = _b.COOL_F32, _b.COOL_BF16, _b.COOL_F16, _b.COOL_F64
EXPLICIT, IMPLICIT = _b.COOL_EXPLICIT_LIMITED, _b.COOL_IMPLICIT_STIFF
PATH_L2WINDOW, PATH_TMA_SMEM, PATH_TEXTURE_POINT, PATH_TEXTURE_HWLERP, PATH_QTOTAL = (
    _b.COOL_PATH_L2WINDOW, _b.COOL_PATH_TMA_SMEM, _b.COOL_PATH_TEXTURE_POINT, _b.COOL_PATH_TEXTURE_HWLERP,
    _b.COOL_PATH_QTOTAL)
CoolError = _b.CoolError

# Axis order of the table: 0 H [cm], 1 |B| [G], 2 n_e [cm^-3], 3 T_e [K],
# 4 Coulomb T [K].  Ranges: the paper's Sec. 2.6 and 2.8.
PAPER_LO = (1e3, 1.0, 1e2, 1e2, 1e2)
PAPER_HI = (1e12, 1e10, 1e25, 1e15, 1e15)


@dataclasses.dataclass
class TableSpec:
    n: tuple = (64, 64, 64, 64, 64)
    lo: tuple = PAPER_LO
    hi: tuple = PAPER_HI
    dtype: int = F32
    row_scaled: int = 0
    k2_switch_T: float = 1e8
    lnLambda: float = 20.0
    theta_i_uses_mp: int = 1
    compton_literal: int = 0

    def c(self):
        if tuple(self.lo[3:4]) != tuple(self.lo[4:5]) or tuple(self.hi[3:4]) != tuple(self.hi[4:5]):
            raise ValueError("the T_e and Coulomb T axes share one range")
        return _b.cool_table_spec(*self.n, self.lo[0], self.hi[0], self.lo[1], self.hi[1],
                                  self.lo[2], self.hi[2], self.lo[3], self.hi[3], self.dtype,
                                  self.row_scaled, self.k2_switch_T, self.lnLambda,
                                  self.theta_i_uses_mp, self.compton_literal)


@dataclasses.dataclass
class Params:
    rho_scale: float = 3e-7
    M_bh_msun: float = 10.0
    gamma_e: float = 5.0 / 3.0
    gamma_i: float = 5.0 / 3.0
    dt: float = 1e-2
    n_sub: int = 8
    mode: int = EXPLICIT
    limiter_frac: float = 0.3
    eq_band: float = 0.1
    coulomb_clamp: float = 1.0
    implicit_iters: int = 60
    path: int = _b.COOL_PATH_L2WINDOW
    fp64_critical: int = 0

    def c(self):
        return _b.cool_params(self.rho_scale, self.M_bh_msun, self.gamma_e, self.gamma_i,
                              self.dt, self.n_sub, self.mode, self.limiter_frac, self.eq_band,
                              self.coulomb_clamp, self.implicit_iters, self.path, self.fp64_critical)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Table:
    """A cooling/Coulomb rate table on the current CUDA device."""

    def __init__(self, spec=None, _handle=None):
        self.spec = spec if spec is not None else TableSpec()
        if _handle is not None:
            self._h = _handle
            return
        L = _b.lib()
        h = C.c_void_p()
        cs = self.spec.c()
        _b.check(L.cool_build_table(_b.ref(cs), _stream_ptr(), _b.ref(h)), "cool_build_table")
        self._h = h

    @classmethod
    def load(cls, path):
        L = _b.lib()
        h = C.c_void_p()
        _b.check(L.cool_table_load(path.encode(), _stream_ptr(), _b.ref(h)), "cool_table_load")
        s = _b.cool_table_spec()
        _b.check(L.cool_table_get_spec(h, _b.ref(s)), "cool_table_get_spec")
        spec = TableSpec(n=(s.n_H, s.n_B, s.n_ne, s.n_Te, s.n_Tc),
                         lo=(s.H_min, s.B_min, s.ne_min, s.T_min, s.T_min),
                         hi=(s.H_max, s.B_max, s.ne_max, s.T_max, s.T_max), dtype=s.dtype,
                         row_scaled=s.row_scaled, k2_switch_T=s.k2_switch_T, lnLambda=s.lnLambda,
                         theta_i_uses_mp=s.theta_i_uses_mp, compton_literal=s.compton_literal)
        return cls(spec, _handle=h)

    @property
    def handle(self):
        if self._h is None:
            raise _b.CoolError(_b.COOL_ESTATE, "table already freed")
        return self._h

    def save(self, path):
        _b.check(_b.lib().cool_table_save(self.handle, path.encode()), "cool_table_save")

    def export(self, channel):
        """FP64 log2 values of channel 0 (brems), 1 (synchrotron), 2 (Coulomb)
        or 3 (the paper's layout, log2 Q_total; made on first use) as numpy."""
        import numpy as np
        n = self.spec.n
        count = {0: n[3], 1: n[0] * n[1] * n[2] * n[3], 2: n[4] * n[4], 3: n[0] * n[1] * n[2] * n[3]}[channel]
        out = np.zeros(count, np.float64)
        _b.check(_b.lib().cool_table_export(self.handle, channel, out.ctypes.data_as(C.c_void_p),
                                            count), "cool_table_export")
        return out

    def packed_bytes(self):
        """Bytes of the 4-D channel as packed for the step."""
        nb = C.c_longlong(0)
        _b.check(_b.lib().cool_table_packed_bytes(self.handle, _b.ref(nb)), "cool_table_packed_bytes")
        return nb.value

    def export_packed(self):
        """The 4-D channel as packed for the step (uint32 words, 8 per block)."""
        import numpy as np
        nb = C.c_longlong(0)
        _b.check(_b.lib().cool_table_packed_bytes(self.handle, _b.ref(nb)), "cool_table_packed_bytes")
        out = np.zeros(nb.value // 4, np.uint32)
        _b.check(_b.lib().cool_table_export_packed(self.handle, out.ctypes.data_as(C.c_void_p), nb.value),
                 "cool_table_export_packed")
        return out

    def nodes(self, axis):
        import numpy as np
        out = np.zeros(self.spec.n[axis], np.float32)
        _b.check(_b.lib().cool_table_nodes(self.handle, axis, out.ctypes.data_as(C.c_void_p),
                                           out.size), "cool_table_nodes")
        return out

    def l2_persist(self, on=True):
        """cool_table_l2_persist: reserve persisting L2 for the packed 4-D
        channel (context-wide; off by default) or give it back."""
        _b.check(_b.lib().cool_table_l2_persist(self.handle, 1 if on else 0), "cool_table_l2_persist")

    def free(self):
        if self._h is not None:
            _b.check(_b.lib().cool_table_free(self._h), "cool_table_free")
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and _b._LIB is not None:
                _b._LIB.cool_table_free(self._h)
                self._h = None
        except Exception:
            pass


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"fields must be float32 or float64, got {t.dtype}")


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def new_counters(device=None):
    """A zeroed device counter block (int64 x 8, cool_counters) for step(..., counters=)."""
    import torch
    return torch.zeros(len(COUNTER_NAMES), dtype=torch.int64, device=device or "cuda")


COUNTER_NAMES = ("clamped", "nonfinite", "stiff", "fp64_coulomb", "implicit_fail", "fallback", "floor",
                 "exact_redo")


def counters_dict(c):
    return dict(zip(COUNTER_NAMES, c.tolist()))


def step(table, params, rho, B, H, ue, ui, ue_out=None, ui_out=None, q_cool=None, q_cc=None,
         counters=None, stream=None):
    """One cooling step (cool_step).  Returns (ue_out, ui_out); outputs are
    allocated when not given (pass ue_out=ue for in place).  q_cool / q_cc:
    optional output tensors of the cooled / Coulomb-exchanged energy."""
    import torch
    fields = (rho, B, H, ue, ui)
    code = _dtype_code(rho)
    n = rho.numel()
    for f in fields:
        if f.dtype != rho.dtype or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("fields must be contiguous CUDA tensors of one dtype and size")
    if ue_out is None:
        ue_out = torch.empty_like(ue)
    if ui_out is None:
        ui_out = torch.empty_like(ui)
    p = params.c()
    cptr = C.c_void_p(counters.data_ptr()) if counters is not None else C.c_void_p(0)
    st = _b.lib().cool_step(table.handle, _b.ref(p), n, code, *[_ptr(f) for f in fields],
                            _ptr(ue_out), _ptr(ui_out), _ptr(q_cool), _ptr(q_cc), cptr,
                            _stream_ptr(stream))
    _b.check(st, "cool_step")
    return ue_out, ui_out


@dataclasses.dataclass
class Disk:
    """Disk geometry for step_disk (cool_disk)."""
    spin: float = 0.9375
    h_floor: float = 0.0
    h_from_state: int = 0

    def c(self):
        return _b.cool_disk(self.spin, self.h_floor, self.h_from_state)


def step_disk(table, params, disk, rho, B, H, ue, ui, r, ue_out=None, ui_out=None, q_cool=None, q_cc=None,
              counters=None, stream=None):
    """cool_step_disk: the step with each cell's radius r (H may be None when
    disk.h_from_state).  float32 CUDA tensors; returns (ue_out, ui_out)."""
    import torch
    n = rho.numel()
    for f in (rho, B, H, ue, ui, r):
        if f is None:
            continue
        if f.dtype != torch.float32 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("fields must be contiguous float32 CUDA tensors of one size")
    if ue_out is None:
        ue_out = torch.empty_like(ue)
    if ui_out is None:
        ui_out = torch.empty_like(ui)
    p = params.c()
    d = disk.c()
    cptr = C.c_void_p(counters.data_ptr()) if counters is not None else C.c_void_p(0)
    _b.check(_b.lib().cool_step_disk(table.handle, _b.ref(p), _b.ref(d), n, _ptr(rho), _ptr(B), _ptr(H), _ptr(ue),
                                     _ptr(ui), _ptr(r), _ptr(ue_out), _ptr(ui_out), _ptr(q_cool), _ptr(q_cc), cptr,
                                     _stream_ptr(stream)), "cool_step_disk")
    return ue_out, ui_out


def step_host(table, params, rho, B, H, ue, ui, ue_out, ui_out, chunk_cells=0, counters=None, stream=None):
    """cool_step_host: the step on host (CPU, preferably pinned) float32
    tensors, streamed through the device in overlapping chunks; asynchronous
    on `stream` (synchronise before reading ue_out / ui_out)."""
    import torch
    fields = (rho, B, H, ue, ui, ue_out, ui_out)
    n = rho.numel()
    for f in fields:
        if f.dtype != torch.float32 or f.numel() != n or f.is_cuda or not f.is_contiguous():
            raise ValueError("fields must be contiguous float32 host tensors of one size")
    p = params.c()
    cptr = C.c_void_p(counters.data_ptr()) if counters is not None else C.c_void_p(0)
    _b.check(_b.lib().cool_step_host(table.handle, _b.ref(p), n, *[_ptr(f) for f in fields], int(chunk_cells), cptr,
                                     _stream_ptr(stream)), "cool_step_host")
    return ue_out, ui_out


A_RAD_PAPER = 7.5646e-15   # erg cm^-3 K^-4, as printed with the total-pressure equation


def radiation_te(params, rho, H, ue, tau_crit=4.6, a_rad=A_RAD_PAPER, te_out=None, thick_out=None, stream=None):
    """cool_radiation_te: the radiation-pressure corrected T_e [K] (float32
    CUDA tensors); returns (te_out, thick_out or None)."""
    import torch
    n = rho.numel()
    for f in (rho, H, ue):
        if f.dtype != torch.float32 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("fields must be contiguous float32 CUDA tensors of one size")
    if te_out is None:
        te_out = torch.empty_like(rho)
    p = params.c()
    _b.check(_b.lib().cool_radiation_te(_b.ref(p), float(tau_crit), float(a_rad), n, _ptr(rho), _ptr(H), _ptr(ue),
                                        _ptr(te_out), _ptr(thick_out), _stream_ptr(stream)), "cool_radiation_te")
    return te_out, thick_out


def step_direct(spec, params, rho, B, H, ue, ui, ue_out=None, ui_out=None, q_cool=None, q_cc=None,
                counters=None, stream=None):
    """cool_step_direct: the step with every rate from the formulas (FP64
    CUDA tensors; `spec` supplies the physics flags only)."""
    import torch
    fields = (rho, B, H, ue, ui)
    n = rho.numel()
    for f in fields:
        if f.dtype != torch.float64 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("fields must be contiguous float64 CUDA tensors of one size")
    if ue_out is None:
        ue_out = torch.empty_like(ue)
    if ui_out is None:
        ui_out = torch.empty_like(ui)
    cs = spec.c()
    p = params.c()
    cptr = C.c_void_p(counters.data_ptr()) if counters is not None else C.c_void_p(0)
    _b.check(_b.lib().cool_step_direct(_b.ref(cs), _b.ref(p), n, *[_ptr(f) for f in fields], _ptr(ue_out),
                                       _ptr(ui_out), _ptr(q_cool), _ptr(q_cc), cptr, _stream_ptr(stream)),
             "cool_step_direct")
    return ue_out, ui_out


def debug_wait_timeout(polls, stream=None):
    """cool_debug_wait_timeout: run a bounded wait on a barrier that never
    completes; returns the error word it reported (1 when the wait ran out).
    Synchronous."""
    import torch
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    _b.check(_b.lib().cool_debug_wait_timeout(int(polls), _ptr(err), _stream_ptr(stream)),
             "cool_debug_wait_timeout")
    torch.cuda.synchronize()
    return int(err.item())


def tma_error(clear=True):
    """cool_tma_error: the TMA_SMEM path's error word on the current device
    (bit 0: a field copy that never completed).  Synchronous."""
    v = C.c_uint(0)
    _b.check(_b.lib().cool_tma_error(C.byref(v), 1 if clear else 0), "cool_tma_error")
    return int(v.value)


def release_scratch():
    """cool_release_scratch: free the deferral-list scratch kept for the
    current device's streams (after synchronising the device)."""
    _b.check(_b.lib().cool_release_scratch(), "cool_release_scratch")


def debug_lookup(table, axis, keys, stream=None):
    """(idx int32, w float32) of the interpolation rule for FP32 keys."""
    import torch
    keys = keys.contiguous()
    idx = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    w = torch.empty(keys.numel(), dtype=torch.float32, device=keys.device)
    _b.check(_b.lib().cool_debug_lookup(table.handle, axis, keys.numel(), _ptr(keys), _ptr(idx),
                                        _ptr(w), _stream_ptr(stream)), "cool_debug_lookup")
    return idx, w


def _check_noalloc_outputs(spec, lb_out, ls_out, lc_out):
    """The library writes exactly n_Te, n_H n_B n_ne n_Te and n_Tc^2 doubles
    through raw pointers: anything else (another dtype, a shorter tensor, a
    tensor on another device) is refused here, before any launch."""
    import torch
    n_h, n_b, n_ne, n_te, n_tc = spec.n
    want = (n_te, n_h * n_b * n_ne * n_te, n_tc * n_tc)
    outs = list(zip(("lb_out", "ls_out", "lc_out"), (lb_out, ls_out, lc_out), want))
    for name, t, m in outs:
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if t.numel() != m:
            raise ValueError(f"{name} must hold exactly {m} elements, got {t.numel()}")
    for name, t, _ in outs:
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must live on the current CUDA device")


def build_channels_noalloc(spec, lb_out, ls_out, lc_out, stream=None):
    """cool_build_channels_noalloc: the table's FP64 log2 channels written into
    caller-allocated CUDA float64 tensors (sizes n_Te, n_H n_B n_ne n_Te,
    n_Tc^2); the library allocates no device memory for it."""
    _check_noalloc_outputs(spec, lb_out, ls_out, lc_out)
    cs = spec.c()
    _b.check(_b.lib().cool_build_channels_noalloc(_b.ref(cs), _ptr(lb_out), _ptr(ls_out), _ptr(lc_out),
                                                  _stream_ptr(stream)), "cool_build_channels_noalloc")


def step_bwd(table, params, rho, B, H, ue, ui, g_ue_out, g_ui_out, table_grads=None, stream=None):
    """Adjoint of step (cool_step_bwd) for FP32 fields: returns (g_rho, g_B,
    g_H, g_ue_in, g_ui_in).  table_grads: optional dict of float32 CUDA
    tensors 'lb' [n_Te], 'ls' [n_H n_B n_ne n_Te], 'lc' [n_Tc^2] into which
    dL/d(log2 table values) is added."""
    import torch
    fields = (rho, B, H, ue, ui, g_ue_out, g_ui_out)
    n = rho.numel()
    for f in fields:
        if f.dtype != torch.float32 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("step_bwd takes contiguous float32 CUDA tensors of one size")
    outs = [torch.empty_like(rho) for _ in range(5)]
    tg = table_grads or {}
    p = params.c()
    st = _b.lib().cool_step_bwd(table.handle, _b.ref(p), n, *[_ptr(f) for f in fields], *[_ptr(o) for o in outs],
                                _ptr(tg.get("lb")), _ptr(tg.get("ls")), _ptr(tg.get("lc")), _stream_ptr(stream))
    _b.check(st, "cool_step_bwd")
    return tuple(outs)


def step_fwd_jac(table, params, rho, B, H, ue, ui, ue_out=None, ui_out=None, jac=None, stream=None):
    """cool_step_fwd_jac for FP32 fields: returns (ue_out, ui_out, jac), jac
    a float32 [10, n] tensor (rows d u_e_out/d(rho, B, H, u_e, u_i), then
    d u_i_out/d(the same))."""
    import torch
    n = rho.numel()
    for f in (rho, B, H, ue, ui):
        if f.dtype != torch.float32 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
            raise ValueError("step_fwd_jac takes contiguous float32 CUDA tensors of one size")
    ue_out = torch.empty_like(ue) if ue_out is None else ue_out
    ui_out = torch.empty_like(ui) if ui_out is None else ui_out
    jac = torch.empty((10, n), dtype=torch.float32, device=rho.device) if jac is None else jac
    for f, m in ((ue_out, n), (ui_out, n), (jac, 10 * n)):
        if f.dtype != torch.float32 or f.numel() != m or not f.is_cuda or not f.is_contiguous():
            raise ValueError("step_fwd_jac: outputs must be contiguous float32 CUDA tensors (jac: 10 n)")
    p = params.c()
    st = _b.lib().cool_step_fwd_jac(table.handle, _b.ref(p), n, *[_ptr(f) for f in (rho, B, H, ue, ui)],
                                    _ptr(ue_out), _ptr(ui_out), _ptr(jac), _stream_ptr(stream))
    _b.check(st, "cool_step_fwd_jac")
    return ue_out, ui_out, jac


def step_bwd_jac(jac, g_ue_out, g_ui_out, stream=None):
    """cool_step_bwd_jac: the input gradients (g_rho, g_B, g_H, g_ue_in,
    g_ui_in) from a Jacobian of step_fwd_jac and the output adjoints."""
    import torch
    n = g_ue_out.numel()
    for f, m in ((jac, 10 * n), (g_ue_out, n), (g_ui_out, n)):
        if f.dtype != torch.float32 or f.numel() != m or not f.is_cuda or not f.is_contiguous():
            raise ValueError("step_bwd_jac takes contiguous float32 CUDA tensors (jac: 10 n)")
    outs = [torch.empty_like(g_ue_out) for _ in range(5)]
    st = _b.lib().cool_step_bwd_jac(n, _ptr(jac), _ptr(g_ue_out), _ptr(g_ui_out), *[_ptr(o) for o in outs],
                                    _stream_ptr(stream))
    _b.check(st, "cool_step_bwd_jac")
    return tuple(outs)


def _make_autograd():
    import torch

    class CoolStepFn(torch.autograd.Function):
        """u_e_out, u_i_out = cool_step(rho, B, H, u_e, u_i) with its adjoint.
        Without table gradients the forward is cool_step_fwd_jac: the same
        outputs, plus each cell's 2x5 Jacobian (40 bytes per cell, kept for
        the backward), and the backward is cool_step_bwd_jac, which contracts
        it with the output adjoints; the gradients are cool_step_bwd's bit
        for bit.  Where that is unsupported (fp64_critical, a 16-bit table,
        another table path) or table gradients are asked for, the forward is
        cool_step, keeps only its inputs, and the backward is cool_step_bwd
        (the sub-cycles recomputed); when no input needs a gradient the
        forward is cool_step alone."""

        @staticmethod
        def forward(ctx, rho, B, H, ue, ui, table, params, table_grads=None):
            ctx.table, ctx.params, ctx.table_grads = table, params, table_grads
            ins = [t.detach() for t in (rho, B, H, ue, ui)]
            if (table_grads is None and any(ctx.needs_input_grad[:5]) and not params.fp64_critical
                    and table.spec.dtype == F32 and params.path == _b.COOL_PATH_L2WINDOW):
                ue_o, ui_o, jac = step_fwd_jac(table, params, *ins)
                ctx.save_for_backward(jac)
                ctx.jac = True
            else:
                ue_o, ui_o = step(table, params, *ins)
                ctx.save_for_backward(rho, B, H, ue, ui)
                ctx.jac = False
            return ue_o, ui_o

        @staticmethod
        def backward(ctx, g_ue, g_ui):
            if ctx.jac:
                (jac,) = ctx.saved_tensors
                n = jac.shape[1]
                z = None
                g_ue = torch.zeros(n, device=jac.device) if g_ue is None else g_ue.contiguous()
                g_ui = torch.zeros(n, device=jac.device) if g_ui is None else g_ui.contiguous()
                g = step_bwd_jac(jac, g_ue, g_ui)
                return g[0], g[1], g[2], g[3], g[4], z, z, z
            rho, B, H, ue, ui = ctx.saved_tensors
            g_ue = torch.zeros_like(ue) if g_ue is None else g_ue.contiguous()
            g_ui = torch.zeros_like(ui) if g_ui is None else g_ui.contiguous()
            g = step_bwd(ctx.table, ctx.params, rho, B, H, ue, ui, g_ue, g_ui, ctx.table_grads)
            return g[0], g[1], g[2], g[3], g[4], None, None, None

    return CoolStepFn


_CoolStepFn = None


def cool_step_fn(rho, B, H, ue, ui, table, params, table_grads=None):
    """Differentiable cool_step (torch.autograd)."""
    global _CoolStepFn
    if _CoolStepFn is None:
        _CoolStepFn = _make_autograd()
    return _CoolStepFn.apply(rho, B, H, ue, ui, table, params, table_grads)


# ---- learned surrogate of the synchrotron channel (not in the paper) ----------
N_PARAMS = 18817


@dataclasses.dataclass
class FitSpec:
    channel: int = 1
    n_samples: int = 1 << 24
    batch: int = 16384
    epochs: int = 16
    lr: float = 2e-3
    lr_final: float = 2e-5
    seed: int = 20250513
    fallback_tol: float = 1e-3

    def c(self):
        return _b.cool_fit_spec(self.channel, self.n_samples, self.batch, self.epochs, self.lr, self.lr_final,
                                self.seed, self.fallback_tol)


class Surrogate:
    """An MLP surrogate of a table's synchrotron channel, trained on the GPU
    (cool_surrogate_fit) by the library's tcgen05 kernels."""

    def __init__(self, table, fit=None, stream=None):
        self.table = table
        self.fit_spec = fit if fit is not None else FitSpec()
        h = C.c_void_p()
        f = self.fit_spec.c()
        _b.check(_b.lib().cool_surrogate_fit(table.handle, _b.ref(f), _stream_ptr(stream), _b.ref(h)),
                 "cool_surrogate_fit")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise _b.CoolError(_b.COOL_ESTATE, "surrogate already freed")
        return self._h

    def info(self):
        s = _b.cool_surrogate_stats()
        _b.check(_b.lib().cool_surrogate_info(self.handle, _b.ref(s)), "cool_surrogate_info")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def params(self):
        import numpy as np
        out = np.zeros(N_PARAMS, np.float32)
        _b.check(_b.lib().cool_surrogate_get_params(self.handle, out.ctypes.data_as(C.c_void_p), N_PARAMS),
                 "cool_surrogate_get_params")
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, np.float32)
        _b.check(_b.lib().cool_surrogate_set_params(self.handle, p.ctypes.data_as(C.c_void_p), N_PARAMS),
                 "cool_surrogate_set_params")

    def grads(self, x4, y_std, stream=None):
        import numpy as np
        g = np.zeros(N_PARAMS, np.float32)
        loss = C.c_float(0.0)
        _b.check(_b.lib().cool_surrogate_grads(self.handle, x4.shape[0], _ptr(x4.contiguous()),
                                               _ptr(y_std.contiguous()), g.ctypes.data_as(C.c_void_p),
                                               _b.ref(loss), _stream_ptr(stream)), "cool_surrogate_grads")
        return g, loss.value

    def eval(self, x4, stream=None):
        import torch
        y = torch.empty(x4.shape[0], dtype=torch.float32, device=x4.device)
        _b.check(_b.lib().cool_surrogate_eval(self.handle, x4.shape[0], _ptr(x4.contiguous()), _ptr(y),
                                              _stream_ptr(stream)), "cool_surrogate_eval")
        return y

    def mask(self):
        import numpy as np
        cells = self.info()["mask_cells"]
        out = np.zeros((cells + 31) // 32, np.uint32)
        _b.check(_b.lib().cool_surrogate_mask(self.handle, out.ctypes.data_as(C.c_void_p), out.size),
                 "cool_surrogate_mask")
        return out

    def set_mask(self, bits):
        """Replace the fallback bits (uint32 words, the layout of mask())."""
        import numpy as np
        bits = np.ascontiguousarray(bits, np.uint32)
        _b.check(_b.lib().cool_surrogate_set_mask(self.handle, bits.ctypes.data_as(C.c_void_p), bits.size),
                 "cool_surrogate_set_mask")

    def step(self, params, rho, B, H, ue, ui, ue_out=None, ui_out=None, q_cool=None, q_cc=None,
             counters=None, stream=None, table=None):
        """cool_surrogate_infer: the explicit step with the synchrotron channel
        from the network (table fallback where the mask says so).  FP32 CUDA
        fields; returns (ue_out, ui_out)."""
        import torch
        table = self.table if table is None else table
        fields = (rho, B, H, ue, ui)
        n = rho.numel()
        for f in fields:
            if f.dtype != torch.float32 or f.numel() != n or not f.is_cuda or not f.is_contiguous():
                raise ValueError("fields must be contiguous float32 CUDA tensors of one size")
        if ue_out is None:
            ue_out = torch.empty_like(ue)
        if ui_out is None:
            ui_out = torch.empty_like(ui)
        p = params.c()
        cptr = C.c_void_p(counters.data_ptr()) if counters is not None else C.c_void_p(0)
        _b.check(_b.lib().cool_surrogate_infer(self.handle, table.handle, _b.ref(p), n, *[_ptr(f) for f in fields],
                                               _ptr(ue_out), _ptr(ui_out), _ptr(q_cool), _ptr(q_cc), cptr,
                                               _stream_ptr(stream)), "cool_surrogate_infer")
        return ue_out, ui_out

    def free(self):
        if self._h is not None:
            _b.check(_b.lib().cool_surrogate_free(self._h), "cool_surrogate_free")
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) is not None and _b._LIB is not None:
                _b._LIB.cool_surrogate_free(self._h)
                self._h = None
        except Exception:
            pass
