"""Thin ctypes binding of libaderdg (include/aderdg.h), same names as the C ABI.

Only argument marshalling happens here: every step of the method runs in the
library's CUDA kernels.  Device buffers may be passed as torch CUDA tensors
(their ``data_ptr()`` is used) or as raw integer pointers; streams as
``torch.cuda.Stream`` or raw handles.  If the library is not built this module
raises on first use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

from . import build as _build

ADERDG_OK, ADERDG_EINVAL, ADERDG_ENOMEM, ADERDG_ECUDA = 0, 1, 2, 3
ADERDG_ENONFINITE, ADERDG_ETIMEOUT, ADERDG_EUNSUPPORTED = 4, 5, 6
ADVECTION, ACOUSTICS, EULER, ELASTICITY = 0, 1, 2, 3
FP32, FP64, FP32_ACC64, FP32_PAIR = 0, 1, 2, 3
FORM_FUSED, FORM_HULL3, FORM_TABLE1 = 0, 1, 2
DT_STRICT, DT_CREEPING = 0, 1
PREDICT_AUTO, PREDICT_SPACETIME, PREDICT_SPACETIME_TF32 = 0, 1, 2
JUMPS_PER_CELL_FLUX, JUMPS_NONCONSERVATIVE = 0, 1

PDE_IDS = {"advection": ADVECTION, "acoustics": ACOUSTICS, "euler": EULER, "elasticity": ELASTICITY}
PREC_IDS = {"fp32": FP32, "fp64": FP64, "fp32_acc64": FP32_ACC64, "fp32_pair": FP32_PAIR}
FORM_IDS = {"fused": FORM_FUSED, "hull3": FORM_HULL3, "table1": FORM_TABLE1}


class AderdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"aderdg status {status}: {msg}")
        self.status = status


class aderdg_params(C.Structure):
    _fields_ = [("pde_const", C.c_double * 8), ("cfl", C.c_double), ("picard_iters", C.c_int),
                ("precision", C.c_int), ("form", C.c_int), ("dt_policy", C.c_int),
                ("predictor", C.c_int), ("inject_step", C.c_int), ("inject_factor", C.c_double),
                ("material_jumps", C.c_int)]


class aderdg_source(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("amp", C.c_double * 9), ("kind", C.c_int), ("pad_", C.c_int),
                ("t0", C.c_double), ("f0", C.c_double), ("coef", C.c_double * 8)]


def source(pos, amp, kind=0, t0=0.0, f0=0.0, coef=()):
    """A point source a s(t) delta(x - pos); kind 0: polynomial coefficients of
    (t - t0), kind 1: Ricker wavelet of peak frequency f0 centred at t0."""
    s = aderdg_source()
    s.pos[:] = list(pos) + [0.0] * (3 - len(pos))
    s.amp[:] = list(amp) + [0.0] * (9 - len(amp))
    s.kind, s.t0, s.f0 = int(kind), float(t0), float(f0)
    s.coef[:] = list(coef) + [0.0] * (8 - len(coef))
    return s


class aderdg_scenario(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int), ("m", C.c_int), ("pde", C.c_int),
                ("grid", C.c_int * 3), ("dx", C.c_double * 3), ("pde_const", C.c_double * 8),
                ("cfl", C.c_double)]


class aderdg_stats(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_old", C.c_double), ("dt_new", C.c_double),
                ("lambda_max", C.c_double), ("steps", C.c_longlong), ("reruns", C.c_longlong),
                ("launches", C.c_longlong), ("device_error", C.c_int)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libaderdg.so (building it first only if asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libaderdg is not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.aderdg_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, ip, dp,
                                    C.POINTER(aderdg_params), C.POINTER(vp)]
        L.aderdg_set_material.argtypes = [vp, vp, vp]
        L.aderdg_set_sources.argtypes = [vp, C.c_int, C.POINTER(aderdg_source), vp]
        L.aderdg_step.argtypes = [vp, vp, C.c_int, C.c_double, dp, vp]
        L.aderdg_step_host.argtypes = [vp, vp, C.c_int, C.c_double, dp, vp]
        L.aderdg_begin.argtypes = [vp, vp, C.c_double, vp]
        L.aderdg_advance.argtypes = [vp, vp, C.c_int, vp]
        L.aderdg_end.argtypes = [vp, vp, dp, vp]
        L.aderdg_get_dt_history.argtypes = [vp, dp, C.c_int, ip]
        L.aderdg_get_stats.argtypes = [vp, C.POINTER(aderdg_stats)]
        L.aderdg_nodes.argtypes = [C.c_int, dp, dp]
        L.aderdg_footprint.argtypes = [vp, dp]
        L.aderdg_profile.argtypes = [vp, C.c_int]
        L.aderdg_profile_read.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_longlong)]
        L.aderdg_destroy.argtypes = [vp]
        L.aderdg_step_adjoint.argtypes = [vp, vp, C.c_int, C.c_double, vp, C.c_int, vp, vp, vp,
                                          C.c_int, dp, vp]
        L.aderdg_batch_create.argtypes = [C.c_int, C.POINTER(aderdg_scenario), C.POINTER(vp)]
        L.aderdg_batch_offsets.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.aderdg_batch_step.argtypes = [vp, vp, C.c_int, C.c_int, vp]
        L.aderdg_batch_autotune.argtypes = [vp, vp, C.c_int, vp]
        L.aderdg_batch_get_tuning.argtypes = [vp, ip, ip, C.POINTER(C.c_longlong)]
        L.aderdg_batch_profile.argtypes = [vp, C.c_int]
        L.aderdg_batch_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.aderdg_batch_destroy.argtypes = [vp]
        L.aderdg_step_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, ip, dp,
                                          C.POINTER(aderdg_params), vp, vp, C.c_int, C.c_double,
                                          dp, vp]
        L.aderdg_fp32_fma_peak.argtypes = [C.c_int, dp, vp]
        L.aderdg_last_error.argtypes = [vp]
        L.aderdg_last_error.restype = C.c_char_p
        _lib = L
        return L


def header_functions() -> list[str]:
    """Entry points declared in include/aderdg.h."""
    with open(os.path.join(_build.INCLUDE, "aderdg.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(aderdg_[a-z_]+)\s*\(", src)))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, h=None):
    if st != ADERDG_OK:
        msg = load().aderdg_last_error(h).decode()
        raise AderdgError(st, msg)


def aderdg_create(d, N, m, pde, grid, dx, params: aderdg_params | None = None):
    L = load()
    g = (C.c_int * 3)(*(list(grid) + [1] * (3 - len(grid))))
    h_ = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    out = C.c_void_p()
    st = L.aderdg_create(d, N, m, pde, g, h_, C.byref(params) if params is not None else None,
                         C.byref(out))
    _check(st)
    return out.value


def aderdg_set_material(h, dev_mat, stream=None):
    _check(load().aderdg_set_material(h, _ptr(dev_mat), _stream(stream)), h)


def aderdg_set_sources(h, sources, stream=None):
    """Replace the handle's point sources (a list of aderdg_source)."""
    arr = (aderdg_source * max(1, len(sources)))(*sources)
    _check(load().aderdg_set_sources(h, len(sources), arr if sources else None, _stream(stream)), h)


def aderdg_step(h, dev_Q, nsteps, fixed_dt=0.0, t=0.0, stream=None) -> float:
    tt = C.c_double(t)
    _check(load().aderdg_step(h, _ptr(dev_Q), int(nsteps), float(fixed_dt), C.byref(tt),
                              _stream(stream)), h)
    return tt.value


def aderdg_step_host(h, host_Q, nsteps, fixed_dt=0.0, t=0.0, stream=None) -> float:
    tt = C.c_double(t)
    _check(load().aderdg_step_host(h, _ptr(host_Q), int(nsteps), float(fixed_dt), C.byref(tt),
                                   _stream(stream)), h)
    return tt.value


def aderdg_begin(h, dev_Q, fixed_dt=0.0, stream=None):
    _check(load().aderdg_begin(h, _ptr(dev_Q), float(fixed_dt), _stream(stream)), h)


def aderdg_advance(h, dev_Q, k, stream=None):
    _check(load().aderdg_advance(h, _ptr(dev_Q), int(k), _stream(stream)), h)


def aderdg_end(h, dev_Q, t=0.0, stream=None) -> float:
    tt = C.c_double(t)
    _check(load().aderdg_end(h, _ptr(dev_Q), C.byref(tt), _stream(stream)), h)
    return tt.value


def aderdg_get_dt_history(h, cap=1 << 16):
    buf = (C.c_double * cap)()
    n = C.c_int(0)
    _check(load().aderdg_get_dt_history(h, buf, cap, C.byref(n)), h)
    return list(buf[: n.value])


def aderdg_get_stats(h) -> aderdg_stats:
    s = aderdg_stats()
    _check(load().aderdg_get_stats(h, C.byref(s)), h)
    return s


def aderdg_nodes(N):
    xi = (C.c_double * (N + 1))()
    w = (C.c_double * (N + 1))()
    _check(load().aderdg_nodes(N, xi, w))
    return list(xi), list(w)


def aderdg_footprint(h) -> float:
    v = C.c_double(0)
    _check(load().aderdg_footprint(h, C.byref(v)), h)
    return v.value


KERNEL_FUSED, KERNEL_STP, KERNEL_CORRECT, KERNEL_RIEMANN = 0, 1, 2, 3
KERNEL_T1_PREDICT, KERNEL_T1_EXTRAPOLATE, KERNEL_T1_RIEMANN, KERNEL_T1_CORRECT = 4, 5, 6, 7


def aderdg_profile(h, enable=True):
    _check(load().aderdg_profile(h, 1 if enable else 0), h)


def aderdg_profile_read(h, kernel):
    """(summed milliseconds, launches) of one kernel since the last read."""
    ms = C.c_double(0)
    n = C.c_longlong(0)
    _check(load().aderdg_profile_read(h, int(kernel), C.byref(ms), C.byref(n)), h)
    return ms.value, n.value


def aderdg_fp32_fma_peak(repeats=5, stream=None) -> float:
    """Measured FP32 FMA rate of the current device, TFLOP/s."""
    v = C.c_double(0)
    _check(load().aderdg_fp32_fma_peak(int(repeats), C.byref(v), _stream(stream)))
    return v.value


def aderdg_destroy(h):
    _check(load().aderdg_destroy(h))


def aderdg_step_noalloc(d, N, m, pde, grid, dx, params: aderdg_params | None, dev_mat, dev_Q,
                        nsteps, fixed_dt=0.0, t=0.0, stream=None) -> float:
    """The fused step without a handle and without device allocation (scratch
    in a fixed 16 MiB device array of the library); see include/aderdg.h."""
    L = load()
    g = (C.c_int * 3)(*(list(grid) + [1] * (3 - len(grid))))
    h_ = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx))))
    tt = C.c_double(t)
    st = L.aderdg_step_noalloc(d, N, m, pde, g, h_, C.byref(params) if params is not None else None,
                               _ptr(dev_mat), _ptr(dev_Q), int(nsteps), float(fixed_dt), C.byref(tt),
                               _stream(stream))
    if st != ADERDG_OK:
        raise AderdgError(st, "aderdg_step_noalloc failed (status code only)")
    return tt.value


def aderdg_step_adjoint(h, dev_Q0, nsteps, fixed_dt, dev_recv_pos, dev_obs, dev_gQ0,
                        dev_gmat=None, checkpoint_every=30, stream=None) -> float:
    """Misfit J and its gradients dJ/dQ0 (into dev_gQ0) and dJ/d(rho,cp,cs)
    (into dev_gmat, or None); see include/aderdg.h."""
    J = C.c_double(0)
    R = int(dev_recv_pos.shape[0]) if hasattr(dev_recv_pos, "shape") else 0
    _check(load().aderdg_step_adjoint(h, _ptr(dev_Q0), int(nsteps), float(fixed_dt), _ptr(dev_recv_pos),
                                      R, _ptr(dev_obs), _ptr(dev_gQ0), _ptr(dev_gmat),
                                      int(checkpoint_every), C.byref(J), _stream(stream)), h)
    return J.value


class ReceiverMisfit:
    """torch.autograd.Function factory: J(Q0, mat) with the library's adjoint
    as the backward.  Usage:
        f = ReceiverMisfit(h, nsteps, recv_pos, obs, dt)
        J = f(Q0, mat)      # mat may be None; Q0 and mat are CUDA tensors
        J.backward()        # fills Q0.grad and mat.grad
    """

    def __new__(cls, h, nsteps, recv_pos, obs, fixed_dt=0.0, checkpoint_every=30):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, Q0, mat):
                gQ = torch.empty_like(Q0)
                gm = torch.empty_like(mat) if mat is not None else None
                if mat is not None:
                    aderdg_set_material(h, mat.contiguous())
                J = aderdg_step_adjoint(h, Q0.contiguous(), nsteps, fixed_dt, recv_pos.contiguous(),
                                        obs.contiguous(), gQ, gm, checkpoint_every)
                ctx.save_for_backward(gQ, gm if gm is not None else torch.empty(0))
                ctx.has_mat = mat is not None
                return torch.tensor(J, dtype=torch.float64, device=Q0.device)

            @staticmethod
            def backward(ctx, gJ):
                gQ, gm = ctx.saved_tensors
                s = gJ.to(gQ.dtype)
                return gQ * s, (gm * s.to(gm.dtype) if ctx.has_mat else None)

        return _Fn.apply


BATCH_GRAPH, BATCH_PERSISTENT, BATCH_PER_SCENARIO = 0, 1, 2


def scenario(pde, N, grid, dx=None, pde_const=(), cfl=0.0):
    """An aderdg_scenario for a 2D problem."""
    sc = aderdg_scenario()
    pid = PDE_IDS[pde] if isinstance(pde, str) else pde
    sc.d, sc.N = 2, N
    sc.m = {ADVECTION: 1, ACOUSTICS: 3, EULER: 4, ELASTICITY: 5}[pid]
    sc.pde = pid
    sc.grid[:] = [grid[0], grid[1], 1]
    dx = dx or (1.0 / grid[0], 1.0 / grid[1])
    sc.dx[:] = [dx[0], dx[1], 1.0]
    sc.pde_const[:] = list(pde_const) + [0.0] * (8 - len(pde_const))
    sc.cfl = cfl
    return sc


def aderdg_batch_create(scenarios):
    arr = (aderdg_scenario * len(scenarios))(*scenarios)
    out = C.c_void_p()
    st = load().aderdg_batch_create(len(scenarios), arr, C.byref(out))
    if st != ADERDG_OK:
        raise AderdgError(st, "aderdg_batch_create failed")
    return out.value


def aderdg_batch_offsets(b, count):
    off = (C.c_longlong * (count + 1))()
    if load().aderdg_batch_offsets(b, off) != ADERDG_OK:
        raise AderdgError(ADERDG_EINVAL, "aderdg_batch_offsets failed")
    return list(off)


def aderdg_batch_step(b, dev_Q, nsteps, mode=BATCH_GRAPH, stream=None):
    st = load().aderdg_batch_step(b, _ptr(dev_Q), int(nsteps), int(mode), _stream(stream))
    if st != ADERDG_OK:
        raise AderdgError(st, "aderdg_batch_step failed")


def aderdg_batch_autotune(b, dev_Q, steps=4, stream=None):
    st = load().aderdg_batch_autotune(b, _ptr(dev_Q), int(steps), _stream(stream))
    if st != ADERDG_OK:
        raise AderdgError(st, "aderdg_batch_autotune failed")


def aderdg_batch_get_tuning(b):
    bps, tpi, n = C.c_int(0), C.c_int(0), C.c_longlong(0)
    load().aderdg_batch_get_tuning(b, C.byref(bps), C.byref(tpi), C.byref(n))
    return bps.value, tpi.value, n.value


def aderdg_batch_profile(b, enable=True):
    load().aderdg_batch_profile(b, int(bool(enable)))


def aderdg_batch_profile_read(b):
    ms, n = C.c_double(0.0), C.c_longlong(0)
    st = load().aderdg_batch_profile_read(b, C.byref(ms), C.byref(n))
    if st != ADERDG_OK:
        raise AderdgError(st, "aderdg_batch_profile_read failed")
    return ms.value, n.value


def aderdg_batch_destroy(b):
    load().aderdg_batch_destroy(b)


def aderdg_last_error(h=None) -> str:
    return load().aderdg_last_error(h).decode()


def params(pde_const=(), cfl=0.0, picard_iters=0, precision="fp32", form="fused",
           dt_policy=DT_STRICT, predictor=PREDICT_AUTO, inject_step=0, inject_factor=1.0,
           material_jumps=JUMPS_PER_CELL_FLUX):
    """Build an aderdg_params from Python values (names as in the header)."""
    p = aderdg_params()
    vals = list(pde_const) + [0.0] * (8 - len(pde_const))
    p.pde_const[:] = vals
    p.cfl = cfl
    p.picard_iters = picard_iters
    p.precision = PREC_IDS[precision] if isinstance(precision, str) else precision
    p.form = FORM_IDS[form] if isinstance(form, str) else form
    p.dt_policy = dt_policy
    p.predictor = predictor
    p.inject_step = inject_step
    p.inject_factor = inject_factor
    p.material_jumps = material_jumps
    return p
