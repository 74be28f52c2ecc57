"""Python access to the FP64 CPU oracle (``aderdg_oracle.c``).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The CUDA product path
never does.

The oracle is plain C compiled with gcc (OpenMP over cells).  It computes
nodal Gauss-Legendre ADER-DG (Eqs. 2-4, Table 1) in the straightforward order
of Algorithm 1 (left), and the shifted optimistic order of Algorithm 2 for the
time-step control.  Every array crossing this interface is float64 and
C-contiguous; states are laid out ``Q[cell][comp][node]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aderdg_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

ADVECTION, ACOUSTICS, EULER, ELASTICITY = 0, 1, 2, 3
PDE_NAMES = {"advection": ADVECTION, "acoustics": ACOUSTICS, "euler": EULER,
             "elasticity": ELASTICITY}
MAXN = 9

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (host-independent flags, no -march)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp",
                               "-fPIC", "-shared", SRC, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Source(C.Structure):
    """A point source a s(t) delta(x - pos) (the delta terms of Eq. 1);
    kind 0: s(t) = sum_p coef[p] (t - t0)^p, kind 1: Ricker wavelet of peak
    frequency f0 centred at t0."""
    _fields_ = [("pos", C.c_double * 3), ("amp", C.c_double * 9), ("kind", C.c_int), ("pad_", C.c_int),
                ("t0", C.c_double), ("f0", C.c_double), ("coef", C.c_double * 8)]


def source(pos, amp, kind=0, t0=0.0, f0=0.0, coef=()):
    s = Source()
    s.pos[:] = list(pos) + [0.0] * (3 - len(pos))
    s.amp[:] = list(amp) + [0.0] * (9 - len(amp))
    s.kind, s.t0, s.f0 = int(kind), float(t0), float(f0)
    s.coef[:] = list(coef) + [0.0] * (8 - len(coef))
    return s


class Cfg(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int), ("m", C.c_int), ("pde", C.c_int),
                ("grid", C.c_int * 3), ("dx", C.c_double * 3), ("cst", C.c_double * 8),
                ("mat", C.POINTER(C.c_double)), ("picard", C.c_int), ("cfl", C.c_double),
                ("ncp", C.c_int), ("nsrc", C.c_int), ("src", C.POINTER(Source))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.orc_gauss_legendre.argtypes = [C.c_int, dp, dp]
            L.orc_operators.argtypes = [C.c_int] + [dp] * 8
            L.orc_lagrange_eval.argtypes = [C.c_int, C.c_double, dp]
            L.orc_num_vars.argtypes = [C.c_int, C.c_int]
            L.orc_flux_point.argtypes = [C.POINTER(Cfg), C.c_long, dp, C.c_int, dp]
            L.orc_speed_point.argtypes = [C.POINTER(Cfg), C.c_long, dp, C.c_int]
            L.orc_speed_point.restype = C.c_double
            L.orc_lambda.argtypes = [C.POINTER(Cfg), dp, dp]
            L.orc_dt_admissible.argtypes = [C.POINTER(Cfg), C.c_double]
            L.orc_dt_admissible.restype = C.c_double
            L.orc_run.argtypes = [C.POINTER(Cfg), dp, C.c_int, dp, C.c_double, dp, dp,
                                  C.POINTER(C.c_int)]
            L.orc_run_shifted.argtypes = [C.POINTER(Cfg), dp, C.c_int, C.c_int, C.c_double,
                                          C.c_int, C.c_double, dp, C.POINTER(C.c_int), dp]
            L.orc_step_cells.argtypes = [C.POINTER(Cfg), dp, C.c_double, C.c_double,
                                         C.POINTER(C.c_long), C.c_long, dp]
            L.orc_predict.argtypes = [C.POINTER(Cfg), C.c_long, dp, C.c_double, C.c_double, dp,
                                      C.POINTER(C.c_int)]
            L.orc_source_weights.argtypes = [C.POINTER(Cfg), C.c_int, dp]
            L.orc_source_weights.restype = C.c_long
            L.orc_source_time.argtypes = [C.POINTER(Cfg), C.c_int, C.c_double]
            L.orc_source_time.restype = C.c_double
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_receivers.argtypes = [C.POINTER(Cfg), dp, dp, C.c_int, C.POINTER(C.c_int), C.c_int, dp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int = 0) -> int:
    """Set (n > 0) and return the number of OpenMP threads the oracle uses."""
    return lib().orc_set_threads(int(n))


def num_vars(pde: int, d: int) -> int:
    return lib().orc_num_vars(pde, d)


def gauss_legendre(N: int):
    n = N + 1
    xi, w = np.zeros(n), np.zeros(n)
    rc = lib().orc_gauss_legendre(N, _p(xi), _p(w))
    assert rc == 0
    return xi, w


def operators(N: int) -> dict:
    n = N + 1
    out = {k: np.zeros(n) for k in ("xi", "w", "FL", "FR")}
    out.update({k: np.zeros((n, n)) for k in ("Dm", "K1", "K1inv", "Kvol")})
    rc = lib().orc_operators(N, _p(out["xi"]), _p(out["w"]), _p(out["Dm"]), _p(out["FL"]),
                             _p(out["FR"]), _p(out["K1"]), _p(out["K1inv"]), _p(out["Kvol"]))
    assert rc == 0
    return out


def lagrange_eval(N: int, x: float) -> np.ndarray:
    phi = np.zeros(N + 1)
    assert lib().orc_lagrange_eval(N, float(x), _p(phi)) == 0
    return phi


class Problem:
    """Problem description mirrored into the oracle's ``orc_cfg``."""

    def __init__(self, d, N, pde, grid, dx, cst=(), mat=None, picard=None, cfl=0.9, ncp=False,
                 sources=()):
        self.d, self.N, self.pde = int(d), int(N), int(pde)
        self.m = num_vars(self.pde, self.d)
        self.grid = tuple(int(g) for g in grid) + (1,) * (3 - len(grid))
        self.dx = tuple(float(h) for h in dx) + (1.0,) * (3 - len(dx))
        self.cst = tuple(float(c) for c in cst) + (0.0,) * (8 - len(cst))
        self.mat = None if mat is None else _f64(mat).reshape(-1, 3)
        self.picard = (self.N + 1) if picard is None else int(picard)
        self.cfl = float(cfl)
        self.ncp = bool(ncp)
        self.sources = list(sources)
        self._src = (Source * max(1, len(self.sources)))(*self.sources)
        self.n = self.N + 1
        self.NS = self.n ** self.d
        self.C = int(np.prod(self.grid[: self.d]))

    def cfg(self) -> Cfg:
        c = Cfg()
        c.d, c.N, c.m, c.pde = self.d, self.N, self.m, self.pde
        c.grid[:] = list(self.grid)
        c.dx[:] = list(self.dx)
        c.cst[:] = list(self.cst)
        c.mat = _p(self.mat) if self.mat is not None else None
        c.picard = self.picard
        c.cfl = self.cfl
        c.ncp = 1 if self.ncp else 0
        c.nsrc = len(self.sources)
        c.src = C.cast(self._src, C.POINTER(Source)) if self.sources else None
        return c

    def zeros(self):
        return np.zeros((self.C, self.m, self.NS))


def run(P: Problem, Q, nsteps, dt_seq=None, fixed_dt=0.0, t=0.0):
    """Algorithm 1 (left) for nsteps; returns (Q, dt_used, t, max_picard)."""
    Q = _f64(Q).copy()
    cfg = P.cfg()
    dts = np.zeros(max(nsteps, 1))
    seq = None if dt_seq is None else _f64(dt_seq)
    tt = np.array([t], dtype=np.float64)
    mi = C.c_int(0)
    rc = lib().orc_run(C.byref(cfg), _p(Q), int(nsteps), None if seq is None else _p(seq),
                       float(fixed_dt), _p(dts), _p(tt), C.byref(mi))
    if rc:
        raise RuntimeError(f"oracle run failed: status {rc}")
    return Q, dts[:nsteps], float(tt[0]), mi.value


def run_shifted(P: Problem, Q, nsteps, policy=0, fixed_dt=0.0, inject_step=0,
                inject_factor=1.0, t=0.0):
    """Algorithm 2 order with optimistic control; returns (Q, dt_used, reruns, t)."""
    Q = _f64(Q).copy()
    cfg = P.cfg()
    dts = np.zeros(max(nsteps, 1))
    tt = np.array([t], dtype=np.float64)
    nre = C.c_int(0)
    rc = lib().orc_run_shifted(C.byref(cfg), _p(Q), int(nsteps), int(policy), float(fixed_dt),
                               int(inject_step), float(inject_factor), _p(dts), C.byref(nre),
                               _p(tt))
    if rc:
        raise RuntimeError(f"oracle shifted run failed: status {rc}")
    return Q, dts[:nsteps], nre.value, float(tt[0])


def step_cells(P: Problem, Q, dt, cells, t=0.0):
    """One Algorithm-1 step (starting at time t) for the listed cells only;
    returns [len(cells)][m][NS]."""
    Q = _f64(Q)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), P.m, P.NS))
    cfg = P.cfg()
    rc = lib().orc_step_cells(C.byref(cfg), _p(Q), float(dt), float(t),
                              cells.ctypes.data_as(C.POINTER(C.c_long)), len(cells), _p(out))
    if rc:
        raise RuntimeError(f"oracle step_cells failed: status {rc}")
    return out


def predict(P: Problem, u, dt, cell=0, t=0.0):
    """Eq. 3 for one cell over the step [t, t + dt]; returns (qhat[k][comp][node],
    picard iterations)."""
    u = _f64(u)
    qh = np.zeros((P.n, P.m, P.NS))
    it = C.c_int(0)
    cfg = P.cfg()
    rc = lib().orc_predict(C.byref(cfg), int(cell), _p(u), float(dt), float(t), _p(qh), C.byref(it))
    if rc:
        raise RuntimeError(f"oracle predict failed: status {rc}")
    return qh, it.value


def lam(P: Problem, Q) -> float:
    Q = _f64(Q)
    out = np.zeros(1)
    cfg = P.cfg()
    rc = lib().orc_lambda(C.byref(cfg), _p(Q), _p(out))
    if rc:
        raise RuntimeError(f"oracle lambda failed: status {rc}")
    return float(out[0])


def dt_admissible(P: Problem, lam_max: float) -> float:
    cfg = P.cfg()
    return lib().orc_dt_admissible(C.byref(cfg), float(lam_max))


def flux_point(P: Problem, q, j, cell=0):
    q = _f64(q)
    f = np.zeros(P.m)
    cfg = P.cfg()
    lib().orc_flux_point(C.byref(cfg), int(cell), _p(q), int(j), _p(f))
    return f


def speed_point(P: Problem, q, j, cell=0) -> float:
    q = _f64(q)
    cfg = P.cfg()
    return lib().orc_speed_point(C.byref(cfg), int(cell), _p(q), int(j))


# ---------------------------------------------------------------------------
# Receiver misfit and its gradient (definition-level, for the adjoint tests)

def source_weights(P: Problem, k: int):
    """(cell, nodal weights [NS]) of point source k: sigma_{c,i} = amp_c w[i]."""
    pw = np.zeros(P.NS)
    cfg = P.cfg()
    cell = lib().orc_source_weights(C.byref(cfg), int(k), _p(pw))
    return int(cell), pw


def source_time(P: Problem, k: int, t: float) -> float:
    cfg = P.cfg()
    return lib().orc_source_time(C.byref(cfg), int(k), float(t))


def receiver_comps(P: Problem):
    """State components recorded by a receiver: the velocity (acoustics,
    elasticity) or the advected scalar."""
    if P.pde == ADVECTION:
        return [0]
    if P.pde == ACOUSTICS:
        return list(range(1, P.d + 1))
    if P.pde == ELASTICITY:
        vo = 6 if P.d == 3 else 3
        return list(range(vo, vo + P.d))
    raise ValueError("no receivers for this PDE")


def receivers(P: Problem, Q, pos):
    Q = _f64(Q)
    pos = _f64(pos)
    comps = receiver_comps(P)
    R = pos.shape[0]
    out = np.zeros((R, len(comps)))
    cc = (C.c_int * len(comps))(*comps)
    cfg = P.cfg()
    rc = lib().orc_receivers(C.byref(cfg), _p(Q), _p(pos), R, cc, len(comps), _p(out))
    if rc:
        raise RuntimeError(f"oracle receivers failed: status {rc}")
    return out


def trajectory(P: Problem, Q0, nsteps, dt, pos):
    """Receiver traces u_r(Q^k), k = 1..nsteps, of fixed-step straightforward
    stepping (Algorithm 1); returns [nsteps][R][nc]."""
    Q = _f64(Q0).copy()
    out = []
    for _ in range(nsteps):
        Q, _, _, _ = run(P, Q, 1, fixed_dt=dt)
        out.append(receivers(P, Q, pos))
    return np.array(out)


def misfit(P: Problem, Q0, nsteps, dt, pos, obs):
    """J = 1/2 sum_k sum_r |u_r(Q^k) - d_r^k|^2 dt."""
    tr = trajectory(P, Q0, nsteps, dt, pos)
    return 0.5 * dt * float(((tr - obs) ** 2).sum())


def grad_q0_tangent(P: Problem, Q0, nsteps, dt, pos, obs):
    """dJ/dQ0 exactly, by tangent runs: for linear PDEs the step is linear in
    Q, so the derivative along a unit vector e is dt sum_k <B S^k e, B S^k Q0 - d>."""
    res = trajectory(P, Q0, nsteps, dt, pos) - obs
    g = np.zeros_like(_f64(Q0))
    flat = g.reshape(-1)
    for e in range(flat.size):
        E = np.zeros_like(flat)
        E[e] = 1.0
        te = trajectory(P, E.reshape(g.shape), nsteps, dt, pos)
        flat[e] = dt * float((te * res).sum())
    return g


def grad_material_fd(P: Problem, Q0, nsteps, dt, pos, obs, h=1e-4):
    """dJ/d(rho, cp, cs) per cell by central differences with one Richardson
    step (error O(h^4)); P must carry a per-cell material."""
    base = P.mat.copy()
    g = np.zeros_like(base)

    def J(mat):
        Pm = Problem(P.d, P.N, P.pde, P.grid[: P.d], P.dx[: P.d], cst=P.cst, mat=mat,
                     picard=P.picard, cfl=P.cfl, ncp=P.ncp, sources=P.sources)
        return misfit(Pm, Q0, nsteps, dt, pos, obs)

    for c in range(base.shape[0]):
        for k in range(3):
            def D(hh):
                mp, mm = base.copy(), base.copy()
                mp[c, k] += hh * base[c, k]
                mm[c, k] -= hh * base[c, k]
                return (J(mp) - J(mm)) / (2 * hh * base[c, k])
            g[c, k] = (4 * D(h / 2) - D(h)) / 3
    return g
