"""Seeded synthetic workloads: problem sizes, random draws and analytic fields.

This module holds no part of the numerical method.  It produces
  * the problem descriptions of the five workloads (grid, order, PDE, sizes),
  * every random number the workloads use, from one counter-based generator
    (splitmix64, Steele/Lea/Flood 2014), and
  * analytic initial fields evaluated at physical points.
Node positions inside a cell (the Gauss-Legendre points) are supplied by the
caller: the CUDA library and the CPU oracle each compute their own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive outputs of splitmix64 started at ``seed`` (uint64)."""
    z0 = np.uint64(seed & MASK64)
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z0 + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal draws by Box-Muller on pairs of uniforms."""
    u = uniform(seed, 2 * count).reshape(count, 2)
    u1 = np.maximum(u[:, 0], 1e-300)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u[:, 1])


# ---------------------------------------------------------------------------
# Problem descriptions

PDE_IDS = {"advection": 0, "acoustics": 1, "euler": 2, "elasticity": 3}


def num_vars(pde: str, d: int) -> int:
    return {"advection": 1, "acoustics": d + 1, "euler": d + 2,
            "elasticity": 9 if d == 3 else 5}[pde]


@dataclass
class Workload:
    name: str
    pde: str
    d: int
    N: int
    grid: tuple
    steps: int
    cst: tuple = ()
    precision: str = "fp32"
    seed: int = 0
    extra: dict = field(default_factory=dict)
    cfl: float = 0.0          # C_dT; 0 = the library default 0.9 - 0.1 N

    @property
    def m(self) -> int:
        return num_vars(self.pde, self.d)

    @property
    def cells(self) -> int:
        return int(np.prod(self.grid[: self.d]))

    @property
    def dofs(self) -> int:
        return self.cells * self.m * (self.N + 1) ** self.d

    @property
    def dx(self) -> tuple:
        return tuple(1.0 / g for g in self.grid[: self.d])

    def resized(self, grid, steps=None) -> "Workload":
        w = Workload(self.name, self.pde, self.d, self.N, tuple(grid),
                     self.steps if steps is None else steps, self.cst, self.precision,
                     self.seed, dict(self.extra), self.cfl)
        return w

    @property
    def cfl_value(self) -> float:
        return self.cfl if self.cfl > 0 else default_cfl(self.N)


def default_cfl(N: int) -> float:
    """Safety factor C_dT of dt = C_dT h / (d (2N+1) lambda_max): 0.1 below the
    largest factor measured stable over 400 steps for N = 2..6 (0.8 .. 0.4)."""
    return max(0.3, min(0.9, 0.9 - 0.1 * N))


def advection_2d(grid=(32, 32), N=3, steps=10) -> Workload:
    """2D linear advection, velocity (1, 0.5), init sin(2 pi x) sin(2 pi y), FP64,
    at the stated CFL 0.9 / (d (2N+1))."""
    return Workload("advection2d", "advection", 2, N, tuple(grid), steps,
                    cst=(1.0, 0.5, 0.0), precision="fp64", seed=1, cfl=0.9)


def acoustics_3d(grid=(64, 64, 64), N=5, steps=100, seed=2) -> Workload:
    """3D linear acoustics, rho = c = 1, Gaussian pressure pulse (sigma 0.05)."""
    return Workload("acoustics3d", "acoustics", 3, N, tuple(grid), steps,
                    cst=(1.0, 1.0), precision="fp32", seed=seed, extra={"sigma": 0.05})


def euler_3d(grid=(128, 128, 128), N=3, steps=200, seed=3) -> Workload:
    """3D compressible Euler, gamma 1.4, rho = 1 + 0.1 R(x), p = 1, v = 0."""
    return Workload("euler3d", "euler", 3, N, tuple(grid), steps, cst=(1.4,),
                    precision="fp32_acc64", seed=seed, extra={"amp": 0.1, "kmax": 4})


def elasticity_3d(grid=(96, 96, 96), N=4, steps=300, seed=4) -> Workload:
    """3D linear elasticity with per-cell rho in U[2,3], cp in U[4,6], cs = cp/sqrt(3)."""
    return Workload("elasticity3d", "elasticity", 3, N, tuple(grid), steps,
                    cst=(2.5, 5.0, 5.0 / math.sqrt(3.0)), precision="fp32", seed=seed,
                    extra={"sigma": 0.05, "receivers": 64, "checkpoint_every": 30})


# ---------------------------------------------------------------------------
# Physical coordinates of nodal points

def node_coords(grid, dx, xi, xp=np, device=None):
    """Physical coordinates [C][NS][d] of the nodes of every cell.

    ``xi`` are the 1D node positions in [0,1] (from the caller).  Cell order:
    axis 0 fastest; node order inside a cell: axis 0 fastest.  ``xp`` is numpy
    (default) or torch (then ``device`` places the result, float64).
    """
    d = len(dx)
    n = len(xi)
    cidx = np.indices(tuple(grid[:d])[::-1]).reshape(d, -1)[::-1]      # [d][C], axis 0 fastest
    nidx = np.indices((n,) * d).reshape(d, -1)[::-1]                    # [d][NS]
    xi = np.asarray(xi, dtype=np.float64)
    if xp is np:
        out = np.empty((cidx.shape[1], nidx.shape[1], d))
        for a in range(d):
            out[:, :, a] = (cidx[a][:, None] + xi[nidx[a]][None, :]) * dx[a]
        return out
    cols = []
    for a in range(d):
        ca = xp.as_tensor(cidx[a], dtype=xp.float64, device=device)
        na = xp.as_tensor(xi[nidx[a]], dtype=xp.float64, device=device)
        cols.append((ca[:, None] + na[None, :]) * dx[a])
    return xp.stack(cols, dim=-1)


# ---------------------------------------------------------------------------
# Initial states Q[C][m][NS] (float64) given node coordinates X[C][NS][d]

def init_state(w: Workload, X, xp=np):
    """Initial state Q[C][m][NS] (float64) at node coordinates X[C][NS][d];
    X and the result are numpy arrays, or torch tensors when xp is torch."""
    C, NS, d = X.shape
    if xp is np:
        Q = np.zeros((C, w.m, NS))
        rnd = np.round
    else:
        Q = xp.zeros((C, w.m, NS), dtype=xp.float64, device=X.device)
        rnd = xp.round
    if w.pde == "advection":
        Q[:, 0, :] = xp.sin(2 * math.pi * X[..., 0]) * xp.sin(2 * math.pi * X[..., 1])
        if d == 3:
            Q[:, 0, :] *= xp.sin(2 * math.pi * X[..., 2])
    elif w.pde in ("acoustics", "elasticity"):
        centre = uniform(w.seed, d)
        r2 = 0.0
        for a in range(d):
            ra = X[..., a] - float(centre[a])
            ra = ra - rnd(ra)                       # minimum image on the unit torus
            r2 = r2 + ra * ra
        s = w.extra.get("sigma", 0.05)
        pulse = xp.exp(-r2 / (2 * s * s))
        if w.pde == "acoustics":
            Q[:, 0, :] = pulse
        else:
            vo = 6 if d == 3 else 3
            Q[:, vo + d - 1, :] = pulse
    elif w.pde == "euler":
        R = fourier_field(w.seed, d, w.extra.get("kmax", 4), X, xp)
        rho = 1.0 + w.extra.get("amp", 0.1) * R
        gamma = w.cst[0]
        Q[:, 0, :] = rho
        Q[:, d + 1, :] = 1.0 / (gamma - 1.0)
    return Q


def fourier_modes(seed: int, d: int, kmax: int):
    """Wave vectors k in Z^d with 1 <= |k| <= kmax, amplitudes ~ N(0,1), phases ~ U[0, 2 pi)."""
    rng = range(-kmax, kmax + 1)
    if d == 2:
        ks = [(a, b) for a in rng for b in rng]
    else:
        ks = [(a, b, c) for a in rng for b in rng for c in rng]
    ks = np.array([k for k in ks if 1 <= math.sqrt(sum(x * x for x in k)) <= kmax], dtype=float)
    amp = normal(seed, len(ks))
    phase = 2 * math.pi * uniform(seed + 1, len(ks))
    return ks, amp, phase


def fourier_field(seed: int, d: int, kmax: int, X, xp=np):
    """R(x) = sum_k a_k cos(2 pi k.x + phi_k) / sum_k |a_k|, so |R| <= 1."""
    ks, amp, phase = fourier_modes(seed, d, kmax)
    out = 0.0
    for k, a, p in zip(ks, amp, phase):
        arg = sum(float(k[i]) * X[..., i] for i in range(d))
        out = out + float(a) * xp.cos(2 * math.pi * arg + float(p))
    return out / np.abs(amp).sum()


def materials(w: Workload) -> np.ndarray:
    """Per-cell (rho, cp, cs): rho ~ U[2,3], cp ~ U[4,6], cs = cp / sqrt(3)."""
    u = uniform(w.seed + 7, 2 * w.cells).reshape(w.cells, 2)
    rho = 2.0 + u[:, 0]
    cp = 4.0 + 2.0 * u[:, 1]
    return np.stack([rho, cp, cp / math.sqrt(3.0)], axis=1)


def receivers(w: Workload) -> np.ndarray:
    """Receiver positions ~ U[0,1]^d, [R][d]."""
    R = w.extra.get("receivers", 64)
    return uniform(w.seed + 11, R * w.d).reshape(R, w.d)


def ensemble(seed: int = 5, count: int = 512):
    """Scenarios of the batched 2D ensemble: side ~ U{16..256}, N ~ U{2..6},
    PDE ~ {acoustics (m=3), elasticity (m=5)}."""
    u = uniform(seed, 4 * count).reshape(count, 4)
    out = []
    for s in range(count):
        side = 16 + int(u[s, 0] * 241)
        N = 2 + int(u[s, 1] * 5)
        pde = "acoustics" if u[s, 2] < 0.5 else "elasticity"
        cst = (1.0, 1.0) if pde == "acoustics" else (2.5, 5.0, 5.0 / math.sqrt(3.0))
        out.append(Workload(f"scenario{s}", pde, 2, N, (side, side), 50, cst=cst,
                            precision="fp32", seed=seed * 1000 + s, extra={"sigma": 0.05}))
    return out
