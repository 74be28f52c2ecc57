"""Pins of the oracle's two terms of Eq. 1 beyond the conservative flux.

Non-conservative products B_j(x) dQ/dx_j (heterogeneous elasticity, Sec. 1:
the B_i anticipate material parameter changes), with the path-conservative
Rusanov fluctuations at material jumps:
  * with a uniform material the strong volume term plus fluctuations is the
    conservative scheme (the two are one discretisation of one PDE);
  * a state with the same velocity and stress everywhere is steady for the
    physical interface conditions (v and the traction continuous): the
    path-conservative scheme keeps it to round-off, the per-cell flux does not;
  * a plane P wave meeting a planar impedance jump splits into the reflected
    and transmitted pulses of the closed-form coefficients
    R = (Z1 - Z2)/(Z1 + Z2), T = 2 Z1/(Z1 + Z2) (Z = rho cp), at the order
    N + 1 of the scheme; the per-cell flux converges to other coefficients.
Point sources a s(t) delta(x - x_s) (the delta terms of Eq. 1):
  * with a zero flux the state changes by the lumped projection of the delta
    times the time integral of s; tested against polynomials p of degree <= N
    per axis (sum_i W_i dx^d dQ_i p(x_i) = a p(x_s) int s dt, exact), and the
    GL time quadrature is exact up to degree 2N+1 in t and not at 2N+2;
  * in a periodic domain the integral of every component grows by exactly
    a_c int s dt (conservation of the flux part);
  * the predictor's time polynomial with a source is u + sigma int_0^tau s
    (exact for s of degree <= N-1).
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from tests.helpers import coords, total, weights_nd

ADV, ACO, ELA = orc.ADVECTION, orc.ACOUSTICS, orc.ELASTICITY


def _random_state(P, seed):
    rng = np.random.default_rng(seed)
    X = coords(P)
    L = np.array(P.grid[: P.d]) * np.array(P.dx[: P.d])
    Q = np.zeros((P.C, P.m, P.NS))
    for c in range(P.m):
        for _ in range(3):
            k = rng.integers(-2, 3, size=P.d)
            Q[:, c] += rng.standard_normal() * np.cos(2 * math.pi * ((X / L) @ k) + rng.random() * 6.28)
    return Q


def _material(C, seed, uniform=False):
    rng = np.random.default_rng(seed)
    if uniform:
        mat = np.tile([2.4, 5.1, 5.1 / math.sqrt(3)], (C, 1))
    else:
        mat = np.stack([rng.uniform(2, 3, C), rng.uniform(4, 6, C), np.zeros(C)], 1)
        mat[:, 2] = mat[:, 1] / math.sqrt(3) * rng.uniform(0.9, 1.0, C)
    return mat


# --------------------------------------------------------------------------
# non-conservative material jumps

@pytest.mark.parametrize("d,N,grid", [(2, 3, (5, 4)), (3, 2, (3, 4, 2))])
def test_ncp_equals_conservative_for_a_uniform_material(d, N, grid):
    C = int(np.prod(grid))
    dx = tuple(1.0 / g for g in grid)
    mat = _material(C, 1, uniform=True)
    Pc = orc.Problem(d, N, ELA, grid, dx, mat=mat, cfl=0.5)
    Pn = orc.Problem(d, N, ELA, grid, dx, mat=mat, cfl=0.5, ncp=True)
    Q0 = _random_state(Pc, 2)
    Qc, dtc, _, _ = orc.run(Pc, Q0, 3)
    Qn, dtn, _, _ = orc.run(Pn, Q0, 3)
    np.testing.assert_array_equal(dtc, dtn)
    assert np.abs(Qn - Qc).max() <= 1e-13 * np.abs(Qc).max()
    assert np.abs(Qc - Q0).max() > 1e-2 * np.abs(Q0).max()


@pytest.mark.parametrize("d", [2, 3])
def test_ncp_keeps_continuous_velocity_and_stress_steady(d):
    """v and sigma equal everywhere across random material jumps: the physical
    system has d Q/dt = 0.  The per-cell flux F_j = -A_j(cell) Q jumps with the
    material at every face and moves the state."""
    grid = (4, 3) if d == 2 else (3, 2, 3)
    C = int(np.prod(grid))
    dx = tuple(1.0 / g for g in grid)
    mat = _material(C, 3)
    Pn = orc.Problem(d, 2, ELA, grid, dx, mat=mat, cfl=0.5, ncp=True)
    Pc = orc.Problem(d, 2, ELA, grid, dx, mat=mat, cfl=0.5)
    rng = np.random.default_rng(4)
    q = rng.standard_normal(Pn.m)
    Q0 = np.broadcast_to(q[None, :, None], (Pn.C, Pn.m, Pn.NS)).copy()
    dt = 0.5 * orc.dt_admissible(Pn, orc.lam(Pn, Q0))
    Qn, _, _, _ = orc.run(Pn, Q0, 4, fixed_dt=dt)
    Qc, _, _, _ = orc.run(Pc, Q0, 4, fixed_dt=dt)
    assert np.abs(Qn - Q0).max() <= 1e-13 * np.abs(q).max()
    assert np.abs(Qc - Q0).max() > 1e-3 * np.abs(q).max()


def _interface_run(ncp, G, N=3, T=0.5):
    """2D elasticity on a (G, 1) periodic grid of length 2 in x: material 1
    (rho = cp = 1) and material 2 (rho = cp = 2) on [0.6, 1.9).  A right-going
    Gaussian P pulse (v_x = f, sigma_xx = -Z1 f, sigma_yy = -(lambda1/cp1) f)
    centred at 0.3 meets the jump at 0.6; at T = 0.5 the reflected pulse is
    centred at 0.4 and the transmitted one at 1.0, both clear of the jumps.
    Returns the relative L2 error of v_x against the closed form."""
    L = 2.0
    dx = (L / G, 0.05)
    xc = (np.arange(G) + 0.5) * dx[0]
    two = (xc >= 0.6) & (xc < 1.9)
    rho = np.where(two, 2.0, 1.0)
    cp = np.where(two, 2.0, 1.0)
    mat = np.stack([rho, cp, cp / 2], 1)
    P = orc.Problem(2, N, ELA, (G, 1), dx, mat=mat, cfl=0.6, ncp=ncp)
    x = coords(P)[..., 0]
    sw = 0.04

    def f(z):
        return np.exp(-((z - 0.3) ** 2) / (2 * sw * sw))

    lam1 = 1.0 * 1.0 - 2 * 1.0 * 0.5 ** 2
    Q0 = np.zeros((P.C, P.m, P.NS))
    Q0[:, 3] = f(x)
    Q0[:, 0] = -1.0 * f(x)
    Q0[:, 1] = -lam1 / 1.0 * f(x)
    K = int(math.ceil(T / (0.6 * dx[0] / (2 * (2 * N + 1) * 2.0))))
    Q, _, _, _ = orc.run(P, Q0, K, fixed_dt=T / K)
    Z1, Z2, c1, c2, x0 = 1.0, 4.0, 1.0, 2.0, 0.6
    R, Tr = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)
    exact = np.where(x < x0, f(x - c1 * T) + R * f(2 * x0 - x - c1 * T),
                     Tr * f(x0 + (c1 / c2) * (x - x0) - c1 * T))
    W = weights_nd(N, 2)
    return math.sqrt(((Q[:, 3] - exact) ** 2 * W).sum() / (exact ** 2 * W).sum())


def test_ncp_reflection_and_transmission_at_an_impedance_jump():
    e80 = _interface_run(True, 80)
    e160 = _interface_run(True, 160)
    assert e160 < 1e-4, e160
    assert e80 / e160 > 2 ** 3.5, (e80, e160)        # order N + 1 = 4
    # the per-cell flux converges to continuity of A_j Q instead: wrong pulses
    assert _interface_run(False, 80) > 0.5


# --------------------------------------------------------------------------
# point sources

def _poly_source(P, pos, amp, coef, t0=0.0):
    return orc.source(pos, amp, kind=0, t0=t0, coef=coef)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_source_projection_and_time_integral_with_zero_flux(N):
    d, grid, dx = 2, (3, 4), (0.5, 0.25)
    rng = np.random.default_rng(N)
    pos = (0.83, 0.61)
    amp = (1.7,)
    deg = 2 * N + 1
    coef = rng.standard_normal(deg + 1)
    src = _poly_source(None, pos, amp, coef, t0=0.05)
    P = orc.Problem(d, N, ADV, grid, dx, cst=(0.0, 0.0), sources=[src])
    Q0 = _random_state(P, 5)[:, :1]
    dt, K, t = 0.07, 3, 0.2
    Q, _, t1, _ = orc.run(P, Q0, K, fixed_dt=dt, t=t)
    # int_t^{t1} s: exact antiderivative of the polynomial in (t - t0)
    anti = np.polynomial.polynomial.polyint(coef)
    S = np.polynomial.polynomial.polyval(t1 - 0.05, anti) - np.polynomial.polynomial.polyval(t - 0.05, anti)
    X = coords(P)
    W = weights_nd(N, d) * float(np.prod(dx))
    for px in range(N + 1):
        for py in range(N + 1):
            p = X[..., 0] ** px * X[..., 1] ** py
            lhs = float(((Q[:, 0] - Q0[:, 0]) * p * W[None, :]).sum())
            rhs = amp[0] * pos[0] ** px * pos[1] ** py * S
            assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (px, py, lhs, rhs)
    # one degree more in time is beyond the Gauss rule of the update (time
    # functions keep eight coefficients: degree 7 at most)
    if deg + 1 > 7:
        return
    coef2 = np.zeros(deg + 2)
    coef2[-1] = 1.0
    P2 = orc.Problem(d, N, ADV, grid, dx, cst=(0.0, 0.0), sources=[_poly_source(None, pos, amp, coef2)])
    Q2, _, t2, _ = orc.run(P2, np.zeros_like(Q0), 1, fixed_dt=dt, t=t)
    S2 = (t2 ** (deg + 2) - t ** (deg + 2)) / (deg + 2)
    got = float((Q2[:, 0] * W[None, :]).sum())
    assert abs(got - amp[0] * S2) > 1e-10 * abs(amp[0] * S2)


@pytest.mark.parametrize("pde,d,N", [(ACO, 2, 3), (ELA, 3, 2), (ELA, 2, 2)])
def test_source_adds_exactly_its_integral_to_every_component(pde, d, N):
    grid = (5, 4) if d == 2 else (3, 3, 2)
    dx = tuple(1.0 / g for g in grid)
    cst = (1.2, 0.9) if pde == ACO else (2.5, 5.0, 5.0 / math.sqrt(3))
    m = orc.num_vars(pde, d)
    rng = np.random.default_rng(7)
    coef = rng.standard_normal(2 * N + 2)
    srcs = [orc.source(rng.uniform(0, 1, d), rng.standard_normal(m), kind=0, t0=0.01, coef=coef),
            orc.source(rng.uniform(0, 1, d), rng.standard_normal(m), kind=0, t0=-0.02, coef=coef[::-1])]
    P = orc.Problem(d, N, pde, grid, dx, cst=cst, cfl=0.5, sources=srcs)
    Q0 = _random_state(P, 8)
    Q, dts, t1, _ = orc.run(P, Q0, 4)
    grow = np.zeros(m)
    anti = np.polynomial.polynomial.polyint
    for s, c0, t0 in ((srcs[0], coef, 0.01), (srcs[1], coef[::-1], -0.02)):
        a = anti(c0)
        S = np.polynomial.polynomial.polyval(t1 - t0, a) - np.polynomial.polynomial.polyval(0.0 - t0, a)
        grow += np.array(s.amp[:m]) * S
    np.testing.assert_allclose(total(P, Q) - total(P, Q0), grow, rtol=0, atol=1e-12 * np.abs(grow).max())


@pytest.mark.parametrize("N", [2, 3, 4])
def test_predictor_with_a_source_integrates_it_in_time(N):
    """Zero flux: d q / d tau = dt sigma s(t + tau dt), so q(tau) = u + sigma
    dt int_0^tau s, a polynomial of degree deg(s) + 1 <= N in time."""
    dx = (0.3, 0.2)
    rng = np.random.default_rng(20 + N)
    coef = rng.standard_normal(N)            # degree N - 1
    src = orc.source((0.11, 0.07), (2.3,), kind=0, t0=0.4, coef=coef)
    P = orc.Problem(2, N, ADV, (1, 1), dx, cst=(0.0, 0.0), sources=[src])
    u = rng.standard_normal((1, P.NS))
    t, dt = 0.35, 0.1
    qh, _ = orc.predict(P, u, dt, t=t)
    cell, pw = orc.source_weights(P, 0)
    assert cell == 0
    xi, _ = orc.gauss_legendre(N)
    anti = np.polynomial.polynomial.polyint(coef)
    for k in range(N + 1):
        S = (np.polynomial.polynomial.polyval(t + xi[k] * dt - 0.4, anti) -
             np.polynomial.polynomial.polyval(t - 0.4, anti))
        np.testing.assert_allclose(qh[k, 0], u[0] + 2.3 * pw * S, rtol=0, atol=1e-12)


def test_source_weights_reproduce_the_delta_and_clamp():
    """The nodal weights are the lumped-mass projection of the delta: tested
    against the Lagrange polynomials themselves, and a position outside the
    grid lands in the boundary cell."""
    N, grid, dx = 3, (4, 3), (0.25, 0.5)
    src = orc.source((2.0, -0.3), (1.0,), kind=1, t0=0.0, f0=3.0)
    P = orc.Problem(2, N, ADV, grid, dx, cst=(0.0, 0.0), sources=[src])
    cell, pw = orc.source_weights(P, 0)
    assert cell == 3                          # x clamped to column 3, y to row 0
    W = weights_nd(N, 2) * float(np.prod(dx))
    xi, _ = orc.gauss_legendre(N)
    loc = (2.0 / 0.25 - 3, -0.3 / 0.5)        # local coordinates, extrapolated
    for i in range(P.NS):
        want = orc.lagrange_eval(N, loc[0])[i % 4] * orc.lagrange_eval(N, loc[1])[i // 4]
        assert abs(W[i] * pw[i] - want) < 1e-13 * max(1.0, abs(want))
    # the Ricker wavelet: peak 1 at t0, zeros at t0 +- 1/(sqrt(2) pi f0)
    assert abs(orc.source_time(P, 0, 0.0) - 1.0) < 1e-15
    assert abs(orc.source_time(P, 0, 1 / (math.sqrt(2) * math.pi * 3.0))) < 1e-15
