"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against closed forms, exact solutions of the
PDE, brute-force polynomial calculus (numpy), the finite-volume special case
of the appendix (Corollary "FV-Rusanov"), convergence order, conservation,
or a structural identity of the paper (Eq. 5 = Eq. 6 executed in the
orders of Algorithms 1 and 2).  None of them re-types an oracle formula.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.helpers import coords, l2, rel_l2, total

ADV, ACO, EUL, ELA = orc.ADVECTION, orc.ACOUSTICS, orc.EULER, orc.ELASTICITY


# --------------------------------------------------------------------------
# 1D basis (Sec. 3: Lagrange basis on Gauss-Legendre points)

CLOSED = {
    0: ([0.0], [2.0]),
    1: ([-1 / math.sqrt(3), 1 / math.sqrt(3)], [1.0, 1.0]),
    2: ([-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)], [5 / 9, 8 / 9, 5 / 9]),
    3: ([-math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5)), -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)),
         math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))],
        [(18 - math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36,
         (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36]),
    4: ([-math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3, -math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, 0.0,
         math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3],
        [(322 - 13 * math.sqrt(70)) / 900, (322 + 13 * math.sqrt(70)) / 900, 128 / 225,
         (322 + 13 * math.sqrt(70)) / 900, (322 - 13 * math.sqrt(70)) / 900]),
}


@pytest.mark.parametrize("N", sorted(CLOSED))
def test_gauss_legendre_closed_forms(N):
    t, wt = CLOSED[N]
    xi, w = orc.gauss_legendre(N)
    np.testing.assert_allclose(xi, (1 + np.array(t)) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, np.array(wt) / 2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", range(0, 10))
def test_quadrature_exactness(N):
    xi, w = orc.gauss_legendre(N)
    assert abs(w.sum() - 1) < 1e-15
    for p in range(2 * N + 2):
        assert abs((w * xi ** p).sum() - 1 / (p + 1)) < 2e-15, p
    # degree 2N+2 = 2n misses by the Gauss error term -(n!)^4 / ((2n+1) ((2n)!)^2) on [0,1]
    n = N + 1
    miss = (w * xi ** (2 * n)).sum() - 1 / (2 * n + 1)
    want = -math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs(miss - want) < 1e-3 * abs(want) + 1e-16, (miss, want)


def lagrange_poly(xi, a):
    """Coefficients (highest first) of the Lagrange polynomial phi_a, via numpy."""
    others = np.delete(xi, a)
    return np.atleast_1d(np.poly(others)) / np.prod(xi[a] - others)


@pytest.mark.parametrize("N", range(0, 8))
def test_operators_against_polynomial_calculus(N):
    O = orc.operators(N)
    xi, n = O["xi"], N + 1
    for p in range(N + 1):
        vals = xi ** p
        # Dm: exact derivative of a degree <= N polynomial at the nodes
        np.testing.assert_allclose(O["Dm"] @ vals, p * xi ** max(p - 1, 0) * (p > 0), atol=5e-12)
        # FL, FR: interpolation to 0 and 1
        assert abs(O["FL"] @ vals - (1.0 if p == 0 else 0.0)) < 1e-12
        assert abs(O["FR"] @ vals - 1.0) < 1e-12
    # K1 is consistent with a constant in time, K1 inverse is its inverse
    np.testing.assert_allclose(O["K1"] @ np.ones(n), O["FL"], atol=1e-12)
    np.testing.assert_allclose(O["K1inv"] @ O["K1"], np.eye(n), atol=1e-11)
    # Kvol: w_i * (Kvol f)_i = int_0^1 phi_i'(x) f(x) dx for polynomial f (degree <= N)
    rng = np.random.default_rng(N)
    fc = rng.standard_normal(N + 1)
    fvals = np.polyval(fc, xi)
    for i in range(n):
        dphi = np.polyder(lagrange_poly(xi, i))
        integ = np.polyint(np.polymul(dphi, fc))
        exact = np.polyval(integ, 1.0) - np.polyval(integ, 0.0)
        assert abs(O["w"][i] * (O["Kvol"][i] @ fvals) - exact) < 1e-11


# --------------------------------------------------------------------------
# predict (Eq. 3): exact for space-time polynomials inside the test space

def test_predictor_constant_state():
    P = orc.Problem(3, 3, EUL, (1, 1, 1), (0.1, 0.2, 0.3), cst=(1.4,))
    u = np.zeros((P.m, P.NS))
    u[0], u[1], u[2], u[3], u[4] = 1.2, 0.3, -0.2, 0.1, 3.0
    qh, _ = orc.predict(P, u, 0.01)
    np.testing.assert_allclose(qh, np.broadcast_to(u, qh.shape), atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("picard", [None, 0])
def test_predictor_exact_for_translated_polynomial(N, picard):
    """Advection of a total-degree-N polynomial: q(x,t) = u(x - a t) lies in the
    space-time polynomial space, so the predictor reproduces it exactly."""
    a = (1.0, -0.5)
    dx = (0.3, 0.2)
    dt = 0.05
    P = orc.Problem(2, N, ADV, (1, 1), dx, cst=a, picard=picard)
    rng = np.random.default_rng(10 + N)
    terms = [(p, q, rng.standard_normal()) for p in range(N + 1) for q in range(N + 1 - p)]

    def u(x, y):
        return sum(c * x ** p * y ** q for p, q, c in terms)

    X = coords(P)[0]                          # [NS][2]
    qh, _ = orc.predict(P, u(X[:, 0], X[:, 1])[None, :], dt)
    xi, _ = orc.gauss_legendre(N)
    for k in range(N + 1):
        t = dt * xi[k]
        np.testing.assert_allclose(qh[k, 0], u(X[:, 0] - a[0] * t, X[:, 1] - a[1] * t), atol=1e-12)


@pytest.mark.parametrize("N", [2, 3])
def test_predictor_exact_acoustic_plane_wave(N):
    rho, c = 1.3, 0.7
    dx, dt = (0.25, 0.25), 0.08
    P = orc.Problem(2, N, ACO, (1, 1), dx, cst=(rho, c))
    coef = np.random.default_rng(3).standard_normal(N + 1)

    def f(s):
        return np.polyval(coef, s)

    X = coords(P)[0]
    u = np.zeros((3, P.NS))
    u[0] = f(X[:, 0])
    u[1] = f(X[:, 0]) / (rho * c)
    qh, _ = orc.predict(P, u, dt)
    xi, _ = orc.gauss_legendre(N)
    for k in range(N + 1):
        s = X[:, 0] - c * dt * xi[k]
        np.testing.assert_allclose(qh[k, 0], f(s), atol=1e-12)
        np.testing.assert_allclose(qh[k, 1], f(s) / (rho * c), atol=1e-12)
        np.testing.assert_allclose(qh[k, 2], 0.0, atol=1e-12)


# --------------------------------------------------------------------------
# PDE fluxes: Jacobian spectra (numerical Jacobian, numpy eigenvalues)

def jacobian(P, q, j, h=1e-6):
    J = np.zeros((P.m, P.m))
    for b in range(P.m):
        e = np.zeros(P.m)
        e[b] = h
        J[:, b] = (orc.flux_point(P, q + e, j) - orc.flux_point(P, q - e, j)) / (2 * h)
    return J


@pytest.mark.parametrize("d", [2, 3])
def test_euler_flux_spectrum(d):
    P = orc.Problem(d, 1, EUL, (1,) * d, (1,) * d, cst=(1.4,))
    rho, v, p = 1.3, np.array([0.4, -0.7, 0.2][:d]), 0.9
    q = np.concatenate([[rho], rho * v, [p / 0.4 + 0.5 * rho * v @ v]])
    c = math.sqrt(1.4 * p / rho)
    for j in range(d):
        ev = np.sort(np.linalg.eigvals(jacobian(P, q, j)).real)
        want = np.sort([v[j] - c] + [v[j]] * d + [v[j] + c])
        np.testing.assert_allclose(ev, want, atol=1e-6)
        assert abs(orc.speed_point(P, q, j) - (abs(v[j]) + c)) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_elasticity_flux_spectrum(d):
    rho, cp = 2.4, 5.2
    cs = cp / math.sqrt(3)
    P = orc.Problem(d, 1, ELA, (1,) * d, (1,) * d, cst=(rho, cp, cs))
    q = np.random.default_rng(1).standard_normal(P.m)
    for j in range(d):
        ev = np.sort(np.linalg.eigvals(jacobian(P, q, j)).real)
        want = [-cp, cp] + [-cs, cs] * (d - 1) + [0.0] * (P.m - 2 * d)
        np.testing.assert_allclose(ev, np.sort(want), atol=1e-6)
        assert orc.speed_point(P, q, j) == cp


@pytest.mark.parametrize("d", [2, 3])
def test_acoustics_flux_spectrum(d):
    rho, c = 1.7, 0.6
    P = orc.Problem(d, 1, ACO, (1,) * d, (1,) * d, cst=(rho, c))
    q = np.random.default_rng(2).standard_normal(P.m)
    for j in range(d):
        ev = np.sort(np.linalg.eigvals(jacobian(P, q, j)).real)
        np.testing.assert_allclose(ev, np.sort([-c, c] + [0.0] * (d - 1)), atol=1e-6)


# --------------------------------------------------------------------------
# Whole steps

def test_advection_matches_translated_solution():
    """32^2 cells, N=3, a=(1, 0.5), sin 2 pi x sin 2 pi y, 10 steps at the CFL step."""
    w = wl.advection_2d()
    P = orc.Problem(2, w.N, ADV, w.grid, w.dx, cst=w.cst)
    X = coords(P)
    Q0 = wl.init_state(w, X)
    Q, dts, t, _ = orc.run(P, Q0, w.steps)
    assert np.allclose(dts, 0.9 / (2 * 7) / 32)
    exact = np.sin(2 * math.pi * (X[..., 0] - t)) * np.sin(2 * math.pi * (X[..., 1] - 0.5 * t))
    err = l2(P, Q[:, 0] - exact)
    assert err < 2e-6, err


def _order(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def _converge(make, exact, grids, T, cfl_dt):
    errs = []
    for g in grids:
        P = make(g)
        X = coords(P)
        nsteps = int(math.ceil(T / (cfl_dt / g)))
        Q, _, t, _ = orc.run(P, exact(X, 0.0), nsteps, fixed_dt=T / nsteps)
        errs.append(l2(P, Q - exact(X, T)))
    return errs


def test_convergence_order_advection():
    N = 2

    def make(g):
        return orc.Problem(2, N, ADV, (g, g), (1 / g, 1 / g), cst=(1.0, 0.5))

    def exact(X, t):
        return (np.sin(2 * math.pi * (X[..., 0] - t)) * np.cos(2 * math.pi * (X[..., 1] - 0.5 * t)))[:, None, :]

    errs = _converge(make, exact, [8, 16, 32], 0.1, 0.09)
    assert min(_order(errs)) > N + 1 - 0.3, errs


def test_convergence_order_acoustics():
    N, rho, c = 2, 1.0, 1.0

    def make(g):
        return orc.Problem(2, N, ACO, (g, g), (1 / g, 1 / g), cst=(rho, c))

    def exact(X, t):
        ph = 2 * math.pi * (X[..., 0] + X[..., 1]) - c * 2 * math.pi * math.sqrt(2) * t
        p = np.sin(ph)
        v = p / (rho * c) / math.sqrt(2)
        return np.stack([p, v, v], axis=1)

    errs = _converge(make, exact, [8, 16, 32], 0.1, 0.09)
    assert min(_order(errs)) > N + 1 - 0.3, errs


def test_convergence_order_euler_entropy_wave():
    N, g_ = 2, 1.4
    v = (1.0, 0.5)

    def make(g):
        return orc.Problem(2, N, EUL, (g, g), (1 / g, 1 / g), cst=(g_,))

    def exact(X, t):
        rho = 1 + 0.2 * np.sin(2 * math.pi * (X[..., 0] - v[0] * t + X[..., 1] - v[1] * t))
        E = 1.0 / (g_ - 1) + 0.5 * rho * (v[0] ** 2 + v[1] ** 2)
        return np.stack([rho, rho * v[0], rho * v[1], E], axis=1)

    errs = _converge(make, exact, [16, 32, 64], 0.1, 0.09 / 2.3)
    assert min(_order(errs)) > N + 1 - 0.3, errs


def test_convergence_order_elastic_p_wave():
    N, rho, cp = 2, 2.5, 5.0
    cs = cp / math.sqrt(3)
    lam = rho * (cp * cp - 2 * cs * cs)

    def make(g):
        return orc.Problem(2, N, ELA, (g, g), (1 / g, 1 / g), cst=(rho, cp, cs))

    def exact(X, t):
        f = np.sin(2 * math.pi * (X[..., 0] - cp * t))
        z = np.zeros_like(f)
        return np.stack([-rho * cp * f, -(lam / cp) * f, z, f, z], axis=1)

    errs = _converge(make, exact, [8, 16, 32], 0.04, 0.09 / cp)
    assert min(_order(errs)) > N + 1 - 0.3, errs


def test_elastic_s_wave_3d_exact():
    N, rho, cp = 3, 2.5, 5.0
    cs = cp / math.sqrt(3)
    P = orc.Problem(3, N, ELA, (6, 2, 2), (1 / 6, 0.5, 0.5), cst=(rho, cp, cs))
    X = coords(P)

    def exact(t):
        f = np.sin(2 * math.pi * (X[..., 0] - cs * t))
        Q = np.zeros((P.C, 9, P.NS))
        Q[:, 3] = -rho * cs * f   # sigma_xy
        Q[:, 7] = f               # v_y
        return Q

    Q, _, t, _ = orc.run(P, exact(0.0), 8)
    assert rel_l2(P, Q, exact(t)) < 2e-3


@pytest.mark.parametrize("pde,d", [(ADV, 2), (ACO, 2), (ACO, 3), (EUL, 2), (EUL, 3), (ELA, 2), (ELA, 3)])
def test_constant_state_preserved(pde, d):
    cst = {ADV: (1.0, -0.5, 0.25), ACO: (1.2, 0.8), EUL: (1.4,), ELA: (2.5, 5.0, 2.9)}[pde]
    P = orc.Problem(d, 2, pde, (3,) * d, (0.3,) * d, cst=cst)
    state = {ADV: [0.7], ACO: [0.3, 0.1, -0.2, 0.4][: d + 1],
             EUL: [1.1, 0.2, -0.1, 0.05][: d + 1] + [2.7],
             ELA: list(np.linspace(-1, 1, P.m))}[pde]
    Q0 = np.broadcast_to(np.array(state)[None, :, None], (P.C, P.m, P.NS)).copy()
    Q, _, _, _ = orc.run(P, Q0, 3)
    np.testing.assert_allclose(Q, Q0, atol=1e-13)


def test_conservation_euler():
    w = wl.euler_3d(grid=(6, 5), N=2).__class__("e2", "euler", 2, 2, (6, 5), 20, cst=(1.4,),
                                                  seed=9, extra={"amp": 0.1, "kmax": 3})
    P = orc.Problem(2, 2, EUL, w.grid, w.dx, cst=w.cst)
    X = coords(P)
    Q0 = wl.init_state(w, X)
    Q0[:, 1] = 0.3 * np.sin(2 * math.pi * X[..., 1])        # add momentum
    Q0[:, 3] += 0.5 * Q0[:, 1] ** 2 / Q0[:, 0]
    Q, _, _, _ = orc.run(P, Q0, 20)
    np.testing.assert_allclose(total(P, Q), total(P, Q0), rtol=1e-13, atol=1e-14)
    assert np.abs(Q - Q0).max() > 1e-3    # the state did evolve


# --------------------------------------------------------------------------
# Appendix A: p = 0 is first-order finite volumes with Rusanov fluxes

def fv_rusanov(flux, speed, Q, dx, dt, steps):
    """Textbook first-order FV on a periodic grid; Q is [gy][gx][m]."""
    Q = Q.copy()
    for _ in range(steps):
        new = Q.copy()
        for j, ax in ((0, 1), (1, 0)):
            QR = np.roll(Q, -1, axis=ax)
            FL, FR = flux(Q, j), flux(QR, j)
            s = np.maximum(speed(Q, j), speed(QR, j))[..., None]
            Fs = 0.5 * (FL + FR) - 0.5 * s * (QR - Q)
            new -= dt / dx[j] * (Fs - np.roll(Fs, 1, axis=ax))
        Q = new
    return Q


def test_fv_special_case_acoustics():
    rho, c = 1.3, 0.8
    P = orc.Problem(2, 0, ACO, (7, 5), (1 / 7, 1 / 5), cst=(rho, c))
    rng = np.random.default_rng(0)
    Q0 = rng.standard_normal((P.C, 3, 1))

    def flux(Q, j):
        F = np.zeros_like(Q)
        F[..., 0] = rho * c * c * Q[..., 1 + j]
        F[..., 1 + j] = Q[..., 0] / rho
        return F

    def speed(Q, j):
        return np.full(Q.shape[:-1], c)

    Q, _, _, _ = orc.run(P, Q0, 4, fixed_dt=0.01)
    ref = fv_rusanov(flux, speed, Q0[:, :, 0].reshape(5, 7, 3), P.dx, 0.01, 4)
    np.testing.assert_allclose(Q[:, :, 0], ref.reshape(-1, 3), atol=1e-14)


def test_fv_special_case_euler():
    g = 1.4
    P = orc.Problem(2, 0, EUL, (6, 4), (1 / 6, 1 / 4), cst=(g,))
    rng = np.random.default_rng(1)
    rho = 1 + 0.2 * rng.random(P.C)
    v = 0.3 * rng.standard_normal((P.C, 2))
    p = 1 + 0.2 * rng.random(P.C)
    Q0 = np.stack([rho, rho * v[:, 0], rho * v[:, 1], p / (g - 1) + 0.5 * rho * (v ** 2).sum(1)], 1)[..., None]

    def prim(Q):
        r = Q[..., 0]
        u = Q[..., 1:3] / r[..., None]
        pr = (g - 1) * (Q[..., 3] - 0.5 * r * (u ** 2).sum(-1))
        return r, u, pr

    def flux(Q, j):
        r, u, pr = prim(Q)
        F = np.empty_like(Q)
        F[..., 0] = r * u[..., j]
        F[..., 1] = r * u[..., j] * u[..., 0] + (pr if j == 0 else 0)
        F[..., 2] = r * u[..., j] * u[..., 1] + (pr if j == 1 else 0)
        F[..., 3] = u[..., j] * (Q[..., 3] + pr)
        return F

    def speed(Q, j):
        r, u, pr = prim(Q)
        return np.abs(u[..., j]) + np.sqrt(g * pr / r)

    Q, _, _, _ = orc.run(P, Q0, 3, fixed_dt=0.005)
    ref = fv_rusanov(flux, speed, Q0[:, :, 0].reshape(4, 6, 4), P.dx, 0.005, 3)
    np.testing.assert_allclose(Q[:, :, 0], ref.reshape(-1, 4), atol=1e-14)


# --------------------------------------------------------------------------
# Structure: periodic shift invariance; Eq. 5 = Eq. 6 in the orders of
# Algorithms 1 and 2; optimistic time stepping with one rerun

def test_periodic_shift_invariance():
    P = orc.Problem(2, 3, ADV, (5, 4), (0.2, 0.25), cst=(0.7, -0.4))
    rng = np.random.default_rng(5)
    Q0 = rng.standard_normal((P.C, 1, P.NS))
    Qa, _, _, _ = orc.run(P, Q0, 3, fixed_dt=0.004)
    shift = lambda Q: np.roll(Q.reshape(4, 5, 1, P.NS), (1, 2), axis=(0, 1)).reshape(P.C, 1, P.NS)
    Qb, _, _, _ = orc.run(P, shift(Q0), 3, fixed_dt=0.004)
    np.testing.assert_allclose(Qb, shift(Qa), atol=1e-15)


def test_shifted_order_equals_straightforward_linear():
    P = orc.Problem(3, 2, ACO, (3, 4, 2), (1 / 3, 0.25, 0.5), cst=(1.0, 1.0))
    Q0 = np.random.default_rng(6).standard_normal((P.C, P.m, P.NS))
    Qa, dta, ta, _ = orc.run(P, Q0, 5)
    Qb, dtb, nre, tb = orc.run_shifted(P, Q0, 5)
    assert nre == 0
    np.testing.assert_allclose(dtb, dta, rtol=1e-15)
    np.testing.assert_allclose(Qb, Qa, atol=1e-14)


def _euler_2d(grid=(5, 4), N=2, seed=3):
    w = wl.Workload("e", "euler", 2, N, grid, 0, cst=(1.4,), seed=seed, extra={"amp": 0.1, "kmax": 2})
    P = orc.Problem(2, N, EUL, grid, w.dx, cst=w.cst)
    Q0 = wl.init_state(w, coords(P))
    return P, Q0


@pytest.mark.parametrize("policy", [0, 1])
def test_shifted_euler_replays_in_straightforward_order(policy):
    P, Q0 = _euler_2d()
    Qs, dts, nre, _ = orc.run_shifted(P, Q0, 6, policy=policy)
    assert nre == 0
    Qa, _, _, _ = orc.run(P, Q0, 6, dt_seq=dts)
    np.testing.assert_allclose(Qs, Qa, atol=1e-13)
    # strict policy lags dt_adm by one step (Technique 5): dt_1 = dt_2
    if policy == 0:
        assert dts[0] == dts[1]


def test_optimistic_rerun_once():
    P, Q0 = _euler_2d()
    Qs, dts, nre, _ = orc.run_shifted(P, Q0, 6, inject_step=2, inject_factor=0.5)
    assert nre == 1
    assert dts[2] < 0.6 * dts[1]
    Qa, _, _, _ = orc.run(P, Q0, 6, dt_seq=dts)
    np.testing.assert_allclose(Qs, Qa, atol=1e-13)


# --------------------------------------------------------------------------
# step_cells: one Algorithm-1 step evaluated for listed cells only (the
# reference of every sampled full-size check) against the whole-grid step

def _smooth(P, seed):
    rng = np.random.default_rng(seed)
    X = coords(P)
    Q = np.zeros((P.C, P.m, P.NS))
    for c in range(P.m):
        for _ in range(3):
            k = rng.integers(-2, 3, size=P.d)
            L = np.array(P.grid[: P.d]) * np.array(P.dx[: P.d])
            Q[:, c] += rng.standard_normal() * np.cos(2 * math.pi * ((X / L) @ k) + rng.random() * 6.28)
    return Q


@pytest.mark.parametrize("case", ["acoustics", "elasticity_material"])
@pytest.mark.parametrize("grid", [(3, 1, 2), (2, 3, 1), (4, 3, 5)])
def test_step_cells_equals_whole_grid_step(case, grid):
    """A size-1 axis makes a cell its own left and right neighbour, a size-2
    axis makes both neighbours one cell: the periodic wrap of the
    neighbour list and the order of the left/right faces are exercised."""
    dx = (0.3, 0.25, 0.2)
    if case == "acoustics":
        P = orc.Problem(3, 3, ACO, grid, dx, cst=(1.3, 0.8))
    else:
        C = int(np.prod(grid))
        rng = np.random.default_rng(7)
        mat = np.stack([rng.uniform(2, 3, C), rng.uniform(4, 6, C), np.zeros(C)], 1)
        mat[:, 2] = mat[:, 1] / math.sqrt(3)
        P = orc.Problem(3, 2, ELA, grid, dx, mat=mat)
    Q0 = _smooth(P, 3)
    dt = 0.3 * orc.dt_admissible(P, orc.lam(P, Q0))
    Q1, _, _, _ = orc.run(P, Q0, 1, fixed_dt=dt)
    scale = np.abs(Q1).max()
    Qs = orc.step_cells(P, Q0, dt, np.arange(P.C))
    assert np.abs(Qs - Q1).max() <= 1e-15 * scale
    # listed in another order, with repeats: row s is cell cells[s]
    cells = np.array([P.C - 1, 0, P.C // 2, 0])
    Qs = orc.step_cells(P, Q0, dt, cells)
    assert np.abs(Qs - Q1[cells]).max() <= 1e-15 * scale
    assert np.abs(Q1 - Q0).max() > 1e-3 * scale   # the step did something


# --------------------------------------------------------------------------
# receivers: point values of the nodal polynomial (Sec. 3 basis)

def _tensor_poly(rng, d, N):
    """A random tensor-product polynomial of degree <= N in every variable."""
    coef = rng.standard_normal((N + 1,) * d)

    def f(x):                                   # x [..., d]
        v = np.zeros(x.shape[:-1])
        for idx in np.ndindex(coef.shape):
            term = coef[idx]
            for a in range(d):
                term = term * x[..., a] ** idx[a]
            v = v + term
        return v
    return f


@pytest.mark.parametrize("d,N,grid", [(2, 3, (4, 3)), (3, 2, (3, 2, 4)), (2, 0, (5, 2))])
def test_receivers_reproduce_a_polynomial(d, N, grid):
    """Within a cell the nodal interpolant of a polynomial of degree <= N per
    axis is that polynomial, so the receivers must return it at any point."""
    dx = (0.5, 0.4, 0.3)[:d]
    P = orc.Problem(d, N, ACO, grid, dx, cst=(1.0, 1.0))
    rng = np.random.default_rng(20 + d * 10 + N)
    polys = [_tensor_poly(rng, d, N) for _ in range(P.m)]
    X = coords(P)                                      # [C][NS][d]
    Q = np.stack([f(X) for f in polys], 1)             # [C][m][NS]
    ext = np.array(grid) * np.array(dx)
    pos = rng.uniform(0.02, 0.98, (9, d)) * ext
    got = orc.receivers(P, Q, pos)
    comps = orc.receiver_comps(P)
    want = np.stack([polys[c](pos) for c in comps], 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_receivers_clamp_to_the_boundary_cell():
    """Positions outside the grid evaluate the nearest boundary cell's
    polynomial (extrapolated): a state that differs from cell to cell tells
    the cells apart."""
    d, N, grid, dx = 2, 2, (4, 3), (0.5, 0.4)
    P = orc.Problem(d, N, ACO, grid, dx, cst=(1.0, 1.0))
    rng = np.random.default_rng(4)
    base = [_tensor_poly(rng, d, N) for _ in range(P.m)]
    off = rng.standard_normal((P.C, P.m))              # per-cell constant
    X = coords(P)
    Q = np.stack([f(X) for f in base], 1) + off[:, :, None]
    pos = np.array([[-0.3, 0.5], [2.4, 0.5], [1.1, -0.2], [1.1, 1.7], [-0.1, 1.5], [2.2, 1.3]])
    cell_of = []
    for x, y in pos:
        i = min(max(int(math.floor(x / dx[0])), 0), grid[0] - 1)
        j = min(max(int(math.floor(y / dx[1])), 0), grid[1] - 1)
        cell_of.append(i + grid[0] * j)
    got = orc.receivers(P, Q, pos)
    comps = orc.receiver_comps(P)
    want = np.stack([base[c](pos) + off[cell_of, c] for c in comps], 1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    assert cell_of == [4, 7, 2, 10, 8, 11]   # every point is outside the grid on some axis


# --------------------------------------------------------------------------
# receiver misfit and its gradients (definition level)

def _elastic_problem(grid=(2, 2), N=1):
    """2D elasticity with a checkerboard cp (4 against 6): every face joins a
    slow and a fast cell, so perturbing one cell's cp by up to 16 % never
    changes which side sets the Rusanov speed s = max(cp_L, cp_R)."""
    C = int(np.prod(grid))
    ci = np.arange(C)
    cb = (ci % grid[0] + ci // grid[0]) % 2
    rng = np.random.default_rng(9)
    mat = np.stack([rng.uniform(2, 3, C), np.where(cb == 0, 6.0, 4.0), np.zeros(C)], 1)
    mat[:, 2] = mat[:, 1] / math.sqrt(3) * rng.uniform(0.9, 1.0, C)
    dx = tuple(1.0 / g for g in grid)
    return orc.Problem(2, N, ELA, grid, dx, mat=mat)


def _gradient_setup(P, nsteps=3, R=3, seed=1):
    rng = np.random.default_rng(seed)
    Q0 = rng.standard_normal((P.C, P.m, P.NS))
    dt = 0.3 * orc.dt_admissible(P, orc.lam(P, Q0))
    ext = np.array(P.grid[: P.d]) * np.array(P.dx[: P.d])
    pos = rng.uniform(0.05, 0.95, (R, P.d)) * ext
    nc = len(orc.receiver_comps(P))
    obs = rng.standard_normal((nsteps, R, nc))
    return Q0, dt, pos, obs


def test_misfit_definition():
    """J = 1/2 dt sum |trace - obs|^2: zero at the model's own traces, the
    squared shift otherwise."""
    P = _elastic_problem()
    Q0, dt, pos, obs = _gradient_setup(P)
    tr = orc.trajectory(P, Q0, 3, dt, pos)
    assert orc.misfit(P, Q0, 3, dt, pos, tr) == 0.0
    delta = np.random.default_rng(2).standard_normal(tr.shape)
    J = orc.misfit(P, Q0, 3, dt, pos, tr + delta)
    assert abs(J - 0.5 * dt * (delta ** 2).sum()) <= 1e-13 * J
    # one trace per step, each equal to the receivers of the state after that step
    Q1, _, _, _ = orc.run(P, Q0, 1, fixed_dt=dt)
    np.testing.assert_allclose(tr[0], orc.receivers(P, Q1, pos), rtol=0, atol=1e-14)


def test_gradient_q0_against_central_differences():
    """J is quadratic in Q0 (the step is linear for linear fluxes), so the
    central difference along any direction is exact up to round-off."""
    P = _elastic_problem()
    Q0, dt, pos, obs = _gradient_setup(P)
    g = orc.grad_q0_tangent(P, Q0, 3, dt, pos, obs)
    rng = np.random.default_rng(3)
    for _ in range(3):
        e = rng.standard_normal(Q0.shape)
        h = 1.0
        fd = (orc.misfit(P, Q0 + h * e, 3, dt, pos, obs) -
              orc.misfit(P, Q0 - h * e, 3, dt, pos, obs)) / (2 * h)
        got = float((g * e).sum())
        assert abs(got - fd) <= 1e-11 * max(abs(fd), 1e-300), (got, fd)


def test_gradient_q0_dot_product():
    """Adjoint dot-product test: with T the linear map from Q0 to the
    receiver traces, <v, T u> dt = <T^T v dt, u> for random u and v, where
    T^T v dt is the gradient of J at Q0 = 0 with observations -v."""
    P = _elastic_problem()
    _, dt, pos, obs = _gradient_setup(P)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((P.C, P.m, P.NS))
    v = rng.standard_normal(obs.shape)
    Tu = orc.trajectory(P, u, 3, dt, pos)
    TtV = orc.grad_q0_tangent(P, np.zeros_like(u), 3, dt, pos, -v)
    lhs = dt * float((v * Tu).sum())
    rhs = float((TtV * u).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def test_gradient_material_fd_is_fourth_order():
    """The Richardson-extrapolated central difference has an O(h^4) error:
    halving h shrinks the difference of successive estimates about 16-fold
    (an O(h^2) slip would give 4)."""
    P = _elastic_problem()
    Q0, dt, pos, obs = _gradient_setup(P, nsteps=2)
    G = [orc.grad_material_fd(P, Q0, 2, dt, pos, obs, h=h) for h in (0.16, 0.08, 0.04)]
    d1 = np.abs(G[0] - G[1]).max()
    d2 = np.abs(G[1] - G[2]).max()
    assert d2 > 1e-9 * np.abs(G[2]).max()            # above round-off
    assert 12.0 < d1 / d2 < 20.0, d1 / d2
