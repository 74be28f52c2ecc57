"""The discrete adjoint (aderdg_step_adjoint) against the oracle.

References
  * dJ/dQ0: exact, from oracle tangent runs (the step is linear in Q for
    linear fluxes, so the derivative along a unit vector is a finite sum).
  * dJ/d(rho, cp, cs): the definition evaluated by the oracle with central
    differences and one Richardson step (error O(h^4) ~ 1e-10).
  * <dJ/dQ0, Q0> = 2 J when the observations are zero (J is then a
    homogeneous quadratic in Q0).
Tolerances: FP64 kernels 1e-9 (Q0) / 1e-6 (material) relative; FP32 kernels
1e-4 relative, the accuracy target of the gradient.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A
from tests.helpers import coords

pytestmark = pytest.mark.gpu

ACO, ELA = orc.ACOUSTICS, orc.ELASTICITY


def smooth(P, seed):
    X = coords(P)
    rng = np.random.default_rng(seed)
    Q = np.zeros((P.C, P.m, P.NS))
    for c in range(P.m):
        for _ in range(2):
            k = rng.integers(-1, 2, size=P.d)
            Q[:, c] += rng.standard_normal() * np.cos(2 * math.pi * (X @ k) + rng.random() * 6.28)
    return Q


def setup(pde, d, N, grid, seed, R=3, nsteps=4):
    dx = tuple(1.0 / g for g in grid)
    cst = (1.0, 1.0) if pde == ACO else (2.5, 5.0, 5 / math.sqrt(3))
    mat = None
    if pde == ELA:
        w = wl.Workload("m", "elasticity", d, N, grid, 0, seed=seed)
        mat = wl.materials(w).astype(np.float32)
    P = orc.Problem(d, N, pde, grid, dx, cst=cst,
                    mat=None if mat is None else mat.astype(np.float64))
    Q0 = smooth(P, seed)
    rng = np.random.default_rng(seed + 1)
    pos = rng.random((R, d)) * 0.98 + 0.01
    nc = len(orc.receiver_comps(P))
    obs = 0.1 * rng.standard_normal((nsteps, R, nc))
    return P, Q0, mat, pos, obs


def gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, precision, ckpt=30, want_mat=True):
    import torch
    tdt = torch.float64 if precision == "fp64" else torch.float32
    h = A.aderdg_create(P.d, P.N, P.m, P.pde, P.grid[: P.d], P.dx[: P.d],
                        A.params(pde_const=P.cst[:8], precision=precision))
    try:
        if mat is not None:
            A.aderdg_set_material(h, torch.from_numpy(mat).cuda())
        Qd = torch.from_numpy(Q0).to(tdt).cuda()
        gQ = torch.zeros_like(Qd)
        gm = torch.zeros(P.C, 3, device="cuda") if (mat is not None and want_mat) else None
        J = A.aderdg_step_adjoint(h, Qd, nsteps, dt, torch.from_numpy(pos.astype(np.float32)).cuda(),
                                  torch.from_numpy(obs.astype(np.float32)).cuda(), gQ, gm, ckpt)
        return J, gQ.double().cpu().numpy(), (gm.double().cpu().numpy() if gm is not None else None)
    finally:
        A.aderdg_destroy(h)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("pde,d,grid", [(ELA, 2, (4, 3)), (ACO, 2, (4, 3)), (ELA, 3, (2, 2, 2))])
def test_adjoint_fp64_matches_oracle(pde, d, grid):
    nsteps, dt = 4, 0.004
    P, Q0, mat, pos, obs = setup(pde, d, 2, grid, 5, nsteps=nsteps)
    obs32 = obs.astype(np.float32).astype(np.float64)
    J, gQ, gm = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp64")
    pos32 = pos.astype(np.float32).astype(np.float64)
    Jo = orc.misfit(P, Q0, nsteps, dt, pos32, obs32)
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    gQo = orc.grad_q0_tangent(P, Q0, nsteps, dt, pos32, obs32)
    assert rel(gQ, gQo) < 1e-9
    if pde == ELA:
        gmo = orc.grad_material_fd(P, Q0, nsteps, dt, pos32, obs32)
        assert rel(gm, gmo) < 1e-6


@pytest.mark.parametrize("pde,N,grid", [(ELA, 3, (5, 4)), (ACO, 2, (4, 5)), (ELA, 2, (3, 4))])
def test_adjoint_fp32_2d_matches_oracle(pde, N, grid):
    """The FP32 builds of the line-owner adjoint kernels in 2D (several tiles per
    block, bipartite groups of both PDEs) against the oracle's exact tangent
    gradient; the material gradient against its Richardson difference."""
    nsteps, dt = 4, 0.002
    P, Q0, mat, pos, obs = setup(pde, 2, N, grid, 21, nsteps=nsteps)
    obs32 = obs.astype(np.float32).astype(np.float64)
    pos32 = pos.astype(np.float32).astype(np.float64)
    J, gQ, gm = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp32", ckpt=3)
    Jo = orc.misfit(P, Q0, nsteps, dt, pos32, obs32)
    assert abs(J - Jo) <= 1e-4 * abs(Jo)
    gQo = orc.grad_q0_tangent(P, Q0, nsteps, dt, pos32, obs32)
    assert rel(gQ, gQo) < 1e-4
    if pde == ELA:
        gmo = orc.grad_material_fd(P, Q0, nsteps, dt, pos32, obs32)
        assert rel(gm, gmo) < 1e-3


def test_adjoint_homogeneity_fp64():
    nsteps, dt = 5, 0.004
    P, Q0, mat, pos, obs = setup(ELA, 2, 2, (4, 3), 9, nsteps=nsteps)
    J, gQ, _ = gpu_adjoint(P, Q0, mat, pos, np.zeros_like(obs), nsteps, dt, "fp64", want_mat=False)
    assert abs(float((gQ * Q0).sum()) - 2 * J) <= 1e-11 * abs(J)


def test_adjoint_q0_only_equals_full_run():
    """Without a material gradient no forward state is kept or recomputed; dJ/dQ0
    and J are those of the run with both gradients, bit for bit."""
    nsteps, dt = 6, 0.004
    P, Q0, mat, pos, obs = setup(ELA, 2, 2, (5, 4), 13, nsteps=nsteps)
    J, gQ, gm = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp64", ckpt=2)
    J1, gQ1, gm1 = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp64", ckpt=2, want_mat=False)
    assert gm is not None and gm1 is None
    assert J1 == J
    np.testing.assert_array_equal(gQ1, gQ)


def test_adjoint_checkpoint_invariance():
    nsteps, dt = 7, 0.004
    P, Q0, mat, pos, obs = setup(ELA, 2, 2, (4, 3), 11, nsteps=nsteps)
    ref = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp64", ckpt=nsteps)
    for ck in (1, 2, 3):
        J, gQ, gm = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp64", ckpt=ck)
        assert abs(J - ref[0]) <= 1e-13 * abs(ref[0])
        assert rel(gQ, ref[1]) < 1e-12 and rel(gm, ref[2]) < 1e-12


def test_adjoint_fp32_elasticity3d_n4_directional():
    """Reduced config-4 problem: 4^3 cells, N=4, 64 receivers, 10 steps,
    checkpoints every 3; FP32 gradients against oracle directional
    derivatives (central differences; J is quadratic in Q0)."""
    nsteps = 10
    w = wl.elasticity_3d(grid=(4, 4, 4), steps=nsteps)
    mat = wl.materials(w).astype(np.float32)
    P = orc.Problem(3, 4, ELA, w.grid, w.dx, cst=w.cst, mat=mat.astype(np.float64))
    w.extra["sigma"] = 0.15
    Q0 = wl.init_state(w, coords(P))
    pos = wl.receivers(w).astype(np.float32).astype(np.float64)
    dt = 0.5 * orc.dt_admissible(P, float(mat[:, 1].max()))
    rng = np.random.default_rng(3)
    obs = (0.01 * rng.standard_normal((nsteps, 64, 3))).astype(np.float32).astype(np.float64)
    J, gQ, gm = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp32", ckpt=3)
    Jo = orc.misfit(P, Q0, nsteps, dt, pos, obs)
    assert abs(J - Jo) <= 1e-4 * abs(Jo)
    for seed in range(2):
        r = np.random.default_rng(100 + seed)
        dQ = r.standard_normal(Q0.shape)
        eps = 1e-3
        fd = (orc.misfit(P, Q0 + eps * dQ, nsteps, dt, pos, obs)
              - orc.misfit(P, Q0 - eps * dQ, nsteps, dt, pos, obs)) / (2 * eps)
        assert abs(float((gQ * dQ).sum()) - fd) <= 1e-4 * abs(fd)
        dm = r.standard_normal(mat.shape) * mat.astype(np.float64)

        def Jm(e):
            Pm = orc.Problem(3, 4, ELA, w.grid, w.dx, cst=w.cst, mat=mat.astype(np.float64) + e * dm)
            return orc.misfit(Pm, Q0, nsteps, dt, pos, obs)

        h1, h2 = 1e-4, 5e-5
        d1 = (Jm(h1) - Jm(-h1)) / (2 * h1)
        d2 = (Jm(h2) - Jm(-h2)) / (2 * h2)
        fdm = (4 * d2 - d1) / 3
        assert abs(float((gm * dm).sum()) - fdm) <= 1e-4 * abs(fdm)


def test_autograd_function():
    import torch
    nsteps, dt = 4, 0.004
    P, Q0, mat, pos, obs = setup(ELA, 2, 2, (4, 3), 13, nsteps=nsteps)
    J0, gQ0, gm0 = gpu_adjoint(P, Q0, mat, pos, obs, nsteps, dt, "fp32")
    h = A.aderdg_create(P.d, P.N, P.m, P.pde, P.grid[: P.d], P.dx[: P.d], A.params(pde_const=P.cst[:8]))
    try:
        f = A.ReceiverMisfit(h, nsteps, torch.from_numpy(pos.astype(np.float32)).cuda(),
                             torch.from_numpy(obs.astype(np.float32)).cuda(), dt)
        Q = torch.from_numpy(Q0).float().cuda().requires_grad_()
        M = torch.from_numpy(mat).cuda().requires_grad_()
        J = f(Q, M)
        (2.0 * J).backward()
        assert abs(float(J) - J0) <= 1e-6 * abs(J0)
        np.testing.assert_allclose(Q.grad.double().cpu().numpy(), 2 * gQ0, rtol=0, atol=1e-6 * np.abs(gQ0).max())
        np.testing.assert_allclose(M.grad.double().cpu().numpy(), 2 * gm0, rtol=0, atol=1e-6 * np.abs(gm0).max())
    finally:
        A.aderdg_destroy(h)
