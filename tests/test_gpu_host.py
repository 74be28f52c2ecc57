"""aderdg_step_host (host-resident state, chunked copies overlapping the first
STP sweep and the last corrector): bitwise equal to aderdg_step on the device."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A

pytestmark = pytest.mark.gpu


def device_and_host(d, N, m, pde, grid, cst, Q0, nsteps, precision="fp32", mat=None, fixed_dt=0.0, cfl=0.0):
    import torch
    dx = tuple(1.0 / g for g in grid)
    prm = A.params(pde_const=cst, precision=precision, cfl=cfl)
    tdt = torch.float64 if precision != "fp32" else torch.float32
    out = []
    for host in (False, True):
        h = A.aderdg_create(d, N, m, pde, grid, dx, prm)
        try:
            if mat is not None:
                A.aderdg_set_material(h, torch.from_numpy(mat.astype(np.float32)).cuda())
            if host:
                q = torch.from_numpy(Q0.astype(np.float64)).to(tdt).pin_memory()
                t = A.aderdg_step_host(h, q, nsteps, fixed_dt)
                out.append((q.double().numpy(), t))
            else:
                q = torch.from_numpy(Q0.astype(np.float64)).to(tdt).cuda()
                t = A.aderdg_step(h, q, nsteps, fixed_dt)
                out.append((q.double().cpu().numpy(), t))
        finally:
            A.aderdg_destroy(h)
    return out


def pulse(w):
    xi, _ = A.aderdg_nodes(w.N)
    return wl.init_state(w, wl.node_coords(w.grid, w.dx, xi))


@pytest.mark.parametrize("nsteps", [1, 3])
def test_acoustics3d_chunked(nsteps):
    w = wl.acoustics_3d(grid=(10, 9, 8))        # 720 cells, 103 tiles of 7: 26 chunks of 4 tiles
    w.extra["sigma"] = 0.15
    (qd, td), (qh, th) = device_and_host(3, 5, 4, A.ACOUSTICS, w.grid, w.cst, pulse(w), nsteps)
    assert th == td
    np.testing.assert_array_equal(qh, qd)


@pytest.mark.parametrize("grid", [(12, 12, 3), (40, 30)])
def test_acoustics_one_step_interleaved(grid):
    """One step: each chunk's corrector and copy-out start once the STP sweeps of
    its neighbours' chunks are done; (12, 12, 3) puts z-neighbours about ten
    chunks away (14-cell chunks of two 7-cell tiles, 144-cell planes), (40, 30)
    is 2D."""
    d = len(grid)
    w = wl.acoustics_3d(grid=grid) if d == 3 else wl.Workload("a2", "acoustics", 2, 4, grid, 1, cst=(1.2, 0.8), seed=4)
    w.extra["sigma"] = 0.15
    (qd, td), (qh, th) = device_and_host(d, w.N, w.m, A.ACOUSTICS, w.grid, w.cst, pulse(w), 1)
    assert th == td
    np.testing.assert_array_equal(qh, qd)


@pytest.mark.parametrize("fixed_dt,cfl", [(1e-4, 0.0), (0.0, 1.0)])
def test_acoustics_one_step_fixed_dt_and_largest_cfl(fixed_dt, cfl):
    """One interleaved step with a fixed dt, and at the largest CFL factor the
    library accepts (dt_new = dt_adm: still no rerun)."""
    w = wl.acoustics_3d(grid=(10, 9, 8))
    w.extra["sigma"] = 0.15
    (qd, td), (qh, th) = device_and_host(3, 5, 4, A.ACOUSTICS, w.grid, w.cst, pulse(w), 1,
                                         fixed_dt=fixed_dt, cfl=cfl)
    assert th == td
    np.testing.assert_array_equal(qh, qd)


@pytest.mark.parametrize("nsteps", [1, 2])
def test_elasticity3d_material_chunked(nsteps):
    w = wl.elasticity_3d(grid=(6, 5, 7))
    w.extra["sigma"] = 0.2
    (qd, td), (qh, th) = device_and_host(3, 4, 9, A.ELASTICITY, w.grid, w.cst, pulse(w), nsteps,
                                         mat=wl.materials(w))
    assert th == td
    np.testing.assert_array_equal(qh, qd)


@pytest.mark.parametrize("nsteps", [1, 2])
def test_euler_copies_first_then_chunked_corrector(nsteps):
    w = wl.euler_3d(grid=(7, 6, 5), steps=2)
    (qd, td), (qh, th) = device_and_host(3, 3, 5, A.EULER, w.grid, w.cst, pulse(w), nsteps,
                                         precision="fp32_acc64")
    assert th == td
    np.testing.assert_array_equal(qh, qd)


def test_nonfinite_host_state_is_reported():
    import torch
    w = wl.acoustics_3d(grid=(6, 5, 4))
    Q0 = pulse(w).astype(np.float32)
    Q0[17, 2, 5] = np.nan
    h = A.aderdg_create(3, 5, 4, A.ACOUSTICS, w.grid, w.dx, A.params(pde_const=w.cst))
    try:
        q = torch.from_numpy(Q0).pin_memory()
        with pytest.raises(A.AderdgError) as ei:
            A.aderdg_step_host(h, q, 2)
        assert ei.value.status == A.ADERDG_ENONFINITE
    finally:
        A.aderdg_destroy(h)
