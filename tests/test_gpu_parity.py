"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances
  * FP64 kernels against the FP64 oracle: max |diff| <= 1e-11 max|Q| (the
    two differ only in summation order and in the time-averaged hull).
  * FP32 kernels: relative L2 <= 1e-5 over all components (the target
    accuracy of the FP32 step against the FP64 oracle).
Grids span several tiles with a ragged last tile; the time-step sequence of
nonlinear runs is replayed in the oracle (shifted stepping lags dt_adm by
one step, Technique 5), and separately checked against the oracle's own
Algorithm-2 control.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, rel_l2_plain, run_gpu
from tests.helpers import coords, l2

pytestmark = pytest.mark.gpu

ADV, ACO, EUL, ELA = orc.ADVECTION, orc.ACOUSTICS, orc.EULER, orc.ELASTICITY


def tight(got, ref, rtol=1e-11):
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(got - ref).max() / scale
    assert err <= rtol, err


def random_smooth(P, seed, amp=1.0, base=None):
    """Seeded smooth fields: a few Fourier modes per component."""
    X = coords(P)
    rng = np.random.default_rng(seed)
    Q = np.zeros((P.C, P.m, P.NS))
    for c in range(P.m):
        for _ in range(3):
            k = rng.integers(-2, 3, size=P.d)
            Q[:, c] += amp * rng.standard_normal() * np.cos(2 * math.pi * (X @ k) + rng.random() * 6.28)
    if base is not None:
        Q += np.asarray(base)[None, :, None]
    return Q


def euler_state(P, seed):
    X = coords(P)
    w = wl.Workload("e", "euler", P.d, P.N, P.grid[: P.d], 0, cst=(1.4,), seed=seed,
                    extra={"amp": 0.1, "kmax": 2})
    Q = wl.init_state(w, X)
    Q[:, 1] = 0.2 * np.sin(2 * math.pi * X[..., 1])           # some momentum
    Q[:, P.m - 1] += 0.5 * Q[:, 1] ** 2 / Q[:, 0]
    return Q


# ---------------------------------------------------------------- FP64 exactness

def test_c1_advection_fp64_matches_oracle_and_exact():
    w = wl.advection_2d()
    P = orc.Problem(2, w.N, ADV, w.grid, w.dx, cst=w.cst)
    X = coords(P)
    Q0 = wl.init_state(w, X)
    Qo, dto, to, _ = orc.run(P, Q0, w.steps)
    for form in ("fused", "hull3"):
        Qg, dtg, tg, st = run_gpu(P, Q0, w.steps, precision="fp64", form=form)
        np.testing.assert_allclose(dtg, dto, rtol=1e-14)
        assert abs(tg - to) < 1e-14
        tight(Qg, Qo)
    exact = np.sin(2 * math.pi * (X[..., 0] - to)) * np.sin(2 * math.pi * (X[..., 1] - 0.5 * to))
    assert l2(P, Qg[:, 0] - exact) < 2.4e-7


@pytest.mark.parametrize("N", [0, 1, 2, 3, 5, 6])
def test_advection_fp64_orders(N):
    P = orc.Problem(2, N, ADV, (7, 5), (1 / 7, 1 / 5), cst=(0.8, -0.6))
    Q0 = random_smooth(P, N)
    Qo, _, _, _ = orc.run(P, Q0, 4)
    Qg, _, _, _ = run_gpu(P, Q0, 4, precision="fp64")
    tight(Qg, Qo)


@pytest.mark.parametrize("d,N", [(2, 0), (2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_acoustics_fp64(d, N):
    grid = (7, 5) if d == 2 else (5, 3, 3)
    P = orc.Problem(d, N, ACO, grid, tuple(1 / g for g in grid), cst=(1.3, 0.7))
    Q0 = random_smooth(P, 10 + N)
    Qo, _, _, _ = orc.run(P, Q0, 3)
    Qg, _, _, _ = run_gpu(P, Q0, 3, precision="fp64")
    tight(Qg, Qo)


@pytest.mark.parametrize("form", ["fused", "hull3", "table1"])
def test_acoustics_fp64_forms(form):
    P = orc.Problem(2, 2, ACO, (7, 5), (1 / 7, 1 / 5), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 3)
    Qo, _, _, _ = orc.run(P, Q0, 4)
    Qg, _, _, _ = run_gpu(P, Q0, 4, precision="fp64", form=form)
    tight(Qg, Qo)


def test_acoustics_fp64_spacetime_predictor():
    P = orc.Problem(2, 2, ACO, (7, 5), (1 / 7, 1 / 5), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 4)
    Qo, _, _, _ = orc.run(P, Q0, 4)
    Qg, _, _, _ = run_gpu(P, Q0, 4, precision="fp64", predictor=A.PREDICT_SPACETIME)
    tight(Qg, Qo)


@pytest.mark.parametrize("form", ["fused", "table1"])
def test_advection_fp64_spacetime(form):
    P = orc.Problem(2, 3, ADV, (6, 5), (1 / 6, 1 / 5), cst=(1.0, 0.5))
    Q0 = random_smooth(P, 5)
    Qo, _, _, _ = orc.run(P, Q0, 3)
    Qg, _, _, _ = run_gpu(P, Q0, 3, precision="fp64", form=form, predictor=A.PREDICT_SPACETIME)
    tight(Qg, Qo)


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4])
def test_euler_fp64_replays_dt(N):
    P = orc.Problem(2, N, EUL, (7, 5), (1 / 7, 1 / 5), cst=(1.4,))
    Q0 = euler_state(P, 20 + N)
    Qg, dtg, tg, st = run_gpu(P, Q0, 5, precision="fp64")
    assert st.reruns == 0
    Qo, _, _, _ = orc.run(P, Q0, 5, dt_seq=dtg)
    tight(Qg, Qo, 1e-10)
    # the GPU's optimistic control equals the oracle's Algorithm 2
    Qs, dts, nre, _ = orc.run_shifted(P, Q0, 5)
    np.testing.assert_allclose(dtg, dts, rtol=1e-12)
    assert nre == 0


@pytest.mark.parametrize("form", ["hull3", "table1"])
def test_euler_fp64_multipass_straightforward_dt(form):
    P = orc.Problem(2, 2, EUL, (7, 5), (1 / 7, 1 / 5), cst=(1.4,))
    Q0 = euler_state(P, 31)
    Qo, dto, _, _ = orc.run(P, Q0, 4)       # Algorithm 1 dt control
    Qg, dtg, _, _ = run_gpu(P, Q0, 4, precision="fp64", form=form)
    np.testing.assert_allclose(dtg, dto, rtol=1e-12)
    tight(Qg, Qo, 1e-10)


def test_euler_fp64_3d():
    P = orc.Problem(3, 2, EUL, (5, 3, 3), (0.2, 1 / 3, 1 / 3), cst=(1.4,))
    Q0 = euler_state(P, 7)
    Qg, dtg, _, _ = run_gpu(P, Q0, 3, precision="fp64")
    Qo, _, _, _ = orc.run(P, Q0, 3, dt_seq=dtg)
    tight(Qg, Qo, 1e-10)


def test_euler_rerun_injection():
    """dt_adm cut by half after step 2: exactly one STP rerun (Technique 5)."""
    P = orc.Problem(2, 2, EUL, (7, 5), (1 / 7, 1 / 5), cst=(1.4,))
    Q0 = euler_state(P, 8)
    Qg, dtg, _, st = run_gpu(P, Q0, 6, precision="fp64", inject_step=2, inject_factor=0.5)
    Qs, dts, nre, _ = orc.run_shifted(P, Q0, 6, inject_step=2, inject_factor=0.5)
    assert st.reruns == 1 and nre == 1
    np.testing.assert_allclose(dtg, dts, rtol=1e-12)
    tight(Qg, Qs, 1e-10)


def test_euler_creeping_policy():
    P = orc.Problem(2, 2, EUL, (7, 5), (1 / 7, 1 / 5), cst=(1.4,))
    Q0 = euler_state(P, 9)
    Qg, dtg, _, _ = run_gpu(P, Q0, 6, precision="fp64", dt_policy=A.DT_CREEPING)
    Qs, dts, _, _ = orc.run_shifted(P, Q0, 6, policy=1)
    np.testing.assert_allclose(dtg, dts, rtol=1e-12)
    tight(Qg, Qs, 1e-10)


def test_elasticity_fp64_material():
    P0 = orc.Problem(2, 2, ELA, (7, 5), (1 / 7, 1 / 5), cst=(2.5, 5.0, 5 / math.sqrt(3)))
    w = wl.Workload("el", "elasticity", 2, 2, (7, 5), 0, seed=4)
    mat = wl.materials(w)
    P = orc.Problem(2, 2, ELA, (7, 5), (1 / 7, 1 / 5), cst=P0.cst, mat=mat.astype(np.float32).astype(np.float64))
    Q0 = random_smooth(P, 12)
    Qo, dto, _, _ = orc.run(P, Q0, 3)
    Qg, dtg, _, _ = run_gpu(P, Q0, 3, precision="fp64", mat=mat)
    np.testing.assert_allclose(dtg, dto, rtol=1e-7)   # cp max is read as float32
    Qo, _, _, _ = orc.run(P, Q0, 3, dt_seq=dtg)
    tight(Qg, Qo)


def test_fixed_dt():
    P = orc.Problem(2, 3, ACO, (6, 5), (1 / 6, 1 / 5), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 13)
    Qo, _, to, _ = orc.run(P, Q0, 3, fixed_dt=0.003)
    Qg, dtg, tg, _ = run_gpu(P, Q0, 3, precision="fp64", fixed_dt=0.003)
    assert np.all(dtg == 0.003) and abs(tg - to) < 1e-15
    tight(Qg, Qo)


# ---------------------------------------------------------------- FP32 accuracy

@pytest.mark.parametrize("form,pred", [("fused", A.PREDICT_AUTO), ("hull3", A.PREDICT_AUTO),
                                       ("table1", A.PREDICT_AUTO), ("fused", A.PREDICT_SPACETIME),
                                       ("table1", A.PREDICT_SPACETIME)])
def test_acoustics3d_n5_fp32(form, pred):
    w = wl.acoustics_3d(grid=(6, 5, 4), steps=6)
    w.extra["sigma"] = 0.15
    P = orc.Problem(3, 5, ACO, w.grid, w.dx, cst=w.cst)
    Q0 = wl.init_state(w, coords(P))
    Qo, dto, _, _ = orc.run(P, Q0, w.steps)
    Qg, dtg, _, _ = run_gpu(P, Q0, w.steps, precision="fp32", form=form, predictor=pred)
    np.testing.assert_allclose(dtg, dto, rtol=1e-14)
    assert rel_l2_plain(Qg, Qo) < 1e-5


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("pde", [ACO, ELA])
def test_ensemble_orders_fp32(pde, N):
    cst = (1.0, 1.0) if pde == ACO else (2.5, 5.0, 5 / math.sqrt(3))
    P = orc.Problem(2, N, pde, (11, 9), (1 / 11, 1 / 9), cst=cst)
    Q0 = random_smooth(P, 40 + N)
    Qo, _, _, _ = orc.run(P, Q0, 5)
    Qg, _, _, _ = run_gpu(P, Q0, 5, precision="fp32")
    assert rel_l2_plain(Qg, Qo) < 1e-5


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
@pytest.mark.parametrize("form", ["fused", "table1"])
def test_euler3d_n3_fp32(precision, form):
    if form == "table1" and precision != "fp32":
        pytest.skip("Table 1 form compiled for FP32 only")
    w = wl.euler_3d(grid=(5, 4, 3), steps=6)
    P = orc.Problem(3, 3, EUL, w.grid, w.dx, cst=w.cst)
    Q0 = wl.init_state(w, coords(P))
    Qg, dtg, _, _ = run_gpu(P, Q0, w.steps, precision=precision, form=form)
    Qo, _, _, _ = orc.run(P, Q0, w.steps, dt_seq=dtg)
    assert rel_l2_plain(Qg, Qo) < 1e-5
    assert rel_l2_plain(Qg - Q0, Qo - Q0) < 1e-3  # the change itself, not just the mean state


@pytest.mark.parametrize("form", ["fused", "table1"])
def test_elasticity3d_n4_fp32_material(form):
    w = wl.elasticity_3d(grid=(5, 3, 3), steps=5)
    w.extra["sigma"] = 0.15
    mat = wl.materials(w)
    P = orc.Problem(3, 4, ELA, w.grid, w.dx, cst=w.cst, mat=mat.astype(np.float32).astype(np.float64))
    Q0 = wl.init_state(w, coords(P))
    Qg, dtg, _, _ = run_gpu(P, Q0, w.steps, precision="fp32", form=form, mat=mat)
    Qo, _, _, _ = orc.run(P, Q0, w.steps, dt_seq=dtg)
    assert rel_l2_plain(Qg, Qo) < 1e-5


# ---------------------------------------------------------------- edge cases

def test_single_cell_periodic_grid():
    P = orc.Problem(3, 2, ACO, (1, 1, 1), (1.0, 1.0, 1.0), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 50)
    Qo, _, _, _ = orc.run(P, Q0, 2)
    Qg, _, _, _ = run_gpu(P, Q0, 2, precision="fp64")
    tight(Qg, Qo)


def test_zero_steps_is_noop():
    import torch
    P = orc.Problem(2, 2, ACO, (3, 3), (1 / 3, 1 / 3), cst=(1.0, 1.0))
    h = A.aderdg_create(2, 2, 3, A.ACOUSTICS, (3, 3), (1 / 3, 1 / 3), A.params(pde_const=(1.0, 1.0)))
    Q = torch.ones(P.C, 3, P.NS, device="cuda")
    assert A.aderdg_step(h, Q, 0) == 0.0
    assert torch.all(Q == 1)
    A.aderdg_destroy(h)


def test_nonfinite_state_is_reported():
    import torch
    P = orc.Problem(2, 2, EUL, (4, 3), (0.25, 1 / 3), cst=(1.4,))
    Q0 = euler_state(P, 1)
    Q0[5, 0, 3] = np.nan
    h = A.aderdg_create(2, 2, 4, A.EULER, (4, 3), (0.25, 1 / 3), A.params(pde_const=(1.4,)))
    Q = torch.from_numpy(Q0.astype(np.float32)).cuda()
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_step(h, Q, 2)
    assert e.value.status == A.ADERDG_ENONFINITE
    A.aderdg_destroy(h)


def test_unsupported_configuration():
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(3, 6, 5, A.EULER, (2, 2, 2), (0.5, 0.5, 0.5), A.params(pde_const=(1.4,), precision="fp64"))
    assert e.value.status == A.ADERDG_EUNSUPPORTED


def test_host_entry_point_matches_device():
    import torch
    P = orc.Problem(2, 3, ACO, (6, 5), (1 / 6, 1 / 5), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 60).astype(np.float32)
    Qd, _, td, _ = run_gpu(P, Q0.astype(np.float64), 4, precision="fp32")
    h = A.aderdg_create(2, 3, 3, A.ACOUSTICS, (6, 5), (1 / 6, 1 / 5), A.params(pde_const=(1.0, 1.0), cfl=P.cfl))
    host = torch.from_numpy(Q0.copy()).pin_memory()
    th = A.aderdg_step_host(h, host, 4)
    A.aderdg_destroy(h)
    assert th == td
    np.testing.assert_array_equal(host.numpy().astype(np.float64), Qd)


def test_begin_advance_end_equals_step():
    import torch
    P = orc.Problem(2, 2, EUL, (7, 5), (1 / 7, 1 / 5), cst=(1.4,))
    Q0 = euler_state(P, 61).astype(np.float32)
    Qa, _, ta, _ = run_gpu(P, Q0.astype(np.float64), 5, precision="fp32")
    h = A.aderdg_create(2, 2, 4, A.EULER, (7, 5), (1 / 7, 1 / 5), A.params(pde_const=(1.4,), cfl=P.cfl))
    Q = torch.from_numpy(Q0.copy()).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())   # torch pool streams do not wait on the default stream
    A.aderdg_begin(h, Q, 0.0, s)
    A.aderdg_advance(h, Q, 2, s)
    A.aderdg_advance(h, Q, 2, s)
    tb = A.aderdg_end(h, Q, 0.0, s)
    A.aderdg_destroy(h)
    assert tb == ta
    np.testing.assert_array_equal(Q.double().cpu().numpy(), Qa)


# ---------------------------------------------------------------- full size

def test_c2_full_size_sampled_cells():
    """64^3 cells, N=5, FP32, two steps through the fused sweep at the
    workload's own CFL factor (the one the benchmark runs); sampled cells
    against the oracle's two-step result computed cell by cell."""
    import torch
    w = wl.acoustics_3d()
    P = orc.Problem(3, 5, ACO, w.grid, w.dx, cst=w.cst, cfl=w.cfl_value)
    xi, _ = orc.gauss_legendre(P.N)
    Q0 = wl.init_state(w, wl.node_coords(w.grid, w.dx, xi))
    Q0f = Q0.astype(np.float32)
    Qg, dtg, _, _ = run_gpu(P, Q0f.astype(np.float64), 2, precision="fp32")
    dt = dtg[0]
    assert w.cfl_value == 0.4
    assert np.allclose(dtg, 0.4 / (3 * 11) / 64)
    # cells near the pulse centre and a few random ones
    centre = (wl.uniform(w.seed, 3) * 64).astype(int)
    rng = np.random.default_rng(0)
    picks = [centre + rng.integers(-2, 3, size=3) for _ in range(10)] + [rng.integers(0, 64, 3) for _ in range(6)]
    cells = np.array(sorted({int((p[0] % 64) + 64 * ((p[1] % 64) + 64 * (p[2] % 64))) for p in picks}))

    def nbrs(c):
        x, y, z = c % 64, (c // 64) % 64, c // 4096
        out = [c]
        for dxyz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            out.append(((x + dxyz[0]) % 64) + 64 * (((y + dxyz[1]) % 64) + 64 * ((z + dxyz[2]) % 64)))
        return out

    ring = np.array(sorted({n for c in cells for n in nbrs(int(c))}))
    Qin = Q0f.astype(np.float64)
    Q1 = Qin.copy()
    Q1[ring] = orc.step_cells(P, Qin, dt, ring)
    Q2 = orc.step_cells(P, Q1, dt, cells)
    err = rel_l2_plain(Qg[cells], Q2)
    assert err < 1e-5, err
    # conservation of every component over the whole grid (GL quadrature)
    from tests.helpers import total
    np.testing.assert_allclose(total(P, Qg), total(P, Qin), rtol=0, atol=1e-6 * np.abs(total(P, Qin)).max() + 1e-9)


@pytest.mark.parametrize("form", ["fused", "hull3", "table1"])
def test_nonfinite_state_is_reported_linear(form):
    """Linear wave speeds do not depend on the state, so the kernels fold a
    finiteness check of the corrected state into the wave-speed reduction."""
    import torch
    P = orc.Problem(2, 2, ACO, (7, 5), (1 / 7, 1 / 5), cst=(1.0, 1.0))
    Q0 = random_smooth(P, 70)
    Q0[9, 1, 4] = np.inf
    h = A.aderdg_create(2, 2, 3, A.ACOUSTICS, (7, 5), (1 / 7, 1 / 5), A.params(pde_const=(1.0, 1.0), form=form))
    Q = torch.from_numpy(Q0.astype(np.float32)).cuda()
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_step(h, Q, 2)
    assert e.value.status == A.ADERDG_ENONFINITE
    A.aderdg_destroy(h)


@pytest.mark.parametrize("pde,d,N,grid", [(ACO, 3, 5, (16, 16, 16)), (ACO, 2, 6, (48, 48)),
                                          (ELA, 3, 4, (16, 16, 16))])
def test_long_run_stable_at_default_cfl(pde, d, N, grid):
    """400 steps of a sharp pulse at the default step size stay bounded."""
    import torch
    name = {ACO: "acoustics", ELA: "elasticity"}[pde]
    cst = (1.0, 1.0) if pde == ACO else (2.5, 5.0, 5 / math.sqrt(3))
    w = wl.Workload("s", name, d, N, grid, 400, cst=cst, seed=2, extra={"sigma": 0.05})
    xi, _ = A.aderdg_nodes(N)
    Q0 = wl.init_state(w, wl.node_coords(w.grid, w.dx, np.array(xi)))
    h = A.aderdg_create(d, N, w.m, pde, grid, w.dx, A.params(pde_const=cst))
    Q = torch.from_numpy(Q0).float().cuda()
    m0 = float(Q.abs().max())
    A.aderdg_step(h, Q, 400)
    A.aderdg_destroy(h)
    assert float(Q.abs().max()) < 8 * m0

@pytest.mark.parametrize("pde,d,N,m,cst", [(ACO, 3, 5, 4, (1.0, 1.0)), (ACO, 2, 2, 3, (1.0, 1.0)),
                                           (ELA, 3, 4, 9, (2.5, 5.0, 2.9)), (EUL, 3, 3, 5, (1.4,))])
def test_footprint_fused_against_table1(pde, d, N, m, cst):
    """Persistent bytes per cell (library scratch plus the FP32 state) of the fused
    form over the Table 1 form, which stores the space-time predictor and its face
    data, stay at or below the ratio of Corollary "hull": the fused form keeps D and
    time-averaged face data only."""
    import bench
    grid = (4, 4, 4)[:d]
    dx = tuple(1.0 / g for g in grid)
    fp = {}
    for form in ("fused", "table1"):
        h = A.aderdg_create(d, N, m, pde, grid, dx, A.params(pde_const=cst, precision="fp32", form=form))
        try:
            fp[form] = A.aderdg_footprint(h) + 4 * m * (N + 1) ** d
        finally:
            A.aderdg_destroy(h)
    assert fp["fused"] / fp["table1"] <= bench.hull_footprint_ratio(d, N)
