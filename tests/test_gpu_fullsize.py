"""Full-size configurations in the launch configuration bench.py times,
checked on sampled cells against the FP64 oracle.

The GPU runs two fused steps of the whole grid.  The oracle repeats them
(Algorithm 1 with the GPU's two dt values, cell by cell) for the sampled cells:
the first step on the sampled cells and their face neighbours, the second on
the sampled cells.  The oracle's state array is allocated full size but only
the pages of the cells it touches are ever written (np.zeros maps lazily)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, rel_l2_plain

pytestmark = pytest.mark.gpu


def face_neighbours(c, grid):
    d = len(grid)
    x = [c % grid[0], (c // grid[0]) % grid[1]] + ([c // (grid[0] * grid[1])] if d == 3 else [])
    out = {c}
    for j in range(d):
        for s in (-1, 1):
            y = list(x)
            y[j] = (y[j] + s) % grid[j]
            out.add(y[0] + grid[0] * (y[1] + (grid[1] * y[2] if d == 3 else 0)))
    return out


def sample_cells(grid, seed, k=12):
    rng = np.random.default_rng(seed)
    C = int(np.prod(grid))
    picks = {int(v) for v in rng.integers(0, C, k)}
    picks |= {0, C - 1}  # the periodic corners
    return sorted(picks)


def gpu_initial_state(w, dtype):
    import torch
    xi, _ = A.aderdg_nodes(w.N)
    X = wl.node_coords(w.grid, w.dx, xi, xp=torch, device="cuda")
    Q = wl.init_state(w, X, xp=torch).to(dtype)
    del X
    return Q


def totals(w, Q):
    """Integral of every variable over the periodic domain (GL quadrature, FP64 sums)."""
    import torch
    _, wq = A.aderdg_nodes(w.N)
    wq = torch.tensor(wq, dtype=torch.float64, device=Q.device)
    W = wq
    for _ in range(w.d - 1):
        W = torch.outer(wq, W).reshape(-1)
    return (Q.double() * W).sum(dim=(0, 2)) * float(np.prod(w.dx))


def two_step_check(w, P, precision, mat=None, tol=1e-5, k=12):
    import torch
    tdt = torch.float64 if precision in ("fp64", "fp32_acc64") else torch.float32
    Q0 = gpu_initial_state(w, tdt)
    h = A.aderdg_create(w.d, w.N, w.m, A.PDE_IDS[w.pde], w.grid, w.dx,
                        A.params(pde_const=w.cst, precision=precision, cfl=w.cfl_value))
    try:
        if mat is not None:
            A.aderdg_set_material(h, torch.from_numpy(mat.astype(np.float32)).cuda())
        Q = Q0.clone()
        torch.cuda.synchronize()
        A.aderdg_step(h, Q, 2)
        dt = A.aderdg_get_dt_history(h)
    finally:
        A.aderdg_destroy(h)
    assert len(dt) == 2
    cells = sample_cells(w.grid, 11, k)
    ring = sorted({n for c in cells for n in face_neighbours(c, w.grid)})
    ring2 = sorted({n for c in ring for n in face_neighbours(c, w.grid)})
    idx = torch.tensor(ring2, device="cuda")
    Qh = np.zeros((P.C, P.m, P.NS))          # touched only where written
    Qh[ring2] = Q0[idx].double().cpu().numpy()
    Qh[ring] = orc.step_cells(P, Qh, dt[0], ring)
    ref = orc.step_cells(P, Qh, dt[1], cells)
    cidx = torch.tensor(cells, device="cuda")
    got = Q[cidx].double().cpu().numpy()
    q0c = Q0[cidx].double().cpu().numpy()
    err = rel_l2_plain(got, ref)
    assert np.isfinite(got).all()
    assert err < tol, err
    # conservation of every variable over the whole periodic grid, relative
    # to the state's magnitude (some variables integrate to exactly zero)
    t0, t2 = totals(w, Q0), totals(w, Q)
    scale = float(totals(w, Q0.abs()).max())
    assert float((t2 - t0).abs().max()) < 1e-6 * scale
    return err, rel_l2_plain(got - q0c, ref - q0c)


def test_c3_euler_128_full_size_sampled_cells():
    """128^3 cells, N=3, FP32 predictor with FP64 Q (the c3 bench workload).
    Only Q is compared: with uniform pressure and zero velocity the state is
    steady up to the Rusanov dissipation of inter-cell density jumps, which at
    this resolution are about 1e-10, so the change itself is at the level of
    FP32 rounding."""
    w = wl.euler_3d()
    P = orc.Problem(3, 3, orc.EULER, w.grid, w.dx, cst=w.cst, cfl=w.cfl_value)
    two_step_check(w, P, "fp32_acc64")


def test_c4_elasticity_96_full_size_sampled_cells():
    """96^3 cells, N=4, per-cell material, FP32 (the c4 workload), with a wider
    pulse so that the sampled cells see non-trivial updates."""
    w = wl.elasticity_3d()
    w.extra["sigma"] = 0.2
    mat = wl.materials(w)
    P = orc.Problem(3, 4, orc.ELASTICITY, w.grid, w.dx, cst=w.cst, cfl=w.cfl_value,
                    mat=mat.astype(np.float32).astype(np.float64))
    two_step_check(w, P, "fp32", mat=mat)


def test_c5_ensemble_full_size_sampled_scenarios():
    """All 512 scenarios packed and stepped together (graph mode, autotuned);
    sampled cells of the largest scenario of each PDE and a few random ones
    against the oracle run of that scenario."""
    import torch
    ws = wl.ensemble()
    b = A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, w.dx, pde_const=w.cst, cfl=w.cfl_value) for w in ws])
    try:
        off = A.aderdg_batch_offsets(b, len(ws))
        Q0 = torch.zeros(off[-1], dtype=torch.float32, device="cuda")
        for s, w in enumerate(ws):
            q = gpu_initial_state(w, torch.float32).reshape(-1)
            Q0[off[s]:off[s] + q.numel()] = q
        A.aderdg_batch_autotune(b, Q0, 3)
        Q = Q0.clone()
        torch.cuda.synchronize()
        A.aderdg_batch_step(b, Q, 2)
    finally:
        A.aderdg_batch_destroy(b)
    picks = {max(range(len(ws)), key=lambda s: ws[s].cells if ws[s].pde == p else -1) for p in ("acoustics", "elasticity")}
    picks |= {3, 100, 257, 511}
    for s in sorted(picks):
        w = ws[s]
        P = orc.Problem(2, w.N, orc.PDE_NAMES[w.pde], w.grid, w.dx, cst=w.cst, cfl=w.cfl_value)
        S = w.cells * w.m * (w.N + 1) ** 2
        q0 = Q0[off[s]:off[s] + S].double().cpu().numpy().reshape(w.cells, w.m, -1)
        q2 = Q[off[s]:off[s] + S].double().cpu().numpy().reshape(w.cells, w.m, -1)
        ref, _, _, _ = orc.run(P, q0, 2) if w.cells <= 4096 else (None, None, None, None)
        if ref is not None:
            assert rel_l2_plain(q2, ref) < 1e-5, s
            continue
        cells = sample_cells(w.grid, s, 8)
        # linear PDE with uniform material: the wave speed, hence dt, is the same every step
        dt0 = w.cfl_value * min(w.dx) / (2 * (2 * w.N + 1)) / orc.lam(P, q0)
        ring = sorted({n for c in cells for n in face_neighbours(c, w.grid)})
        qh = q0.copy()
        qh[ring] = orc.step_cells(P, q0, dt0, ring)
        ref = orc.step_cells(P, qh, dt0, cells)
        assert rel_l2_plain(q2[cells], ref) < 1e-5, s


def test_state_beyond_2_31_elements():
    """3D acoustics N=5 on 160^3 cells: 3.54e9 state elements, past the 32-bit
    index range; sampled cells at the end of the state against the oracle."""
    w = wl.acoustics_3d(grid=(160, 160, 160))
    w.extra["sigma"] = 0.3
    assert w.cells * w.m * (w.N + 1) ** 3 > 2 ** 31
    P = orc.Problem(3, 5, orc.ACOUSTICS, w.grid, w.dx, cst=w.cst, cfl=w.cfl_value)
    try:
        probe = np.zeros((P.C, P.m, P.NS))   # the oracle's full-size (lazily touched) state
        del probe
    except MemoryError:
        pytest.skip("host cannot reserve the oracle's full-size state array")
    import torch
    Q0 = gpu_initial_state(w, torch.float32)
    h = A.aderdg_create(3, 5, 4, A.ACOUSTICS, w.grid, w.dx, A.params(pde_const=w.cst, cfl=w.cfl_value))
    try:
        Q = Q0.clone()
        torch.cuda.synchronize()
        A.aderdg_step(h, Q, 2)
        dt = A.aderdg_get_dt_history(h)
    finally:
        A.aderdg_destroy(h)
    C = w.cells
    cells = [C - 1, C - 2, C - 161, C - 160 * 160 - 5, C // 2 + 7, 1234567]
    ring = sorted({n for c in cells for n in face_neighbours(c, w.grid)})
    ring2 = sorted({n for c in ring for n in face_neighbours(c, w.grid)})
    Qh = np.zeros((P.C, P.m, P.NS))
    Qh[ring2] = Q0[torch.tensor(ring2, device="cuda")].double().cpu().numpy()
    Qh[ring] = orc.step_cells(P, Qh, dt[0], ring)
    ref = orc.step_cells(P, Qh, dt[1], cells)
    got = Q[torch.tensor(cells, device="cuda")].double().cpu().numpy()
    assert rel_l2_plain(got, ref) < 1e-5


def test_c4_adjoint_full_size_properties():
    """96^3 cells, N=4, per-cell material, 64 receivers, FP32: with zero
    observations J is quadratic in Q0, so <dJ/dQ0, Q0> = 2 J; the gradients do
    not depend on the checkpoint spacing."""
    import torch
    w = wl.elasticity_3d()
    w.extra["sigma"] = 0.1
    mat = torch.from_numpy(wl.materials(w).astype(np.float32)).cuda()
    Q0 = gpu_initial_state(w, torch.float32)
    pos = torch.from_numpy(wl.receivers(w).astype(np.float32)).cuda()
    K = 12
    obs = torch.zeros((K, pos.shape[0], 3), dtype=torch.float32, device="cuda")
    h = A.aderdg_create(3, 4, 9, A.ELASTICITY, w.grid, w.dx, A.params(pde_const=w.cst, cfl=w.cfl_value))
    try:
        A.aderdg_set_material(h, mat)
        out = []
        for ck in (4, 12):
            gQ = torch.zeros_like(Q0)
            gm = torch.zeros_like(mat)
            J = A.aderdg_step_adjoint(h, Q0, K, 0.0, pos, obs, gQ, gm, ck)
            out.append((J, gQ, gm))
    finally:
        A.aderdg_destroy(h)
    (J, gQ, gm), (J2, gQ2, gm2) = out
    assert J > 0 and math.isfinite(J)
    dot = float((gQ.double() * Q0.double()).sum())
    assert abs(dot - 2 * J) <= 1e-3 * 2 * J, (dot, 2 * J)
    assert abs(J2 - J) <= 1e-6 * J
    assert float((gQ2 - gQ).norm() / gQ.norm()) < 1e-5
    assert float((gm2 - gm).norm() / gm.norm()) < 1e-5
