"""Ensembles (aderdg_batch_*): every scenario of a packed batch, advanced by
the persistent launch (with and without the CUDA graph) and by per-scenario
launches, equals the same scenario advanced alone through aderdg_step, and a
few scenarios equal the FP64 oracle within the FP32 tolerance."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, rel_l2_plain

pytestmark = pytest.mark.gpu


def make_scenarios(seed=7, count=10):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        N = 2 + s % 5
        pde = "acoustics" if s % 2 == 0 else "elasticity"
        side = (int(rng.integers(3, 12)), int(rng.integers(3, 12)))
        cst = (1.0, 1.0) if pde == "acoustics" else (2.5, 5.0, 5 / math.sqrt(3))
        w = wl.Workload(f"s{s}", pde, 2, N, side, 0, cst=cst, seed=100 + s, extra={"sigma": 0.12})
        out.append(w)
    return out


def state(w):
    xi, _ = A.aderdg_nodes(w.N)
    return wl.init_state(w, wl.node_coords(w.grid, w.dx, np.array(xi)))


def pack(Q0s, off):
    assert all(o % 32 == 0 for o in off)
    buf = np.full(off[-1], np.nan, np.float32)   # the gaps must never be read
    for s, q in enumerate(Q0s):
        assert off[s] + q.size <= off[s + 1]
        buf[off[s]:off[s] + q.size] = q.reshape(-1)
    return buf


def alone(w, Q0, nsteps):
    import torch
    h = A.aderdg_create(2, w.N, w.m, A.PDE_IDS[w.pde], w.grid, w.dx, A.params(pde_const=w.cst))
    Q = torch.from_numpy(Q0).float().cuda()
    A.aderdg_step(h, Q, nsteps)
    A.aderdg_destroy(h)
    return Q.double().cpu().numpy()


@pytest.mark.parametrize("mode", [A.BATCH_PER_SCENARIO, A.BATCH_GRAPH, A.BATCH_PERSISTENT])
def test_batch_matches_single_scenarios(mode):
    """Per-scenario mode first: its kernels must not depend on a single-scenario
    handle having been created in the process before."""
    import torch
    ws = make_scenarios()
    nsteps = 7   # odd: graph pairs plus one direct sweep
    b = A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, pde_const=w.cst) for w in ws])
    try:
        off = A.aderdg_batch_offsets(b, len(ws))
        Q0s = [state(w) for w in ws]
        Q = torch.from_numpy(pack(Q0s, off)).cuda()
        A.aderdg_batch_step(b, Q, nsteps, mode)
        A.aderdg_batch_step(b, Q, nsteps, mode)   # second call reuses the captured graph
        out = Q.double().cpu().numpy()
        assert np.isnan(out[off[1] - 1]) or off[0] + Q0s[0].size == off[1]   # gaps untouched
        for s, w in enumerate(ws):
            ref = alone(w, alone(w, Q0s[s], nsteps).reshape(Q0s[s].shape), nsteps)
            got = out[off[s]:off[s] + ref.size].reshape(ref.shape)
            assert rel_l2_plain(got, ref) < 1e-6, (s, w.pde, w.N)
    finally:
        A.aderdg_batch_destroy(b)


def test_batch_against_oracle_and_autotune():
    import torch
    ws = make_scenarios(seed=9, count=6)
    nsteps = 4
    b = A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, pde_const=w.cst) for w in ws])
    try:
        off = A.aderdg_batch_offsets(b, len(ws))
        Q0s = [state(w) for w in ws]
        Q = torch.from_numpy(pack(Q0s, off)).cuda()
        A.aderdg_batch_autotune(b, Q, 3)
        bps, tpi, _ = A.aderdg_batch_get_tuning(b)
        assert 1 <= bps <= 3 and tpi in (1, 2, 4, 8)
        A.aderdg_batch_step(b, Q, nsteps)
        out = Q.double().cpu().numpy()
        for s in (0, 1, 5):
            w = ws[s]
            P = orc.Problem(2, w.N, orc.PDE_NAMES[w.pde], w.grid, w.dx, cst=w.cst,
                            cfl=w.cfl_value)
            Qo, _, _, _ = orc.run(P, Q0s[s].astype(np.float32).astype(np.float64), nsteps)
            got = out[off[s]:off[s] + Qo.size].reshape(Qo.shape)
            assert rel_l2_plain(got, Qo) < 1e-5, s
    finally:
        A.aderdg_batch_destroy(b)


def test_batch_profile_counts_direct_fused_sweeps():
    import torch
    ws = make_scenarios(seed=3, count=4)
    b = A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, pde_const=w.cst) for w in ws])
    try:
        off = A.aderdg_batch_offsets(b, len(ws))
        Q = torch.from_numpy(pack([state(w) for w in ws], off)).cuda()
        A.aderdg_batch_profile(b, True)
        A.aderdg_batch_step(b, Q, 5, A.BATCH_PERSISTENT)
        ms, n = A.aderdg_batch_profile_read(b)
        assert n == 4 and ms > 0.0          # nsteps - 1 fused sweeps
        A.aderdg_batch_step(b, Q, 5, A.BATCH_GRAPH)
        assert A.aderdg_batch_profile_read(b)[1] == 0   # graph replays are not instrumented
        A.aderdg_batch_profile(b, False)
        _, _, launches = A.aderdg_batch_get_tuning(b)
        assert launches > 0
    finally:
        A.aderdg_batch_destroy(b)


def test_batch_degenerate_grids():
    """1 x 1, 1 x 7, 7 x 1 and 2 x 1 scenarios (periodic neighbours are the
    cell itself or its only partner) mixed with a normal one."""
    import torch
    specs = [("acoustics", 3, (1, 1)), ("elasticity", 2, (1, 7)), ("acoustics", 6, (7, 1)),
             ("elasticity", 4, (2, 1)), ("acoustics", 2, (9, 6))]
    ws = []
    for i, (pde, N, grid) in enumerate(specs):
        cst = (1.0, 1.0) if pde == "acoustics" else (2.5, 5.0, 5 / math.sqrt(3))
        ws.append(wl.Workload(f"g{i}", pde, 2, N, grid, 0, cst=cst, seed=40 + i, extra={"sigma": 0.3}))
    for mode in (A.BATCH_GRAPH, A.BATCH_PER_SCENARIO):
        b = A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, pde_const=w.cst) for w in ws])
        try:
            off = A.aderdg_batch_offsets(b, len(ws))
            Q0s = [state(w) for w in ws]
            Q = torch.from_numpy(pack(Q0s, off)).cuda()
            A.aderdg_batch_step(b, Q, 4, mode)
            out = Q.double().cpu().numpy()
            for s, w in enumerate(ws):
                ref = alone(w, Q0s[s], 4)
                got = out[off[s]:off[s] + ref.size].reshape(ref.shape)
                assert rel_l2_plain(got, ref) < 1e-6, (mode, s)
        finally:
            A.aderdg_batch_destroy(b)
