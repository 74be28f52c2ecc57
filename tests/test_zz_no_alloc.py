"""aderdg_step_noalloc: the fused step for callers that may not allocate device
memory while they run (its scratch is a fixed device array inside the
library).  Checked against the handle-based aderdg_step on two calls in a row,
which also checks that the shared scratch left by the first call does not leak
into the second.  Both paths run the same kernels on the same inputs with the
same time-step sequence, and the wave-speed maximum does not depend on the
order of its atomic updates, so the states must agree bit for bit.  This file
is collected last."""
import math

import numpy as np
import pytest

import paper_1801_08682_gb300.aderdg as A
from paper_1801_08682_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def smooth_state(grid, N, m, seed):
    d = len(grid)
    xi, _ = A.aderdg_nodes(N)
    X = wl.node_coords(grid, tuple(1.0 / g for g in grid), np.array(xi))
    rng = np.random.default_rng(seed)
    Q = np.zeros((X.shape[0], m, X.shape[1]))
    for c in range(m):
        for _ in range(3):
            k = rng.integers(-2, 3, size=d)
            Q[:, c] += rng.standard_normal() * np.cos(2 * math.pi * (X @ k) + rng.random() * 6.28)
    return Q


@pytest.mark.parametrize("case", ["acoustics3d_fp32", "euler2d_fp64", "elasticity2d_fp32", "acoustics3d_pair"])
def test_noalloc_matches_step_on_two_calls(case):
    import torch
    if case == "acoustics3d_fp32":
        d, N, pde, grid, cst, prec = 3, 3, A.ACOUSTICS, (8, 6, 5), (1.0, 1.0), "fp32"
    elif case == "acoustics3d_pair":
        d, N, pde, grid, cst, prec = 3, 3, A.ACOUSTICS, (8, 6, 5), (1.0, 1.0), "fp32_pair"
    elif case == "euler2d_fp64":
        d, N, pde, grid, cst, prec = 2, 2, A.EULER, (9, 7), (1.4,), "fp64"
    else:
        d, N, pde, grid, cst, prec = 2, 3, A.ELASTICITY, (9, 7), (2.5, 5.0, 5 / math.sqrt(3)), "fp32"
    m = wl.num_vars({A.ACOUSTICS: "acoustics", A.EULER: "euler", A.ELASTICITY: "elasticity"}[pde], d)
    dx = tuple(1.0 / g for g in grid)
    Q0 = smooth_state(grid, N, m, 5)
    if pde == A.EULER:
        Q0[:, 0] = 1.0 + 0.1 * Q0[:, 0]
        Q0[:, 1:d + 1] *= 0.1
        Q0[:, d + 1] = 2.5 + 0.5 * (Q0[:, 1:d + 1] ** 2).sum(1) / Q0[:, 0]
    mat = None
    if pde == A.ELASTICITY:
        w = wl.Workload("m", "elasticity", d, N, grid, 0, seed=3)
        mat = torch.from_numpy(wl.materials(w).astype(np.float32)).cuda()
    prm = A.params(pde_const=cst, precision=prec)
    tdt = torch.float64 if prec == "fp64" else torch.float32

    h = A.aderdg_create(d, N, m, pde, grid, dx, prm)
    if mat is not None:
        A.aderdg_set_material(h, mat)
    if prec == "fp32_pair":   # two float planes: the FP32 state and its low-order words
        Q0 = np.stack([Q0, Q0 - Q0.astype(np.float32).astype(np.float64)])
    Qa = torch.from_numpy(Q0).to(tdt).cuda()
    ta1 = A.aderdg_step(h, Qa, 5)
    Qa1 = Qa.cpu().clone()
    ta2 = A.aderdg_step(h, Qa, 4, 0.0, ta1)
    Qa2 = Qa.cpu().clone()
    A.aderdg_destroy(h)

    Qb = torch.from_numpy(Q0).to(tdt).cuda()
    tb1 = A.aderdg_step_noalloc(d, N, m, pde, grid, dx, prm, mat, Qb, 5)
    Qb1 = Qb.cpu().clone()
    tb2 = A.aderdg_step_noalloc(d, N, m, pde, grid, dx, prm, mat, Qb, 4, 0.0, tb1)
    Qb2 = Qb.cpu().clone()

    assert tb1 == ta1 and tb2 == ta2
    assert torch.equal(Qb1, Qa1)
    assert torch.equal(Qb2, Qa2)
    assert np.abs(Qa2.double().numpy() - Q0).max() > 1e-4   # the state did change
    if prec == "fp32_pair":
        assert float(Qa2[1].abs().max()) > 0.0                # the low words are in use


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    import torch
    Q = torch.zeros(16, device="cuda")
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_step_noalloc(3, 5, 4, A.ACOUSTICS, (64, 64, 64), (1 / 64,) * 3,
                              A.params(pde_const=(1.0, 1.0)), None, Q, 1)
    assert e.value.status == A.ADERDG_EINVAL
