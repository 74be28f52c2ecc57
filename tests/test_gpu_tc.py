"""Tensor-core (TF32) flux-divergence contractions of the space-time
predictor (ADERDG_PREDICT_SPACETIME_TF32) against the FP64 oracle.

Tolerance: 1e-3 relative L2 on Q (the tensor-core target; TF32 keeps 10
mantissa bits, about 5e-4 relative per operand).  The change Q - Q0 is
checked too (1e-2), and the result must differ from the FP32 CUDA-core
form, so that a silent fall-back to it would fail."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, rel_l2_plain, run_gpu
from tests.helpers import coords

pytestmark = pytest.mark.gpu

ACO, EUL = orc.ACOUSTICS, orc.EULER


def euler_state(P, seed):
    X = coords(P)
    w = wl.Workload("e", "euler", P.d, P.N, P.grid[: P.d], 0, cst=(1.4,), seed=seed,
                    extra={"amp": 0.1, "kmax": 2})
    Q = wl.init_state(w, X)
    Q[:, 1] = 0.2 * np.sin(2 * math.pi * X[..., 1])
    Q[:, P.m - 1] += 0.5 * Q[:, 1] ** 2 / Q[:, 0]
    return Q


def check(P, Q0, steps, precision="fp32", ref_pred=A.PREDICT_SPACETIME):
    Qt, dtt, _, _ = run_gpu(P, Q0, steps, precision=precision, predictor=A.PREDICT_SPACETIME_TF32)
    Qf, _, _, _ = run_gpu(P, Q0, steps, precision=precision, predictor=ref_pred)
    Qo, _, _, _ = orc.run(P, Q0, steps, dt_seq=dtt)
    assert np.isfinite(Qt).all()
    assert rel_l2_plain(Qt, Qo) < 1e-3
    assert rel_l2_plain(Qt - Q0, Qo - Q0) < 1e-2
    assert rel_l2_plain(Qt, Qf) > 1e-9      # the TF32 path ran, not the FP32 one
    return rel_l2_plain(Qt, Qo), rel_l2_plain(Qf, Qo)


@pytest.mark.parametrize("N,grid", [(2, (7, 5)), (3, (6, 5))])
def test_euler2d_tf32(N, grid):
    P = orc.Problem(2, N, EUL, grid, tuple(1.0 / g for g in grid), cst=(1.4,))
    check(P, euler_state(P, 70 + N), 5)


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64"])
def test_euler3d_n3_tf32(precision):
    w = wl.euler_3d(grid=(5, 4, 3), steps=6)
    P = orc.Problem(3, 3, EUL, w.grid, w.dx, cst=w.cst)
    Q0 = wl.init_state(w, coords(P))
    check(P, Q0, w.steps, precision)


def test_euler3d_n2_tf32_ragged_tile():
    # 24 cells in tiles of 9 (the last holds 6); N=2 pads K and N from 3 to 8
    P = orc.Problem(3, 2, EUL, (4, 3, 2), (0.25, 1 / 3, 0.5), cst=(1.4,))
    check(P, euler_state(P, 5), 4)


def test_acoustics3d_n3_tf32_spacetime():
    w = wl.acoustics_3d(grid=(4, 3, 5), N=3, steps=5)
    w.extra["sigma"] = 0.15
    P = orc.Problem(3, 3, ACO, w.grid, w.dx, cst=w.cst)
    Q0 = wl.init_state(w, coords(P))
    check(P, Q0, w.steps, ref_pred=A.PREDICT_AUTO)   # FP32 reference: the time-modal form


def test_tf32_not_compiled_for_fp64():
    with pytest.raises(A.AderdgError):
        A.aderdg_create(2, 3, 4, A.EULER, (4, 4), (0.25, 0.25),
                        A.params(pde_const=(1.4,), precision="fp64", predictor=A.PREDICT_SPACETIME_TF32))
