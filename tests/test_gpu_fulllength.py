"""Error against the FP64 oracle at each 3D workload's stated run length.

The three 3D workloads are run for their full step counts (3D acoustics N = 5:
100 steps; 3D Euler N = 3: 200; 3D elasticity N = 4 with per-cell material:
300) at their own CFL factor, order, PDE constants and initial data, on a grid
the oracle finishes in well under a minute on the host cores (12^3, 16^3 and
8^3 cells; the same seeded fields, sampled on the coarser grid).  Every state
precision the workload is offered in is checked: plain FP32, the compensated
FP32 pair and (Euler) FP64 accumulation.  The oracle replays the GPU's step
sizes.  Tolerance: relative L2 (GL quadrature) <= 1e-5, the FP32 target; the
maximum norm is printed beside it.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import run_gpu
from tests.helpers import coords, rel_l2

pytestmark = pytest.mark.gpu

CASES = {
    "acoustics3d_n5_100_steps": (wl.acoustics_3d, 12, ("fp32", "fp32_pair")),
    "euler3d_n3_200_steps": (wl.euler_3d, 16, ("fp32_acc64", "fp32_pair")),
    "elasticity3d_n4_300_steps": (wl.elasticity_3d, 8, ("fp32", "fp32_pair")),
}


@pytest.mark.parametrize("name", list(CASES))
def test_error_at_the_workloads_full_length(name):
    make, side, precisions = CASES[name]
    w0 = make()
    w = w0.resized((side,) * 3)
    assert w.steps == w0.steps
    mat = None
    if w.pde == "elasticity":
        mat = wl.materials(w).astype(np.float32).astype(np.float64)
    P = orc.Problem(3, w.N, orc.PDE_NAMES[w.pde], w.grid, w.dx, cst=w.cst, mat=mat, cfl=w.cfl_value)
    Q0 = wl.init_state(w, coords(P))
    refs = {}
    for prec in precisions:
        Qg, dtg, _, _ = run_gpu(P, Q0, w.steps, precision=prec, mat=mat)
        assert len(dtg) == w.steps
        key = dtg.tobytes()
        if key not in refs:
            refs[key] = orc.run(P, Q0, w.steps, dt_seq=dtg)[0]
        Qo = refs[key]
        e2 = rel_l2(P, Qg, Qo)
        emax = float(np.abs(Qg - Qo).max() / np.abs(Qo).max())
        print(f"{name} {prec}: rel L2 {e2:.3e}, rel max {emax:.3e}")
        assert e2 <= 1e-5, (prec, e2)
