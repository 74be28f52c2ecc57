"""The compensated FP32 pair (precision FP32_PAIR): the state keeps an FP32
plane and a plane of low-order words, and the corrector adds each update by
TwoSum into the pair.  The predictor and the Riemann solver stay FP32.

What pins it
  * against the FP64 oracle: relative L2 <= 1e-5, the FP32 tolerance;
  * against FP64 accumulation of the same FP32 updates (FP32_ACC64): both feed
    the predictor the state rounded to FP32 and add the same FP32 increments,
    one exactly up to 2^-48 (hi + lo), the other in FP64; so after many steps
    hi + lo agrees with the FP64 state to far better than the plain FP32 state
    does (its accumulation rounds to 2^-24 every step);
  * the pair stays normalised: fl32(hi + lo) = hi for every DoF;
  * the host-resident entry point moves both planes (bitwise equal results).
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, device_state, host_values, rel_l2_plain, run_gpu
from tests.test_gpu_parity import euler_state, random_smooth

pytestmark = pytest.mark.gpu

ACO, EUL, ELA = orc.ACOUSTICS, orc.EULER, orc.ELASTICITY


@pytest.mark.parametrize("case", ["acoustics2d_n3", "acoustics3d_n2", "euler2d_n2", "elasticity2d_n3",
                                  "acoustics2d_n3_hull3"])
def test_pair_matches_oracle(case):
    form = "hull3" if case.endswith("hull3") else "fused"
    if case.startswith("acoustics2d"):
        P = orc.Problem(2, 3, ACO, (9, 7), (1 / 9, 1 / 7), cst=(1.2, 0.8), cfl=0.6)
        Q0 = random_smooth(P, 3)
    elif case == "acoustics3d_n2":
        P = orc.Problem(3, 2, ACO, (5, 4, 6), (1 / 5, 1 / 4, 1 / 6), cst=(1.0, 1.0), cfl=0.7)
        Q0 = random_smooth(P, 4)
    elif case == "euler2d_n2":
        P = orc.Problem(2, 2, EUL, (9, 7), (1 / 9, 1 / 7), cst=(1.4,), cfl=0.7)
        Q0 = euler_state(P, 5)
    else:
        C = 9 * 7
        rng = np.random.default_rng(6)
        mat = np.stack([rng.uniform(2, 3, C), rng.uniform(4, 6, C), np.zeros(C)], 1)
        mat[:, 2] = mat[:, 1] / math.sqrt(3)
        mat = mat.astype(np.float32).astype(np.float64)
        P = orc.Problem(2, 3, ELA, (9, 7), (1 / 9, 1 / 7), cst=(2.5, 5.0, 5 / math.sqrt(3)), mat=mat, cfl=0.6)
        Q0 = random_smooth(P, 6)
    Qg, dtg, _, _ = run_gpu(P, Q0, 6, precision="fp32_pair", form=form,
                            mat=P.mat if P.pde == ELA else None)
    Qo, _, _, _ = orc.run(P, Q0, 6, dt_seq=dtg)
    assert rel_l2_plain(Qg, Qo) <= 1e-5


def _acoustics_long(precision, steps=200):
    P = orc.Problem(2, 3, ACO, (16, 16), (1 / 16, 1 / 16), cst=(1.0, 1.0), cfl=0.6)
    Q0 = random_smooth(P, 11, base=(2.0, 0.5, -0.3))
    import torch
    prm = A.params(pde_const=P.cst[:8], cfl=P.cfl, precision=precision)
    h = A.aderdg_create(2, 3, 3, A.ACOUSTICS, (16, 16), P.dx[:2], prm)
    try:
        Q = device_state(Q0.astype(np.float32).astype(np.float64), precision)
        A.aderdg_step(h, Q, steps)
        return Q
    finally:
        A.aderdg_destroy(h)


def test_pair_tracks_fp64_accumulation():
    Q32 = host_values(_acoustics_long("fp32"), "fp32")
    Qp_dev = _acoustics_long("fp32_pair")
    Qp = host_values(Qp_dev, "fp32_pair")
    Q64 = host_values(_acoustics_long("fp32_acc64"), "fp32_acc64")
    e32 = rel_l2_plain(Q32, Q64)
    ep = rel_l2_plain(Qp, Q64)
    print(f"200 steps: FP32 state vs FP64 accumulation {e32:.2e}, pair {ep:.2e}")
    assert e32 > 1e-8                     # plain FP32 accumulation does drift
    assert ep <= 1e-9 and ep <= 1e-2 * e32
    # normalised: the FP32 plane is the pair rounded to FP32
    q = Qp_dev.double().cpu().numpy()
    np.testing.assert_array_equal((q[0] + q[1]).astype(np.float32), Qp_dev[0].cpu().numpy())


@pytest.mark.parametrize("nsteps", [1, 3])
def test_pair_host_entry_point_matches_device(nsteps):
    import torch
    w = wl.acoustics_3d(grid=(10, 9, 8))
    w.extra["sigma"] = 0.15
    xi, _ = A.aderdg_nodes(w.N)
    Q0 = wl.init_state(w, wl.node_coords(w.grid, w.dx, xi))
    prm = A.params(pde_const=w.cst, precision="fp32_pair")
    out = []
    for host in (False, True):
        h = A.aderdg_create(3, 5, 4, A.ACOUSTICS, w.grid, w.dx, prm)
        try:
            q = device_state(Q0, "fp32_pair")
            if host:
                qh = q.cpu().pin_memory()
                t = A.aderdg_step_host(h, qh, nsteps)
                out.append((qh.clone(), t))
            else:
                t = A.aderdg_step(h, q, nsteps)
                out.append((q.cpu(), t))
        finally:
            A.aderdg_destroy(h)
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])
    assert float(out[0][0][1].abs().max()) > 0.0      # the low words are in use


def test_pair_not_offered_where_no_low_words_are_kept():
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(3, 5, 4, A.ACOUSTICS, (4, 4, 4), (0.25,) * 3,
                        A.params(pde_const=(1.0, 1.0), precision="fp32_pair", form="table1"))
    assert e.value.status == A.ADERDG_EUNSUPPORTED
