"""Helpers for the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np

import paper_1801_08682_gb300.aderdg as A
from oracle import oracle as orc

TORCH_DT = {"fp32": "float32", "fp64": "float64", "fp32_acc64": "float64"}


def run_gpu(P: orc.Problem, Q0, nsteps, precision="fp32", form="fused", fixed_dt=0.0,
            predictor=A.PREDICT_AUTO, dt_policy=A.DT_STRICT, inject_step=0, inject_factor=1.0,
            mat=None, picard=None):
    """Step Q0 (float64 numpy, [C][m][NS]) on the GPU; returns (Q, dt history, t, stats)."""
    import torch
    prm = A.params(pde_const=P.cst[:8], cfl=P.cfl, picard_iters=picard or 0, precision=precision,
                   form=form, dt_policy=dt_policy, predictor=predictor, inject_step=inject_step,
                   inject_factor=inject_factor)
    h = A.aderdg_create(P.d, P.N, P.m, P.pde, P.grid[: P.d], P.dx[: P.d], prm)
    try:
        if mat is not None:
            A.aderdg_set_material(h, torch.from_numpy(np.asarray(mat, np.float32)).cuda())
        Q = torch.from_numpy(np.ascontiguousarray(Q0).astype(TORCH_DT[precision])).cuda()
        t = A.aderdg_step(h, Q, nsteps, fixed_dt)
        dts = A.aderdg_get_dt_history(h)
        stats = A.aderdg_get_stats(h)
        return Q.double().cpu().numpy(), np.array(dts), t, stats
    finally:
        A.aderdg_destroy(h)


def rel_l2_plain(A_, B):
    A_, B = np.asarray(A_), np.asarray(B)
    return float(np.sqrt(((A_ - B) ** 2).sum() / max((B ** 2).sum(), 1e-300)))
