"""Helpers for the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np

import paper_1801_08682_gb300.aderdg as A
from oracle import oracle as orc

TORCH_DT = {"fp32": "float32", "fp64": "float64", "fp32_acc64": "float64", "fp32_pair": "float32"}


def device_state(Q0, precision):
    """The device state of Q0 (float64 numpy): the compensated pair keeps the
    FP32 state and its low-order words lo = fl(Q0 - hi) as two planes."""
    import torch
    Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
    if precision == "fp32_pair":
        hi = Q0.astype(np.float32)
        lo = (Q0 - hi.astype(np.float64)).astype(np.float32)
        return torch.from_numpy(np.stack([hi, lo])).cuda()
    return torch.from_numpy(Q0.astype(TORCH_DT[precision])).cuda()


def host_values(Q, precision):
    """float64 numpy values of a device state (hi + lo for the pair)."""
    q = Q.double().cpu().numpy()
    return q[0] + q[1] if precision == "fp32_pair" else q


def library_sources(P: orc.Problem):
    """The oracle problem's point sources as the library's aderdg_source list."""
    return [A.source(tuple(s.pos), tuple(s.amp), kind=s.kind, t0=s.t0, f0=s.f0, coef=tuple(s.coef))
            for s in P.sources]


def run_gpu(P: orc.Problem, Q0, nsteps, precision="fp32", form="fused", fixed_dt=0.0,
            predictor=A.PREDICT_AUTO, dt_policy=A.DT_STRICT, inject_step=0, inject_factor=1.0,
            mat=None, picard=None):
    """Step Q0 (float64 numpy, [C][m][NS]) on the GPU; returns (Q, dt history, t, stats).
    The problem's material-jump form and point sources carry over."""
    import torch
    prm = A.params(pde_const=P.cst[:8], cfl=P.cfl, picard_iters=picard or 0, precision=precision,
                   form=form, dt_policy=dt_policy, predictor=predictor, inject_step=inject_step,
                   inject_factor=inject_factor,
                   material_jumps=A.JUMPS_NONCONSERVATIVE if P.ncp else A.JUMPS_PER_CELL_FLUX)
    h = A.aderdg_create(P.d, P.N, P.m, P.pde, P.grid[: P.d], P.dx[: P.d], prm)
    try:
        if mat is not None:
            A.aderdg_set_material(h, torch.from_numpy(np.asarray(mat, np.float32)).cuda())
        if P.sources:
            A.aderdg_set_sources(h, library_sources(P))
        Q = device_state(Q0, precision)
        t = A.aderdg_step(h, Q, nsteps, fixed_dt)
        dts = A.aderdg_get_dt_history(h)
        stats = A.aderdg_get_stats(h)
        return host_values(Q, precision), np.array(dts), t, stats
    finally:
        A.aderdg_destroy(h)


def rel_l2_plain(A_, B):
    A_, B = np.asarray(A_), np.asarray(B)
    return float(np.sqrt(((A_ - B) ** 2).sum() / max((B ** 2).sum(), 1e-300)))
