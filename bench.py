"""Benchmark of the single-touch ADER-DG step on GB300; prints one JSON line.

Default workload: 3D linear acoustics, m = 4, N = 5, 64^3 periodic cells,
Gaussian pressure pulse, FP32 state (the workload the headline metric is
quoted on).  A timed "step" is one fused single-touch sweep (corrector of
step s and predictor of step s+1, Algorithm 2) on inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload acoustics3d|euler3d|elasticity3d|advection2d|ensemble]
                  [--form fused|hull3|table1] [--predictor auto|spacetime|tf32]
                  [--no-compare] [--no-cpu-baseline]

--workload elasticity3d_adjoint times the discrete adjoint of the 3D
elasticity workload (96^3, N=4, per-cell material, 64 receivers): one
aderdg_step_adjoint call over `steps` steps with checkpoints every 30 steps
(forward, checkpointed recompute, adjoint sweeps, receiver misfit and the
gradients with respect to Q0 and the material).

--workload ensemble times the batched ensemble instead: 512 independent 2D
acoustic/elastic scenarios (side 16..256, N 2..6, FP32), one persistent
launch per sweep replayed from a CUDA graph, autotuned, against the same
scenarios advanced with one launch per scenario and sweep.

The default run (the 3D acoustics workload, one GPU) keeps the FP32 state with
its accumulation in the compensated FP32 pair (FP32 predictor and Riemann
solver).  It also measures every other workload and state precision and adds
them to the same JSON line under "configs": the acoustics workload with plain
FP32 and with FP64 accumulation of the state, 3D Euler (N=3, 128^3, FP64
state and the pair), 3D elasticity (N=4, 96^3, per-cell material; plain FP32
and the pair), the batched ensemble, and the
discrete adjoint of the elasticity workload at its stated 300 steps with
checkpoints every 30 steps.  Each sub-record carries its own value,
ms_per_step, roofline, clocks and accuracy against the oracle on a sample.
--no-configs leaves them out.

With N > 1 (torchrun) every rank runs an independent replica of the workload
on its own GPU (the method has no data-path exchange on one GPU per rank);
``value`` is the sum of all ranks' DoF updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoF-updates/s"
UNIT = "DoF-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="acoustics3d",
                    choices=["acoustics3d", "euler3d", "elasticity3d", "advection2d", "ensemble",
                             "elasticity3d_adjoint"])
    ap.add_argument("--checkpoint-every", type=int, default=30,
                    help="elasticity3d_adjoint: forward states kept every k steps")
    ap.add_argument("--no-material-gradient", action="store_true",
                    help="elasticity3d_adjoint: dJ/dQ0 only")
    ap.add_argument("--form", default="fused", choices=["fused", "hull3", "table1"])
    ap.add_argument("--precision", default="", choices=["", "fp32", "fp64", "fp32_acc64", "fp32_pair"],
                    help="state precision (default: the workload's)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default run: leave out the other workloads and precisions")
    ap.add_argument("--predictor", default="auto", choices=["auto", "spacetime", "tf32"],
                    help="tf32: space-time Picard with tensor-core flux-divergence contractions")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20,
                    help="host calls timed for the end-to-end rate (one step each)")
    ap.add_argument("--grid", type=int, default=0,
                    help="cells per axis (smaller case of the same workload, for profiling)")
    ap.add_argument("--rerun-study", action="store_true",
                    help="add the optimistic time-stepping study (rerun corollary of Sec. 5): "
                         "sweep times, the C_rerun bound, reruns per dt policy and C_dT")
    return ap.parse_args()


def workload(name):
    from paper_1801_08682_gb300 import workloads as wl
    return {"acoustics3d": wl.acoustics_3d, "euler3d": wl.euler_3d,
            "elasticity3d": wl.elasticity_3d, "advection2d": wl.advection_2d}[name]()


def precision_of(w, override=""):
    return override or {"fp32": "fp32", "fp64": "fp64", "fp32_acc64": "fp32_acc64"}[w.precision]


def dtype_tag(prec):
    """Arithmetic of the path: FP32 predictor and Riemann solver, and the type
    the state is accumulated in."""
    return {"fp32": "f32", "fp64": "f64", "fp32_acc64": "f32+f64acc", "fp32_pair": "f32+f32pairacc"}[prec]


STATE_DOC = {"fp32": "FP32 state, FP32 accumulation", "fp64": "FP64 throughout",
             "fp32_acc64": "FP64 state, FP64 accumulation of the FP32 update",
             "fp32_pair": "compensated FP32 pair state (hi, lo), TwoSum accumulation of the FP32 update"}


PRED_NAMES = {"auto": 0, "spacetime": 1, "tf32": 2}


def config_of(w, form, world, predictor="auto", prec=None):
    prec = prec or w.precision
    return {"workload": f"{w.name} {w.pde} d={w.d} N={w.N} m={w.m} grid={'x'.join(map(str, w.grid))}",
            "pde": w.pde, "d": w.d, "N": w.N, "m": w.m, "grid": list(w.grid), "cells": w.cells,
            "dofs": w.dofs, "precision": prec, "state": STATE_DOC[prec], "form": form, "predictor": predictor,
            "cfl": w.cfl_value,
            "picard_iters": w.N + 1, "parallelism": f"replicas{world}",
            "l2": "no flush: every timed sweep streams Q, D and the hull (>> 129 MB L2)"}


_FP32_PEAK = []


def fp32_peak_tflops():
    """FP32 FMA rate of this GPU, measured once per process by the library."""
    if not _FP32_PEAK:
        try:
            import paper_1801_08682_gb300.aderdg as A
            _FP32_PEAK.append(A.aderdg_fp32_fma_peak(5))
        except Exception:   # measurement only: a failure leaves the compute fraction out
            _FP32_PEAK.append(None)
    return _FP32_PEAK[0]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes of one fused sweep (per cell): Q r+w, D r+w, own hull
# write, own + neighbour hull read, per-cell material

def fused_bytes_per_cell(w, prec, per_cell_material=None):
    """Q read+write, D read+write, the cell's own face hull written, its own and
    its neighbours' facing face hull read, per-cell material.  Linear PDEs
    keep only q on the faces (the normal flux is A_j q), nonlinear ones keep
    q and F_j . n."""
    qb = 8 if prec in ("fp64", "fp32_acc64", "fp32_pair") else 4   # the pair: hi and lo
    rb = 8 if prec == "fp64" else 4
    n = w.N + 1
    S = w.m * n ** w.d
    Fs = w.m * n ** (w.d - 1)
    per_side = Fs * rb * (1 if w.pde != "euler" else 2)
    b = 2 * S * qb + 2 * S * rb + 2 * w.d * per_side + 4 * w.d * per_side
    if per_cell_material is None:
        per_cell_material = w.pde == "elasticity"
    if per_cell_material:
        b += 12 * (1 + 2 * w.d)
    return b


def operator_nnz(w, j):
    """Non-zero entries of the flux Jacobian A_j of a linear PDE."""
    if w.pde == "advection":
        return 1
    if w.pde == "acoustics":
        return 2
    return 3 * w.d + 1   # elasticity: d normal-stress, j+1 and d-j shear, d velocity entries


def sweep_flops_per_cell(w, picard=None):
    """Straightforward FP32 operation count of one fused sweep per cell
    (a multiply-add counts 2, other arithmetic 1; the kernels' even/odd and
    other savings are not subtracted).  n = N+1, NS = n^d, S = m NS,
    NF = n^(d-1), R Picard iterations (default N+1).
    Linear PDEs (time-modal predictor): R Horner passes and one Kvol pass,
    each with the line contractions of the components A_j reads (2n per
    output) and the application of A_j (2 per non-zero); extrapolation of
    q_bar to the 2d faces; the corrector's Rusanov fluxes on the 2d faces,
    the face integration and the update.
    Euler (space-time Picard, first iteration at one time node): per
    space-time node and iteration the flux in all d directions (about 30),
    the d derivative contractions of the m components (2 n each) and the
    time solve (2 n per component); time averages of q and of the fluxes,
    integrateVolume, extrapolation of q and F_j . n, and the corrector."""
    n, d, m = w.N + 1, w.d, w.m
    NS, NF, S = n ** d, n ** (d - 1), m * n ** d
    R = picard or (w.N + 1)
    if w.pde == "euler":
        per_tn = 30 + d * m * 2 * n + m * 2 * n
        picard_ops = NS * ((30 + d * m * 2 * n + m * 2 * n) + (R - 1) * n * per_tn)
        averages = NS * (m * 2 * n + n * 30 + d * m * 2 * n)
        volume = NS * d * m * 2 * n
        extrap = 2 * d * NF * 2 * m * 2 * n
        corrector = 2 * d * NF * (2 * 10 + 3 * m) + S * (4 * d + 2) + NS * 10
        return picard_ops + averages + volume + extrap + corrector
    reads = {"advection": lambda j: 1, "acoustics": lambda j: 2,
             "elasticity": lambda j: 2 * d}[w.pde]
    per_pass = sum(reads(j) * NS * 2 * n + NS * 2 * operator_nnz(w, j) for j in range(d))
    predictor = R * (per_pass + 2 * S) + per_pass
    extrap = 2 * d * m * NF * 2 * n
    corrector = 2 * d * NF * (4 * max(operator_nnz(w, j) for j in range(d)) + 4 * m) + S * (4 * d + 2)
    return predictor + extrap + corrector


def adjoint_bytes_per_cell(w, ce, material_gradient=True):
    """Algorithmic bytes per cell of one step of aderdg_step_adjoint on the
    elasticity workload (FP32, state S = m (N+1)^d values, face side
    Fs = m (N+1)^(d-1) values, per-cell material), summed over its sweeps:
      * forward run and checkpointed recompute: two fused sweeps (their own
        byte count), the segment's state copied out once (read + write) and
        every ce-th state checkpointed (read + write);
      * the STP sweep of the forward state: Q read, D and the face hull written;
      * adj_faces: lambda read, the face adjoints psi written (2d face sides);
      * adj_cell: lambda, Q and (own + neighbours') psi and hull read, the
        materials of the cell and its 2d neighbours read, lambda written, the
        material gradient (3 doubles) accumulated.
    Without the material gradient only the forward run, adj_faces and adj_cell
    without Q and hull remain."""
    n = w.N + 1
    S = w.m * n ** w.d * 4
    Fs = w.m * n ** (w.d - 1) * 4
    mat = 12 * (1 + 2 * w.d)
    sweep = fused_bytes_per_cell(w, "fp32")
    faces = S + 2 * w.d * Fs
    if not material_gradient:
        return sweep + faces + (S + 2 * 2 * w.d * Fs + mat + S)
    copies = 2 * S + 2 * S / ce
    stp = S + 12 + S + 2 * w.d * Fs
    cell = S + S + 2 * 2 * w.d * Fs + 2 * 2 * w.d * Fs + mat + S + 24
    return 2 * sweep + copies + stp + faces + cell


# the sources that define and launch the fused sweeps (line-owner and
# node-owner): the measured DRAM traffic of a profile summary stands while
# these are unchanged
FUSED_SWEEP_SOURCES = ("sweep_lin.cuh", "sweep.cuh", "tc.cuh", "common.cuh", "pde.cuh", "tma.cuh",
                       "kernels.cuh", "api.cu")


def hull_footprint_ratio(d, p):
    """Persistent footprint of the single-touch realisation over a straightforward
    three-step code (Corollary "hull", Sec. 5): Q, D, the extrapolated face data
    and the Riemann output, (2 + 6d) m (p+1)^d values, against the space-time
    predictor and fluxes plus Q, face data and Riemann output,
    (d+1) m (p+1)^(d+1) + (1 + 6d) m (p+1)^d."""
    return (2 + 6 * d) / ((d + 1) * (p + 1) + 1 + 6 * d)


def kernel_source_hash():
    from paper_1801_08682_gb300 import build as B
    h = hashlib.sha1()
    for name in FUSED_SWEEP_SOURCES:
        with open(os.path.join(B.CSRC, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def profiled_traffic(w, form, prec=None):
    """dram bytes per launch of the fused sweep from the committed ncu summary,
    if it was taken on the current kernel sources and the same state precision;
    else None."""
    path = os.path.join(ROOT, "profiles", f"fused_sweep_{w.name}.md")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            if line.startswith("bench-key:"):
                k, _, v = line.partition(":")[2].strip().partition("=")
                rec[k.strip()] = v.strip()
    if rec.get("source_hash") != kernel_source_hash() or form != "fused":
        return None
    try:   # one key per state precision the profile captured
        return float(rec[f"dram_bytes_per_launch_full.{prec or w.precision}"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# multi-rank aggregation (one process per GPU, each an independent replica)

def max_over_ranks(x, world, device="cuda"):
    """The largest x over all ranks (the slowest rank's time); x itself at N = 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units of all ranks over the slowest rank's time."""
    return units_per_rank * world / seconds_max


# ---------------------------------------------------------------------------
# GPU arm

def gpu_state(w, A):
    """The workload's initial state as a float64 CUDA tensor (fields evaluated on the GPU)."""
    import torch
    from paper_1801_08682_gb300 import workloads as wl
    xi, _ = A.aderdg_nodes(w.N)
    X = wl.node_coords(w.grid, w.dx, xi, xp=torch, device="cuda")
    Q = wl.init_state(w, X, xp=torch)
    del X
    return Q


def to_state(Q64, prec):
    """The device state of a float64 CUDA tensor in the given precision (the
    compensated pair: the FP32 plane and the low-order words fl(Q - hi))."""
    import torch
    if prec == "fp32_pair":
        hi = Q64.float()
        return torch.stack([hi, (Q64 - hi.double()).float()])
    return Q64.to(torch.float64 if prec in ("fp64", "fp32_acc64") else torch.float32)


def state_values(Q, prec):
    """float64 values of a device state (hi + lo for the pair)."""
    return Q[0].double() + Q[1].double() if prec == "fp32_pair" else Q.double()


def make_handle(w, A, form, prec, pred=0):
    import torch
    from paper_1801_08682_gb300 import workloads as wl
    pde = A.PDE_IDS[w.pde]
    h = A.aderdg_create(w.d, w.N, w.m, pde, w.grid[: w.d], w.dx,
                        A.params(pde_const=w.cst, precision=prec, form=form, cfl=w.cfl_value, predictor=pred))
    if w.pde == "elasticity":
        import numpy as np
        A.aderdg_set_material(h, torch.from_numpy(wl.materials(w).astype(np.float32)).cuda())
    return h


def time_form(w, A, Q0t, form, prec, steps, warmup, stream, profile_kernel=None, pred=0):
    """Time `steps` sweeps of one form; returns (ms, launches, kernel ms, kernel launches)."""
    import torch
    h = make_handle(w, A, form, prec, pred)
    try:
        Q = Q0t.clone()
        stream.wait_stream(torch.cuda.current_stream())   # the clone runs on torch's stream
        A.aderdg_begin(h, Q, 0.0, stream)
        A.aderdg_advance(h, Q, warmup, stream)
        stream.synchronize()
        l0 = A.aderdg_get_stats(h).launches
        if profile_kernel is not None:
            A.aderdg_profile(h, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A.aderdg_advance(h, Q, steps, stream)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1)
        launches = A.aderdg_get_stats(h).launches - l0
        kms, kn = (A.aderdg_profile_read(h, profile_kernel) if profile_kernel is not None else (0.0, 0))
        A.aderdg_profile(h, False)
        A.aderdg_end(h, Q, 0.0, stream)
        return ms, launches, kms, kn
    finally:
        A.aderdg_destroy(h)


def c_rerun_bound(t3, tf, tstp, r):
    """Largest sweeps-per-step count C_rerun at which the fused optimistic step
    still beats three separate sweeps (the rerun corollary, Sec. 5): one sweep
    per step plus one STP sweep per rerun, with the fused step's dt r times the
    baseline's."""
    return 1.0 + (t3 * r - tf) / tstp


def rerun_study(w, A, Q0t, prec, stream, steps):
    """The trade-off of the rerun corollary (Sec. 5): the fused optimistic step
    beats three separate sweeps while C_rerun < 1 + (T_3steps r - T_fused) /
    T_STP, with C_rerun the sweeps per step counting STP reruns and r the fused
    form's dt over the three-sweep form's (the corollary's damping C_dT; 1 when
    both use the same CFL factor, as the library does).  Measured: the three
    times (CUDA events; T_STP the STP sweep of the three-sweep form), the bound
    for several r, and `steps` Algorithm-2 steps from the workload's initial
    state per dt policy and CFL factor C_dT: reruns, observed C_rerun, simulated
    time reached per wall second; one more strict run has dt_adm cut in half
    after step steps/2 (a forced rerun) to price one rerun."""
    import torch
    ksteps = 10
    m3, _, kstp, nstp = time_form(w, A, Q0t, "hull3", prec, ksteps, 3, stream, profile_kernel=A.KERNEL_STP)
    mf, _, _, _ = time_form(w, A, Q0t, "fused", prec, ksteps, 3, stream)
    t3, tf, tstp = m3 / ksteps, mf / ksteps, kstp / max(nstp, 1)
    out = {"T_3steps_ms": t3, "T_fused_ms": tf, "T_STP_ms": tstp,
           "C_rerun_bound_by_dt_ratio": {f"{r:g}": c_rerun_bound(t3, tf, tstp, r) for r in (1.0, 0.99, 0.95, 0.9)},
           "steps": steps, "runs": []}
    pde = A.PDE_IDS[w.pde]
    cases = [(pol, c, 0, 1.0) for pol in (A.DT_STRICT, A.DT_CREEPING) for c in (0.4, 0.5, 0.6, 0.7)]
    cases.append((A.DT_STRICT, w.cfl_value, steps // 2, 0.5))
    for pol, c, inj, fac in cases:
        h = A.aderdg_create(w.d, w.N, w.m, pde, w.grid[: w.d], w.dx,
                            A.params(pde_const=w.cst, precision=prec, cfl=c, dt_policy=pol,
                                     inject_step=inj, inject_factor=fac))
        try:
            Q = Q0t.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t_sim = A.aderdg_step(h, Q, steps, 0.0, 0.0, stream)
            wall = time.perf_counter() - t0
            st = A.aderdg_get_stats(h)
        finally:
            A.aderdg_destroy(h)
        out["runs"].append({"policy": "strict" if pol == A.DT_STRICT else "creeping", "C_dT": c,
                            "forced_rerun_after_step": inj or None, "reruns": st.reruns,
                            "C_rerun": 1.0 + st.reruns / steps, "simulated_time": t_sim,
                            "wall_ms": wall * 1e3, "simulated_time_per_s": t_sim / wall})
    return out


def init_rank():
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def bench_workload(w, prec, form, pred_name, steps, warmup, rank, world, local, e2e_steps=20,
                   compare=False, cpu=False, rerun=False, oracle_budget=15.0):
    """One workload through the handle API: `steps` timed fused sweeps on the
    resident state (CUDA events on the library's stream, between barriers),
    the main kernel's own event time for the roofline, clocks during the timed
    region; optionally the end-to-end rate through the host entry point, the
    forms side by side, the rerun study and the oracle on a sample."""
    import torch
    import paper_1801_08682_gb300.aderdg as A

    Q0t = to_state(gpu_state(w, A), prec)
    stream = torch.cuda.Stream()
    pred = PRED_NAMES[pred_name]
    h = make_handle(w, A, form, prec, pred)
    Q = Q0t.clone()
    stream.wait_stream(torch.cuda.current_stream())   # the clone runs on torch's stream
    A.aderdg_begin(h, Q, 0.0, stream)
    A.aderdg_advance(h, Q, warmup, stream)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    l0 = A.aderdg_get_stats(h).launches
    main_kernel = {"fused": A.KERNEL_FUSED, "hull3": A.KERNEL_STP, "table1": A.KERNEL_T1_PREDICT}[form]
    A.aderdg_profile(h, True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.15)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    A.aderdg_advance(h, Q, steps, stream)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = A.aderdg_get_stats(h).launches - l0
    kms, kn = A.aderdg_profile_read(h, main_kernel)
    A.aderdg_profile(h, False)
    t_sim = A.aderdg_end(h, Q, 0.0, stream)
    A.aderdg_destroy(h)
    del Q
    ms_max = max_over_ranks(ms, world)
    value = whole_job_rate(w.dofs * steps, world, ms_max / 1e3)

    # roofline of the dominant kernel (the fused sweep)
    peak, peak_src = peaks()
    bpc = fused_bytes_per_cell(w, prec)
    alg_bytes = bpc * w.cells
    avg_s = (kms / kn) / 1e3 if kn else float("nan")
    achieved = alg_bytes / avg_s / 1e9 if kn else None
    kname = "lin_sweep_kernel" if (w.pde != "euler" and pred == 0) else "sweep_kernel"
    roof = {"bound": "hbm", "kernel": f"{kname}<{w.pde} d={w.d} N={w.N}, {prec}, fused>",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "peak_source": f"hbm_gbs of {peak_src}",
            "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_dof": bpc / (w.m * (w.N + 1) ** w.d),
            "kernel_ms_avg": avg_s * 1e3, "kernel_share_of_step": (kms / ms) if ms else None,
            "traffic": profiled_traffic(w, form, prec) if pred == 0 else None}
    if form != "fused":
        roof["kernel"] = f"main kernel of the {form} form"
    elif kn and fp32_peak_tflops():
        # the FP32 arithmetic beside the bytes: the binding roof is the larger fraction
        fpc = sweep_flops_per_cell(w)
        tflops = fpc * w.cells / avg_s / 1e12
        peak_f = fp32_peak_tflops()
        roof["compute"] = {"flops_per_dof": fpc / (w.m * (w.N + 1) ** w.d), "achieved_tflops": tflops,
                           "peak_tflops": peak_f, "peak_source": "aderdg_fp32_fma_peak on this GPU",
                           "frac": tflops / peak_f}
        if roof["frac"] is not None and tflops / peak_f > roof["frac"]:
            roof["binding"] = "alu"
        else:
            roof["binding"] = "hbm"

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
           "warmup": warmup, "ms_per_step": ms_max / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": dtype_tag(prec),
           "data": "synthetic (seeded Gaussian pulse / Fourier modes, generated on the GPU)",
           "config": config_of(w, form, world, pred_name, prec), "gpu_launches": launches,
           "launches_per_step": launches / steps, "simulated_time": t_sim,
           "roofline": roof, "clocks": clocks}

    if e2e_steps > 0:
        # end to end through the host entry point: H2D + step + D2H per step (every
        # rank: the slowest rank's time counts)
        hq = Q0t.cpu().pin_memory()
        torch.cuda.synchronize()
        h = make_handle(w, A, form, prec, pred)
        A.aderdg_step_host(h, hq, 1, 0.0, 0.0, stream)      # warm-up (allocates the staging buffer)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            A.aderdg_step_host(h, hq, 1, 0.0, 0.0, stream)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        A.aderdg_destroy(h)
        e2e_s = max_over_ranks(e2e_s, world)
        qbytes = hq.numel() * hq.element_size()
        out["e2e"] = {"value": whole_job_rate(w.dofs * e2e_steps, world, e2e_s), "unit": UNIT,
                      "h2d_bytes_per_step": qbytes, "d2h_bytes_per_step": qbytes,
                      "call": "aderdg_step_host(nsteps=1) per step: H2D Q, first STP sweep, "
                              "corrector sweep, D2H Q"}
        del hq

    if rank == 0 and compare and world == 1:
        # the multi-pass forms keep no low words: the forms are compared at plain FP32
        fprec = "fp32" if prec == "fp32_pair" else prec
        Qf = Q0t if fprec == prec else to_state(gpu_state(w, A), fprec)
        out["forms"] = compare_forms(w, A, Qf, fprec, pred, stream, max(5, min(30, steps // 10)))
        out["forms"]["precision"] = fprec
        del Qf
    if rank == 0 and rerun and world == 1:
        out["rerun_study"] = rerun_study(w, A, Q0t, prec, stream, max(20, min(steps, 100)))
    del Q0t
    if rank == 0 and cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, A, prec, pred, oracle_budget)
        out["accuracy"] = out["cpu_baseline"].pop("accuracy", None)
    torch.cuda.empty_cache()
    return out


def compare_forms(w, A, Q0t, prec, pred, stream, ksteps):
    """The fused form beside the three-sweep and Table 1 forms (same steps),
    and the persistent footprints of the fused and Table 1 forms."""
    cmp = {}
    for f in ("fused", "hull3", "table1"):
        try:
            mf, lf, _, _ = time_form(w, A, Q0t, f, prec, ksteps, 3, stream)
            cmp[f] = {"value": w.dofs * ksteps / (mf / 1e3), "ms_per_step": mf / ksteps,
                      "launches_per_step": lf / ksteps}
        except A.AderdgError as e:
            cmp[f] = {"unavailable": str(e)}
    if w.pde == "euler" or pred:
        # the space-time predictor with FP32 CUDA-core and TF32 tensor-core contractions
        for name, pv in (("fused_spacetime_fp32", 1), ("fused_spacetime_tf32", 2)):
            try:
                mf, lf, _, _ = time_form(w, A, Q0t, "fused", prec, ksteps, 3, stream, pred=pv)
                cmp[name] = {"value": w.dofs * ksteps / (mf / 1e3), "ms_per_step": mf / ksteps,
                             "launches_per_step": lf / ksteps}
            except A.AderdgError as e:
                cmp[name] = {"unavailable": str(e)}
    # persistent bytes per cell (library scratch + the state), fused against Table 1
    try:
        qb = Q0t.element_size() * w.m * (w.N + 1) ** w.d * (2 if prec == "fp32_pair" else 1)
        fp = {}
        for f in ("fused", "table1"):
            hf = make_handle(w, A, f, prec, pred)
            try:
                fp[f] = A.aderdg_footprint(hf) + qb
            finally:
                A.aderdg_destroy(hf)
        cmp["footprint"] = {"fused_bytes_per_cell": fp["fused"], "table1_bytes_per_cell": fp["table1"],
                            "ratio": fp["fused"] / fp["table1"],
                            "paper_corollary_ratio": hull_footprint_ratio(w.d, w.N)}
    except A.AderdgError as e:
        cmp["footprint"] = {"unavailable": str(e)}
    if "value" in cmp.get("fused", {}):
        for f in ("hull3", "table1"):
            if "value" in cmp.get(f, {}):
                cmp[f]["fused_speedup"] = cmp["fused"]["value"] / cmp[f]["value"]
    return cmp


def sub_record(rec):
    """The keys of a workload's line kept in the configs object of the default run."""
    keep = ("value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "gpu_launches",
            "launches_per_step", "roofline", "clocks", "accuracy", "cpu_baseline", "e2e", "forms",
            "misfit", "gradients_finite", "roofline_note", "timing")
    return {k: rec[k] for k in keep if k in rec}


def run_ours(args):
    import paper_1801_08682_gb300.aderdg as A
    rank, world, local = init_rank()
    A.load(build_if_missing=True)
    w = workload(args.workload)
    if args.grid:
        w = w.resized((args.grid,) * w.d)
    default = (args.workload == "acoustics3d" and not args.grid and args.form == "fused"
               and args.predictor == "auto" and not args.precision)
    # the headline keeps the workload's FP32 state and accumulates it in the
    # compensated FP32 pair: FP32 predictor and Riemann solver, compensated
    # accumulation of Q^{n+1} = Q^n + dt update
    prec = "fp32_pair" if default else precision_of(w, args.precision)
    out = bench_workload(w, prec, args.form, args.predictor, args.steps, args.warmup, rank, world, local,
                         e2e_steps=args.e2e_steps, compare=not args.no_compare,
                         cpu=not args.no_cpu_baseline, rerun=args.rerun_study)
    if default and not args.no_configs and world == 1:
        out["configs"] = other_configs(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def other_configs(args, rank, world, local):
    """The other workloads and state precisions, each with fewer timed steps
    than the headline line (the grids are the workloads' own)."""
    from paper_1801_08682_gb300 import workloads as wl
    k = max(3, min(args.steps, 10))
    wu = max(3, min(args.warmup, 5))
    cfg = {}
    wa = wl.acoustics_3d()
    for prec in ("fp32", "fp32_acc64"):
        cfg[f"acoustics3d_{prec}"] = sub_record(bench_workload(
            wa, prec, "fused", "auto", k * 2, wu, rank, world, local, e2e_steps=0, cpu=True, oracle_budget=3.0))
    we = wl.euler_3d()
    for prec in ("fp32_acc64", "fp32_pair"):
        cfg[f"euler3d_{prec}"] = sub_record(bench_workload(
            we, prec, "fused", "auto", k, wu, rank, world, local, e2e_steps=0, cpu=True, oracle_budget=3.0))
    for prec in ("fp32", "fp32_pair"):
        cfg[f"elasticity3d_{prec}"] = sub_record(bench_workload(
            wl.elasticity_3d(), prec, "fused", "auto", k, wu, rank, world, local, e2e_steps=0, cpu=True,
            oracle_budget=3.0))
    ea = argparse.Namespace(**vars(args))
    ea.steps, ea.warmup, ea.e2e_steps = k * 2, wu, 3
    cfg["ensemble"] = sub_record(ensemble_record(ea, rank, world, local, oracle_budget=3.0))
    aa = argparse.Namespace(**vars(args))
    aa.steps, aa.warmup, aa.checkpoint_every, aa.no_material_gradient = 300, 2, 30, False
    cfg["elasticity3d_adjoint"] = sub_record(adjoint_record(aa, rank, world, local))
    return cfg


# ---------------------------------------------------------------------------
# Batched ensemble

ENSEMBLE_NAME = "ensemble of 512 2D acoustics/elasticity scenarios, side 16..256, N 2..6, FP32"


def ensemble_state(ws, A, off):
    """Packed initial states of the scenarios (fields evaluated on the GPU)."""
    import torch
    from paper_1801_08682_gb300 import workloads as wl
    Q = torch.zeros(off[-1], dtype=torch.float32, device="cuda")
    for s, w in enumerate(ws):
        xi, _ = A.aderdg_nodes(w.N)
        X = wl.node_coords(w.grid, w.dx, xi, xp=torch, device="cuda")
        q = wl.init_state(w, X, xp=torch).float().reshape(-1)
        Q[off[s]:off[s] + q.numel()] = q
        del X
    return Q


def ensemble_batch(ws, A):
    return A.aderdg_batch_create([A.scenario(w.pde, w.N, w.grid, w.dx, pde_const=w.cst, cfl=w.cfl_value)
                                  for w in ws])


def ensemble_oracle_sample(budget_s):
    """The first scenarios of the ensemble, each on 16x16 cells (the smallest
    side drawn), as many as one FP64 oracle step covers in about budget_s."""
    from oracle import oracle as orc
    from paper_1801_08682_gb300 import workloads as wl
    cores = orc.set_threads(0)
    out, spent = [], 0.0
    for w in wl.ensemble():
        ws = w.resized((16, 16), steps=1)
        P = orc.Problem(2, ws.N, orc.PDE_NAMES[ws.pde], ws.grid, ws.dx, cst=ws.cst, cfl=ws.cfl_value)
        xi, _ = orc.gauss_legendre(ws.N)
        Q0 = wl.init_state(ws, wl.node_coords(ws.grid, ws.dx, xi))
        t0 = time.perf_counter()
        orc.run(P, Q0, 1)
        spent += time.perf_counter() - t0
        out.append((ws, P, Q0))
        if spent >= budget_s:
            break
    return out, cores


def run_ensemble(args):
    import paper_1801_08682_gb300.aderdg as A
    rank, world, local = init_rank()
    A.load(build_if_missing=True)
    out = ensemble_record(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def ensemble_record(args, rank, world, local, oracle_budget=12.0):
    import numpy as np
    import torch
    import paper_1801_08682_gb300.aderdg as A
    from paper_1801_08682_gb300 import workloads as wl

    ws = wl.ensemble()
    dofs = sum(w.dofs for w in ws)
    cells = sum(w.cells for w in ws)
    stream = torch.cuda.Stream()
    b = ensemble_batch(ws, A)
    try:
        off = A.aderdg_batch_offsets(b, len(ws))
        Q0 = ensemble_state(ws, A, off)
        torch.cuda.synchronize()
        A.aderdg_batch_autotune(b, Q0, 3, stream)
        bps, tpi, _ = A.aderdg_batch_get_tuning(b)
        Q = Q0.clone()
        stream.wait_stream(torch.cuda.current_stream())
        A.aderdg_batch_step(b, Q, max(3, args.warmup), A.BATCH_GRAPH, stream)   # captures the graph
        torch.cuda.synchronize()
        barrier(world)
        _, _, l0 = A.aderdg_batch_get_tuning(b)
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.15)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        A.aderdg_batch_step(b, Q, args.steps, A.BATCH_GRAPH, stream)
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        _, _, l1 = A.aderdg_batch_get_tuning(b)
        ms = max_over_ranks(ms, world)
        value = whole_job_rate(dofs * args.steps, world, ms / 1e3)

        # the persistent fused sweep timed on its own (mode 1: same kernel and grid, no graph)
        ksteps = max(5, min(40, args.steps // 5))
        Qk = Q0.clone()
        stream.wait_stream(torch.cuda.current_stream())
        A.aderdg_batch_profile(b, True)
        e0.record(stream)
        A.aderdg_batch_step(b, Qk, ksteps, A.BATCH_PERSISTENT, stream)
        e1.record(stream)
        stream.synchronize()
        ms_p = e0.elapsed_time(e1)
        kms, kn = A.aderdg_batch_profile_read(b)
        A.aderdg_batch_profile(b, False)
        peak, peak_src = peaks()
        alg = sum(fused_bytes_per_cell(w, "fp32", per_cell_material=False) * w.cells for w in ws)
        avg_s = kms / kn / 1e3
        achieved = alg / avg_s / 1e9
        roof = {"bound": "hbm", "kernel": "batch_kernel<fused> (persistent, all scenarios)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"hbm_gbs of {peak_src}", "algorithmic_bytes_per_launch": alg,
                "bytes_per_dof": alg / dofs, "kernel_ms_avg": avg_s * 1e3,
                "kernel_share_of_step": (avg_s * 1e3) / (ms / args.steps), "traffic": None}

        # one launch per scenario and sweep (the unbatched form)
        Qs = Q0.clone()
        stream.wait_stream(torch.cuda.current_stream())
        e0.record(stream)
        A.aderdg_batch_step(b, Qs, ksteps, A.BATCH_PER_SCENARIO, stream)
        e1.record(stream)
        stream.synchronize()
        ms_s = e0.elapsed_time(e1)
        same = bool(torch.equal(Qs, Qk))
        forms = {"persistent+graph": {"value": value, "ms_per_step": ms / args.steps},
                 "persistent": {"value": dofs * ksteps / (ms_p / 1e3), "ms_per_step": ms_p / ksteps},
                 "per_scenario": {"value": dofs * ksteps / (ms_s / 1e3), "ms_per_step": ms_s / ksteps,
                                  "launches_per_step": 3 * len(ws)},
                 "per_scenario_equals_persistent_bitwise": same}
        forms["speedup_vs_per_scenario"] = value / forms["per_scenario"]["value"]

        # end to end: pinned host state in, one step, state out, per step
        hq = Q0.cpu().pin_memory()
        dq = torch.empty_like(Q0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            with torch.cuda.stream(stream):
                dq.copy_(hq, non_blocking=True)
            A.aderdg_batch_step(b, dq, 1, A.BATCH_GRAPH, stream)
            with torch.cuda.stream(stream):
                hq.copy_(dq, non_blocking=True)
            stream.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        qbytes = hq.numel() * 4
    finally:
        A.aderdg_batch_destroy(b)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded scenario draw and Gaussian pulses, generated on the GPU)",
           "config": {"workload": ENSEMBLE_NAME, "scenarios": len(ws), "cells": cells, "dofs": dofs,
                      "mode": "persistent launch per sweep, replayed from a CUDA graph",
                      "tuning": {"blocks_per_sm": bps, "tiles_per_item": tpi},
                      "parallelism": f"replicas{world}",
                      "l2": "no flush: every timed sweep streams Q, D and the hull (>> 129 MB L2)"},
           "gpu_launches": l1 - l0, "launches_per_step": (l1 - l0) / args.steps,
           "roofline": roof, "clocks": clocks, "forms": forms,
           "e2e": {"value": dofs * args.e2e_steps * world / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": qbytes, "d2h_bytes_per_step": qbytes,
                   "call": "H2D of the packed state, aderdg_batch_step(nsteps=1), D2H, per step"}}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"], out["accuracy"] = ensemble_cpu_baseline(A, oracle_budget)
    del Q, Q0, Qk, Qs, dq, hq
    torch.cuda.empty_cache()
    return out


def ensemble_cpu_baseline(A, budget=12.0):
    """The oracle on a sample of the ensemble, and the batch path's error on it."""
    import numpy as np
    import torch
    from oracle import oracle as orc
    sample, cores = ensemble_oracle_sample(budget)
    steps = 2
    t0 = time.perf_counter()
    ref = [orc.run(P, Q0, steps)[0] for (_, P, Q0) in sample]
    sec = time.perf_counter() - t0
    sdofs = sum(ws.dofs for (ws, _, _) in sample)
    base = {"value": sdofs * steps / sec, "unit": UNIT, "cores": cores, "host_cpus": os.cpu_count(),
            "kind": "oracle",
            "sample": f"the first {len(sample)} scenarios of the ensemble on 16x16 cells each, "
                      f"{steps} straightforward FP64 steps (Algorithm 1)", "seconds": sec}
    b = ensemble_batch([ws for (ws, _, _) in sample], A)
    try:
        off = A.aderdg_batch_offsets(b, len(sample))
        buf = np.zeros(off[-1], np.float32)
        for s, (_, _, Q0) in enumerate(sample):
            buf[off[s]:off[s] + Q0.size] = Q0.reshape(-1)
        Q = torch.from_numpy(buf).cuda()
        A.aderdg_batch_step(b, Q, steps, A.BATCH_GRAPH)
        got = Q.double().cpu().numpy()
    finally:
        A.aderdg_batch_destroy(b)
    worst = 0.0
    for s, (ws, _, Q0) in enumerate(sample):
        g = got[off[s]:off[s] + Q0.size].reshape(Q0.shape)
        w1 = np.asarray(orc.gauss_legendre(ws.N)[1])
        W = np.multiply.outer(w1, w1).reshape(-1)
        e = math.sqrt(((g - ref[s]) ** 2 * W).sum() / (ref[s] ** 2 * W).sum())
        worst = max(worst, e)
    return base, {"l2_rel_vs_fp64_oracle_max_over_sample": worst, "on": base["sample"]}


# ---------------------------------------------------------------------------
# CPU baseline and reference arm: the FP64 oracle on host cores

def oracle_sample(w, budget_s):
    """Choose a periodic sub-grid of the workload so that one oracle step takes
    about budget_s seconds on the host cores; returns (sample workload, cores)."""
    from oracle import oracle as orc
    from paper_1801_08682_gb300 import workloads as wl
    cores = orc.set_threads(0)
    side0 = 4 if w.d == 3 else 8
    probe = w.resized((side0,) * w.d, steps=1)
    P = orc.Problem(w.d, w.N, orc.PDE_NAMES[w.pde], probe.grid, probe.dx, cst=w.cst,
                    mat=wl.materials(probe) if w.pde == "elasticity" else None, cfl=w.cfl_value)
    xi, _ = orc.gauss_legendre(w.N)
    Q0 = wl.init_state(probe, wl.node_coords(probe.grid, probe.dx, xi))
    t0 = time.perf_counter()
    orc.run(P, Q0, 1)
    per_cell = (time.perf_counter() - t0) / probe.cells
    cells = max(probe.cells, budget_s / max(per_cell, 1e-9))
    side = max(side0, min(w.grid[0], int(round(cells ** (1.0 / w.d)))))
    return w.resized((side,) * w.d, steps=1), cores


def oracle_problem(ws, w):
    from oracle import oracle as orc
    from paper_1801_08682_gb300 import workloads as wl
    return orc.Problem(ws.d, ws.N, orc.PDE_NAMES[ws.pde], ws.grid, ws.dx, cst=w.cst,
                       mat=(wl.materials(ws).astype("float32").astype("float64")
                            if ws.pde == "elasticity" else None), cfl=w.cfl_value)


def cpu_baseline(w, A, prec, pred=0, budget=15.0):
    """Time the oracle (Algorithm 1, FP64, OpenMP) on a bounded sample and
    compare the GPU path with it on that same sample."""
    import numpy as np
    import torch
    from oracle import oracle as orc
    from paper_1801_08682_gb300 import workloads as wl
    ws, cores = oracle_sample(w, budget)
    P = oracle_problem(ws, w)
    xi, _ = orc.gauss_legendre(w.N)
    Q0 = wl.init_state(ws, wl.node_coords(ws.grid, ws.dx, xi))
    steps = 2
    t0 = time.perf_counter()
    Qo, dto, _, _ = orc.run(P, Q0, steps)
    sec = time.perf_counter() - t0
    rate = ws.dofs * steps / sec
    res = {"value": rate, "unit": UNIT, "cores": cores, "host_cpus": os.cpu_count(), "kind": "oracle",
           "sample": f"{'x'.join(map(str, ws.grid))} cells of the same PDE/N/m and CFL step, "
                     f"{steps} straightforward FP64 steps (Algorithm 1)",
           "seconds": sec}
    # accuracy of the GPU path on the same sample (shifted fused form, same dt)
    pde = A.PDE_IDS[w.pde]
    h = A.aderdg_create(ws.d, ws.N, ws.m, pde, ws.grid[: ws.d], ws.dx,
                        A.params(pde_const=w.cst, precision=prec, cfl=w.cfl_value, predictor=pred))
    try:
        if w.pde == "elasticity":
            A.aderdg_set_material(h, torch.from_numpy(wl.materials(ws).astype(np.float32)).cuda())
        Q = to_state(torch.from_numpy(Q0).cuda(), prec)
        A.aderdg_step(h, Q, steps)
        dtg = np.array(A.aderdg_get_dt_history(h))
        Qg = state_values(Q, prec).cpu().numpy()
    finally:
        A.aderdg_destroy(h)
    if not np.allclose(dtg, dto, rtol=1e-12):
        Qo, _, _, _ = orc.run(P, Q0, steps, dt_seq=dtg)
    w1 = np.asarray(orc.gauss_legendre(w.N)[1])
    W = w1
    for _ in range(w.d - 1):
        W = np.multiply.outer(w1, W).reshape(-1)   # node = i0 + n (i1 + n i2)
    diff = ((Qg - Qo) ** 2 * W[None, None, :]).sum()
    ref = (Qo ** 2 * W[None, None, :]).sum()
    res["accuracy"] = {"l2_rel_vs_fp64_oracle": math.sqrt(diff / ref),
                       "linf_rel_vs_fp64_oracle": float(np.abs(Qg - Qo).max() / np.abs(Qo).max()),
                       "on": res["sample"]}
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_1801_08682_gb300 import workloads as wl
    if args.workload == "ensemble":
        return run_reference_ensemble(args)
    if args.workload == "elasticity3d_adjoint":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no adjoint: its gradients are "
                          "tangent and finite-difference runs, used by the tests on small grids"}), flush=True)
        return None
    w = workload(args.workload)
    budget = max(0.2, min(2.0, 150.0 / max(1, args.steps + args.warmup)))
    ws, cores = oracle_sample(w, budget)
    P = oracle_problem(ws, w)
    xi, _ = orc.gauss_legendre(w.N)
    Q0 = wl.init_state(ws, wl.node_coords(ws.grid, ws.dx, xi))
    Q, _, _, _ = orc.run(P, Q0, args.warmup) if args.warmup else (Q0, None, None, None)
    t0 = time.perf_counter()
    orc.run(P, Q, args.steps)
    sec = time.perf_counter() - t0
    value = ws.dofs * args.steps / sec
    sample = (f"each step: {'x'.join(map(str, ws.grid))} cells of the same PDE/N/m and CFL step, "
              f"straightforward FP64 (Algorithm 1)")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": config_of(w, "oracle (Algorithm 1)", 1),
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                                       "host_cpus": os.cpu_count(), "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_adjoint(args):
    import paper_1801_08682_gb300.aderdg as A
    rank, world, local = init_rank()
    A.load(build_if_missing=True)
    out = adjoint_record(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def adjoint_record(args, rank, world, local):
    import numpy as np
    import torch
    import paper_1801_08682_gb300.aderdg as A
    from paper_1801_08682_gb300 import workloads as wl
    w = wl.elasticity_3d()
    if args.grid:   # a smaller case of the same workload (profiling)
        w = w.resized((args.grid,) * 3)
    mat = torch.from_numpy(wl.materials(w).astype(np.float32)).cuda()
    Q0 = gpu_state(w, A).float()
    pos = torch.from_numpy(wl.receivers(w).astype(np.float32)).cuda()
    rng = np.random.default_rng(5)
    K = args.steps
    obs = torch.from_numpy((0.01 * rng.standard_normal((max(K, args.warmup), pos.shape[0], 3))).astype(np.float32)).cuda()
    h = make_handle(w, A, "fused", "fp32")
    try:
        A.aderdg_set_material(h, mat)
        gQ = torch.zeros_like(Q0)
        gm = None if args.no_material_gradient else torch.zeros_like(mat)
        dt = 0.0   # one fixed step size for the whole run: the CFL step of Q0
        A.aderdg_step_adjoint(h, Q0, args.warmup, dt, pos, obs, gQ, gm, args.checkpoint_every)
        torch.cuda.synchronize()
        barrier(world)
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.15)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        J = A.aderdg_step_adjoint(h, Q0, K, dt, pos, obs, gQ, gm, args.checkpoint_every)
        e1.record()
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        finite = bool(torch.isfinite(gQ).all().item() and (gm is None or torch.isfinite(gm).all().item()))
    finally:
        A.aderdg_destroy(h)
    value = whole_job_rate(w.dofs * K, world, ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded pulse, material, receivers, observations)",
           "config": {"workload": f"elasticity3d adjoint d=3 N=4 m=9 grid={'x'.join(map(str, w.grid))}, "
                                  f"{pos.shape[0]} receivers"
                                  + ("" if args.no_material_gradient else f", checkpoint every {args.checkpoint_every}"),
                      "gradients": "dJ/dQ0" + ("" if args.no_material_gradient else " and dJ/d(rho, cp, cs)"),
                      "unit_of_work": "one forward step and its adjoint step of every DoF"
                                      + (" (no forward state kept: the transposed step is state-independent)"
                                         if args.no_material_gradient else " (checkpointed recompute included)"),
                      "dofs": w.dofs, "parallelism": f"replicas{world}",
                      "l2": "no flush: every sweep streams the state (>> 129 MB L2)"},
           "misfit": J, "gradients_finite": finite, "clocks": clocks}
    peak, peak_src = peaks()
    bpc = adjoint_bytes_per_cell(w, args.checkpoint_every, not args.no_material_gradient)
    achieved = bpc * w.cells / (ms / K / 1e3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "whole adjoint step (forward and recomputed fused sweeps, "
                       "state copies, STP sweep, adj_faces_lin_kernel, adj_lin_kernel)",
                       "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                       "peak_source": f"hbm_gbs of {peak_src}", "algorithmic_bytes_per_step": bpc * w.cells,
                       "bytes_per_dof": bpc / (w.m * (w.N + 1) ** w.d), "traffic": None,
                       "note": "the step's own time (CUDA events), not one kernel's"}
    del gQ, gm, Q0, mat
    torch.cuda.empty_cache()
    return out


def run_reference_ensemble(args):
    from oracle import oracle as orc
    budget = max(0.2, min(2.0, 150.0 / max(1, args.steps + args.warmup)))
    sample, cores = ensemble_oracle_sample(budget)
    Qs = [Q0 for (_, _, Q0) in sample]
    if args.warmup:
        Qs = [orc.run(P, Q, args.warmup)[0] for (_, P, _), Q in zip(sample, Qs)]
    t0 = time.perf_counter()
    for (_, P, _), Q in zip(sample, Qs):
        orc.run(P, Q, args.steps)
    sec = time.perf_counter() - t0
    value = sum(ws.dofs for (ws, _, _) in sample) * args.steps / sec
    desc = (f"each step: the first {len(sample)} scenarios of the ensemble on 16x16 cells each, "
            f"straightforward FP64 (Algorithm 1)")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": ENSEMBLE_NAME, "form": "oracle (Algorithm 1)"},
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                                       "host_cpus": os.cpu_count(), "kind": "oracle", "sample": desc},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "elasticity3d_adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
