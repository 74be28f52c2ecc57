"""GPU parity of the two terms of Eq. 1 beyond the conservative flux: material
jumps in non-conservative form (path-conservative Rusanov, heterogeneous
elasticity) and point sources, through the C ABI, against the FP64 oracle.

Tolerances as in the other parity tests: FP64 kernels max |diff| <= 1e-11
max|Q|, FP32 kernels relative L2 <= 1e-5.  The oracle takes the jump terms in
strong form with fluctuations and the sources in the Picard right-hand side;
the line-owner kernel takes the equivalent own-side flux and the Horner form
with source terms, so agreement checks the two derivations against each
other.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1801_08682_gb300 import workloads as wl
from tests.gpu_util import A, rel_l2_plain, run_gpu
from tests.helpers import coords, weights_nd
from tests.test_gpu_parity import random_smooth, tight

pytestmark = pytest.mark.gpu

ADV, ACO, ELA = orc.ADVECTION, orc.ACOUSTICS, orc.ELASTICITY


def _material(C, seed):
    rng = np.random.default_rng(seed)
    mat = np.stack([rng.uniform(2, 3, C), rng.uniform(4, 6, C), np.zeros(C)], 1)
    mat[:, 2] = mat[:, 1] / math.sqrt(3) * rng.uniform(0.9, 1.0, C)
    return mat.astype(np.float32).astype(np.float64)     # the library keeps float materials


ELA_CST = (2.5, 5.0, 5.0 / math.sqrt(3))


@pytest.mark.parametrize("d,N,prec,grid", [(2, 3, "fp32", (9, 7)), (2, 2, "fp64", (7, 5)),
                                            (3, 2, "fp64", (5, 4, 3)), (3, 4, "fp32", (6, 5, 4)),
                                            (2, 3, "fp64", (8, 6))])
def test_ncp_material_jumps_match_oracle(d, N, prec, grid):
    C = int(np.prod(grid))
    dx = tuple(1.0 / g for g in grid)
    mat = _material(C, 10 + d + N)
    P = orc.Problem(d, N, ELA, grid, dx, cst=ELA_CST, mat=mat, cfl=0.5, ncp=True)
    Q0 = random_smooth(P, 11)
    Qg, dtg, _, _ = run_gpu(P, Q0, 5, precision=prec, mat=mat)
    Qo, dto, _, _ = orc.run(P, Q0, 5, dt_seq=dtg)
    if prec == "fp64":
        tight(Qg, Qo)
    else:
        assert rel_l2_plain(Qg, Qo) <= 1e-5
    # and the jump terms matter here: the per-cell flux gives another state
    Pc = orc.Problem(d, N, ELA, grid, dx, cst=ELA_CST, mat=mat, cfl=0.5)
    Qc, _, _, _ = orc.run(Pc, Q0, 5, dt_seq=dtg)
    assert rel_l2_plain(Qc, Qo) > 1e-3


def test_ncp_reflection_and_transmission_on_the_gpu():
    """The impedance-jump problem of the oracle pins on the GPU (FP64): the
    reflected and transmitted pulses of R = (Z1 - Z2)/(Z1 + Z2),
    T = 2 Z1/(Z1 + Z2)."""
    from tests.test_oracle_pins_ncp_sources import _interface_run
    G, N, T = 160, 3, 0.5
    L = 2.0
    dx = (L / G, 0.05)
    xc = (np.arange(G) + 0.5) * dx[0]
    two = (xc >= 0.6) & (xc < 1.9)
    rho = np.where(two, 2.0, 1.0)
    cp = np.where(two, 2.0, 1.0)
    mat = np.stack([rho, cp, cp / 2], 1)
    P = orc.Problem(2, N, ELA, (G, 1), dx, cst=(1.0, 1.0, 0.5), mat=mat, cfl=0.6, ncp=True)
    x = coords(P)[..., 0]
    sw = 0.04

    def f(z):
        return np.exp(-((z - 0.3) ** 2) / (2 * sw * sw))

    Q0 = np.zeros((P.C, P.m, P.NS))
    Q0[:, 3] = f(x)
    Q0[:, 0] = -f(x)
    Q0[:, 1] = -0.5 * f(x)
    K = int(math.ceil(T / (0.6 * dx[0] / (2 * (2 * N + 1) * 2.0))))
    Qg, _, _, _ = run_gpu(P, Q0, K, precision="fp64", fixed_dt=T / K, mat=mat)
    Z1, Z2, c1, c2, x0 = 1.0, 4.0, 1.0, 2.0, 0.6
    R, Tr = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)
    exact = np.where(x < x0, f(x - c1 * T) + R * f(2 * x0 - x - c1 * T),
                     Tr * f(x0 + (c1 / c2) * (x - x0) - c1 * T))
    W = weights_nd(N, 2)
    err = math.sqrt(((Qg[:, 3] - exact) ** 2 * W).sum() / (exact ** 2 * W).sum())
    assert err < 1e-4, err
    assert abs(err - _interface_run(True, G)) < 1e-7


def _sources(d, m, seed, n=2, t0=0.0):
    rng = np.random.default_rng(seed)
    out = [orc.source(rng.uniform(0, 1, d), rng.standard_normal(m), kind=1, t0=t0 + 0.01, f0=25.0)]
    for _ in range(n - 1):
        out.append(orc.source(rng.uniform(0, 1, d), rng.standard_normal(m), kind=0, t0=t0,
                              coef=rng.standard_normal(4)))
    return out


@pytest.mark.parametrize("case", ["acoustics2d_n3_fp32", "acoustics2d_n3_fp64", "acoustics3d_n3_fp32",
                                  "elasticity3d_n2_fp64", "elasticity2d_n3_fp32", "elasticity3d_n4_fp32"])
def test_point_sources_match_oracle(case):
    pde_name, dn, prec = case.split("_")
    d, N = int(pde_name[-2]), int(dn[1:])
    pde = ACO if pde_name.startswith("acoustics") else ELA
    grid = {2: (9, 7), 3: (5, 4, 6)}[d]
    dx = tuple(1.0 / g for g in grid)
    m = orc.num_vars(pde, d)
    mat = None
    if pde == ELA:
        mat = _material(int(np.prod(grid)), 3)
        cst = ELA_CST
    else:
        cst = (1.2, 0.8)
    srcs = _sources(d, m, 4, n=3)
    srcs.append(orc.source(srcs[0].pos[:d], [1.0] * m, kind=0, coef=(0.5, -1.0)))   # two in one cell
    P = orc.Problem(d, N, pde, grid, dx, cst=cst, mat=mat, cfl=0.5, sources=srcs)
    Q0 = random_smooth(P, 5, amp=0.1)
    Qg, dtg, _, _ = run_gpu(P, Q0, 6, precision=prec, mat=mat)
    Qo, _, _, _ = orc.run(P, Q0, 6, dt_seq=dtg)
    if prec == "fp64":
        tight(Qg, Qo)
    else:
        assert rel_l2_plain(Qg, Qo) <= 1e-5
    Pn = orc.Problem(d, N, pde, grid, dx, cst=cst, mat=mat, cfl=0.5)
    Qn, _, _, _ = orc.run(Pn, Q0, 6, dt_seq=dtg)
    assert rel_l2_plain(Qn, Qo) > 1e-3          # the sources do act


def test_point_source_with_zero_flux_integrates_exactly():
    """Advection with a = 0 (fixed dt): the state changes by the projected delta
    times the exact integral of a degree-7 polynomial (N = 3: GL in time is
    exact to degree 2N + 1)."""
    N, grid, dx = 3, (3, 4), (0.5, 0.25)
    rng = np.random.default_rng(1)
    coef = rng.standard_normal(8)
    src = orc.source((0.83, 0.61), (1.7,), kind=0, t0=0.05, coef=coef)
    P = orc.Problem(2, N, ADV, grid, dx, cst=(0.0, 0.0), sources=[src])
    Q0 = random_smooth(P, 2)
    Qg, _, t1, _ = run_gpu(P, Q0, 4, precision="fp64", fixed_dt=0.07)
    anti = np.polynomial.polynomial.polyint(coef)
    S = np.polynomial.polynomial.polyval(t1 - 0.05, anti) - np.polynomial.polynomial.polyval(-0.05, anti)
    cell, pw = orc.source_weights(P, 0)
    want = Q0.copy()
    want[cell, 0] += 1.7 * pw * S
    tight(Qg, want, rtol=1e-12)


def test_point_sources_with_a_rerun():
    """Sources in the rerun STP sweep (Technique 5): an injected cut of dt_adm
    forces one rerun; the state equals the oracle's Algorithm-2 run."""
    P = orc.Problem(2, 3, ACO, (9, 7), (1 / 9, 1 / 7), cst=(1.2, 0.8), cfl=0.5, sources=_sources(2, 3, 7))
    Q0 = random_smooth(P, 8, amp=0.1)
    # dt_new = C dt_adm with C = 0.5: a cut below one half of dt_adm forces the rerun
    Qg, dtg, _, st = run_gpu(P, Q0, 6, precision="fp64", inject_step=3, inject_factor=0.3)
    Qo, dto, nre, _ = orc.run_shifted(P, Q0, 6, inject_step=3, inject_factor=0.3)
    assert st.reruns == 1 and nre == 1
    np.testing.assert_allclose(dtg, dto, rtol=1e-13)
    tight(Qg, Qo)


def test_point_sources_host_entry_point_matches_device():
    import torch
    w = wl.Workload("s", "elasticity", 3, 4, (6, 5, 4), 3, cst=ELA_CST, seed=4)
    xi, _ = A.aderdg_nodes(4)
    Q0 = 0.1 * wl.init_state(w, wl.node_coords(w.grid, w.dx, np.array(xi)))
    srcs = [A.source((0.3, 0.5, 0.2), [0.0] * 8 + [1.0], kind=1, t0=0.01, f0=30.0)]
    out = []
    for host in (False, True):
        h = A.aderdg_create(3, 4, 9, A.ELASTICITY, w.grid, w.dx, A.params(pde_const=ELA_CST))
        try:
            A.aderdg_set_sources(h, srcs)
            if host:
                q = torch.from_numpy(Q0.astype(np.float32)).pin_memory()
                t = A.aderdg_step_host(h, q, 3)
                out.append((q.clone(), t))
            else:
                q = torch.from_numpy(Q0.astype(np.float32)).cuda()
                t = A.aderdg_step(h, q, 3)
                out.append((q.cpu(), t))
        finally:
            A.aderdg_destroy(h)
    assert out[0][1] == out[1][1]
    assert torch.equal(out[0][0], out[1][0])


def test_sources_and_jumps_rejected_where_not_built():
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(2, 2, 5, A.ELASTICITY, (4, 4), (0.25, 0.25),
                        A.params(pde_const=ELA_CST, form="hull3", material_jumps=A.JUMPS_NONCONSERVATIVE))
    assert e.value.status == A.ADERDG_EINVAL
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(2, 2, 4, A.EULER, (4, 4), (0.25, 0.25),
                        A.params(pde_const=(1.4,), material_jumps=A.JUMPS_NONCONSERVATIVE))
    assert e.value.status == A.ADERDG_EINVAL
    h = A.aderdg_create(2, 2, 4, A.EULER, (4, 4), (0.25, 0.25), A.params(pde_const=(1.4,)))
    try:
        with pytest.raises(A.AderdgError) as e:
            A.aderdg_set_sources(h, [A.source((0.1, 0.1), (1.0,))])
        assert e.value.status == A.ADERDG_EUNSUPPORTED
    finally:
        A.aderdg_destroy(h)
    h = A.aderdg_create(2, 3, 3, A.ACOUSTICS, (4, 4), (0.25, 0.25), A.params(pde_const=(1.0, 1.0)))
    try:
        with pytest.raises(A.AderdgError) as e:
            A.aderdg_set_sources(h, [A.source((0.1, 0.1), (1.0,), kind=2)])
        assert e.value.status == A.ADERDG_EINVAL
        A.aderdg_set_sources(h, [A.source((0.1, 0.1), (1.0,))])
        with pytest.raises(A.AderdgError) as e:   # the adjoint covers the source-free step
            A.aderdg_step_adjoint(h, None, 1, 0.0, None, None, None)
        assert e.value.status in (A.ADERDG_EINVAL, A.ADERDG_EUNSUPPORTED)
    finally:
        A.aderdg_destroy(h)
