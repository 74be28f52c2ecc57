"""The C-ABI library loads, exports every entry point of include/aderdg.h, and
rejects bad arguments before any CUDA call (no GPU needed)."""
import ctypes as C

import numpy as np
import pytest

import paper_1801_08682_gb300.aderdg as A
from oracle import oracle as orc


@pytest.fixture(scope="module")
def lib():
    return A.load(build_if_missing=True)


def test_exports_every_declared_symbol(lib):
    names = A.header_functions()
    assert len(names) >= 13
    raw = C.CDLL(A.library_path())
    for name in names:
        assert hasattr(raw, name), name


def test_nodes_agree_with_oracle(lib):
    # two independent constructions: Golub-Welsch (library) and Newton (oracle)
    for N in range(0, 10):
        xi, w = A.aderdg_nodes(N)
        xo, wo = orc.gauss_legendre(N)
        np.testing.assert_allclose(xi, xo, atol=2e-15)
        np.testing.assert_allclose(w, wo, atol=2e-15)


@pytest.mark.parametrize("args,what", [
    ((4, 2, 3, A.ACOUSTICS, (4, 4), (0.25, 0.25)), "d"),
    ((2, 7, 3, A.ACOUSTICS, (4, 4), (0.25, 0.25)), "N"),
    ((2, 2, 4, A.ACOUSTICS, (4, 4), (0.25, 0.25)), "m"),
    ((2, 2, 3, A.ACOUSTICS, (0, 4), (0.25, 0.25)), "grid"),
    ((2, 2, 3, A.ACOUSTICS, (4, 4), (0.0, 0.25)), "dx"),
])
def test_create_rejects_bad_arguments(lib, args, what):
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(*args, A.params(pde_const=(1.0, 1.0)))
    assert e.value.status == A.ADERDG_EINVAL, what


def test_create_rejects_bad_params(lib):
    for p in (A.params(pde_const=(1.0, 1.0), cfl=1.5), A.params(pde_const=(1.0, 1.0), picard_iters=17),
              A.params(pde_const=(0.0, 1.0)), A.params(pde_const=(1.0, 1.0), form=7)):
        with pytest.raises(A.AderdgError) as e:
            A.aderdg_create(2, 2, 3, A.ACOUSTICS, (4, 4), (0.25, 0.25), p)
        assert e.value.status == A.ADERDG_EINVAL
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_create(2, 2, 4, A.EULER, (4, 4), (0.25, 0.25), A.params(pde_const=(1.0,)))
    assert e.value.status == A.ADERDG_EINVAL
    assert "gamma" in A.aderdg_last_error()


def test_null_handle_calls(lib):
    assert lib.aderdg_step(None, None, 1, 0.0, None, None) == A.ADERDG_EINVAL
    assert lib.aderdg_destroy(None) == A.ADERDG_OK
    assert isinstance(A.aderdg_last_error(), str)


@pytest.mark.parametrize("change,status", [
    (dict(N=7), "EINVAL"), (dict(N=1), "EINVAL"), (dict(d=3), "EINVAL"), (dict(m=4), "EINVAL"),
    (dict(pde=A.EULER, m=4), "EINVAL"), (dict(grid=(0, 5)), "EINVAL"), (dict(dx=(0.0, 0.1)), "EINVAL"),
    (dict(pde_const=(0.0, 1.0)), "EINVAL"), (dict(pde_const=(1.0, -1.0)), "EINVAL"), (dict(cfl=1.5), "EINVAL"),
])
def test_batch_create_rejects_bad_scenarios(lib, change, status):
    """Checked for every scenario before any device call (the bad one is last)."""
    good = A.scenario("acoustics", 3, (8, 8), pde_const=(1.0, 1.0))
    spec = dict(pde="acoustics", N=3, pde_const=(1.0, 1.0), cfl=0.0)
    spec.update({k: v for k, v in change.items() if k in spec})
    bad = A.scenario(spec["pde"], spec["N"], (8, 8), pde_const=spec["pde_const"], cfl=spec["cfl"])
    if "grid" in change:
        bad.grid[0], bad.grid[1] = change["grid"]
    if "dx" in change:
        bad.dx[0], bad.dx[1] = change["dx"]
    for k in ("d", "m"):
        if k in change:
            setattr(bad, k, change[k])
    with pytest.raises(A.AderdgError) as e:
        A.aderdg_batch_create([good, good, bad])
    assert e.value.status == getattr(A, "ADERDG_" + status)


def test_batch_and_host_entry_points_reject_null(lib):
    assert lib.aderdg_batch_create(0, None, None) == A.ADERDG_EINVAL
    assert lib.aderdg_batch_step(None, None, 1, 0, None) == A.ADERDG_EINVAL
    assert lib.aderdg_step_host(None, None, 1, 0.0, None, None) == A.ADERDG_EINVAL


def test_handle_entry_points_reject_null_handle(lib):
    """Every entry point that takes a handle returns EINVAL for a NULL one,
    before any device call."""
    calls = [
        lambda: A.aderdg_begin(None, None),
        lambda: A.aderdg_advance(None, None, 1),
        lambda: A.aderdg_end(None, None),
        lambda: A.aderdg_set_material(None, None),
        lambda: A.aderdg_get_stats(None),
        lambda: A.aderdg_footprint(None),
        lambda: A.aderdg_profile(None, True),
        lambda: A.aderdg_profile_read(None, A.KERNEL_FUSED),
    ]
    for call in calls:
        with pytest.raises(A.AderdgError) as e:
            call()
        assert e.value.status == A.ADERDG_EINVAL
    assert lib.aderdg_step_adjoint(None, None, 1, 0.0, None, 1, None, None, None, 0, None, None) == A.ADERDG_EINVAL
    assert lib.aderdg_get_dt_history(None, None, 0, None) == A.ADERDG_EINVAL


# aderdg_step_noalloc checks every argument before any CUDA call, so on a
# machine without a GPU a rejected argument still returns EINVAL (a missed
# check would reach the CUDA runtime and return ECUDA instead).  The state
# pointer is a made-up, 16-byte aligned address that is never dereferenced.
_FAKE_Q = 1 << 20
_NOALLOC_GOOD = dict(d=2, N=2, m=3, pde=A.ACOUSTICS, grid=(4, 4), dx=(0.25, 0.25),
                     prm=dict(pde_const=(1.0, 1.0)), mat=None, Q=_FAKE_Q, nsteps=1, fixed_dt=0.0)


@pytest.mark.parametrize("change", [
    dict(d=4), dict(N=7), dict(N=-1), dict(pde=5), dict(m=4), dict(pde=A.EULER),
    dict(grid=None), dict(dx=None), dict(Q=None), dict(Q=_FAKE_Q + 8), dict(nsteps=-1),
    dict(fixed_dt=-1.0), dict(fixed_dt=float("nan")), dict(fixed_dt=float("inf")),
    dict(grid=(0, 4)), dict(dx=(0.0, 0.25)), dict(dx=(float("inf"), 0.25)),
    dict(prm=dict(pde_const=(1.0, 1.0), cfl=1.5)), dict(prm=dict(pde_const=(1.0, 1.0), cfl=-0.1)),
    dict(prm=dict(pde_const=(1.0, 1.0), picard_iters=17)),
    dict(prm=dict(pde_const=(1.0, 1.0), precision=4)),
    dict(prm=dict(pde_const=(1.0, 1.0), form=1)), dict(prm=dict(pde_const=(1.0, 1.0), form=2)),
    dict(prm=dict(pde_const=(1.0, 1.0), dt_policy=2)),
    dict(prm=dict(pde_const=(1.0, 1.0), predictor=3)),
    dict(mat=_FAKE_Q),                                  # a material for a PDE without one
    dict(prm=None),                                     # all-zero constants: rho = c = 0
    dict(prm=dict(pde_const=(0.0, 1.0))), dict(prm=dict(pde_const=(1.0, 0.0))),
    dict(prm=dict(pde_const=(1.0, -2.0))),
    dict(pde=A.EULER, m=4, prm=dict(pde_const=(1.0,))), dict(pde=A.EULER, m=4, prm=dict(pde_const=(0.5,))),
    dict(pde=A.EULER, m=4, prm=None),
    dict(pde=A.ELASTICITY, m=5, prm=dict(pde_const=(2.5, 0.0, 1.0))),
    dict(pde=A.ELASTICITY, m=5, prm=dict(pde_const=(0.0, 5.0, 2.0))),
    dict(d=3, N=5, m=4, grid=(64, 64, 64), dx=(1 / 64,) * 3),          # scratch does not fit
    dict(d=3, m=4, grid=(1 << 30, 1 << 30, 1 << 30), dx=(1.0,) * 3),    # cell count past 2^64
    dict(d=3, m=4, grid=(1 << 21, 1 << 21, 1 << 22), dx=(1.0,) * 3),    # wraps to 0 in 64 bits
    dict(d=3, m=4, grid=(65537, 65537, 1), dx=(1.0,) * 3),
])
def test_noalloc_rejects_bad_arguments_before_any_cuda_call(lib, change):
    a = dict(_NOALLOC_GOOD)
    a.update(change)
    prm = None if a["prm"] is None else A.params(**a["prm"])
    grid = None if a["grid"] is None else (C.c_int * 3)(*(list(a["grid"]) + [1] * (3 - len(a["grid"]))))
    dx = None if a["dx"] is None else (C.c_double * 3)(*(list(a["dx"]) + [1.0] * (3 - len(a["dx"]))))
    st = lib.aderdg_step_noalloc(a["d"], a["N"], a["m"], a["pde"], grid, dx,
                                 C.byref(prm) if prm is not None else None, a["mat"], a["Q"],
                                 a["nsteps"], a["fixed_dt"], None, None)
    assert st == A.ADERDG_EINVAL, change


def test_noalloc_zero_steps_is_a_no_op_after_the_checks(lib):
    g = (C.c_int * 3)(4, 4, 1)
    h = (C.c_double * 3)(0.25, 0.25, 1.0)
    prm = A.params(pde_const=(1.0, 1.0))
    assert lib.aderdg_step_noalloc(2, 2, 3, A.ACOUSTICS, g, h, C.byref(prm), None, _FAKE_Q, 0, 0.0,
                                   None, None) == A.ADERDG_OK
    bad = A.params(pde_const=(0.0, 1.0))
    assert lib.aderdg_step_noalloc(2, 2, 3, A.ACOUSTICS, g, h, C.byref(bad), None, _FAKE_Q, 0, 0.0,
                                   None, None) == A.ADERDG_EINVAL


def test_fp32_peak_rejects_bad_arguments_before_any_cuda_call(lib):
    v = C.c_double(0)
    assert lib.aderdg_fp32_fma_peak(5, None, None) == A.ADERDG_EINVAL
    assert lib.aderdg_fp32_fma_peak(0, C.byref(v), None) == A.ADERDG_EINVAL
    assert lib.aderdg_fp32_fma_peak(1001, C.byref(v), None) == A.ADERDG_EINVAL
