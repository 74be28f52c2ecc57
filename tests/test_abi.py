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
