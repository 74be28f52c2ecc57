"""Host logic of bench.py: the algorithmic byte model and the lookup of the
DRAM traffic that a committed ncu summary measured."""
import os

import pytest

import bench
from paper_1801_08682_gb300 import workloads as wl


def dof_per_cell(w):
    return w.m * (w.N + 1) ** w.d


@pytest.mark.parametrize("w,prec,bpd", [
    (wl.acoustics_3d(), "fp32", 28.0),        # Q, D read and written, q-only face hull
    (wl.acoustics_3d(), "fp32_pair", 36.0),   # plus the low-word plane read and written
    (wl.acoustics_3d(), "fp32_acc64", 36.0),  # FP64 state
    (wl.euler_3d(), "fp32_acc64", 60.0),      # nonlinear: q and F.n on the faces
])
def test_fused_bytes_per_dof(w, prec, bpd):
    assert bench.fused_bytes_per_cell(w, prec) / dof_per_cell(w) == pytest.approx(bpd, rel=1e-12)


def test_elasticity_bytes_count_the_materials():
    """Per-cell material: the cell's own and its 2d neighbours' (rho, cp, cs)."""
    w = wl.elasticity_3d()
    with_mat = bench.fused_bytes_per_cell(w, "fp32")
    assert with_mat == 34284
    assert with_mat / dof_per_cell(w) == pytest.approx(30.47, abs=0.01)


def write_profile(root, name, lines):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", f"fused_sweep_{name}.md"), "w") as f:
        f.write("# summary\n\n" + "\n".join(lines) + "\n")


def test_profiled_traffic_lookup(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    w = wl.acoustics_3d()
    h = bench.kernel_source_hash()
    write_profile(str(tmp_path), w.name, [f"bench-key: source_hash = {h}",
                                          "bench-key: dram_bytes_per_launch_full.fp32 = 123456"])
    assert bench.profiled_traffic(w, "fused", "fp32") == 123456.0
    assert bench.profiled_traffic(w, "fused", "fp32_pair") is None   # no capture of that precision
    assert bench.profiled_traffic(w, "hull3", "fp32") is None        # another form's kernel
    write_profile(str(tmp_path), w.name, ["bench-key: source_hash = 000000000000",
                                          "bench-key: dram_bytes_per_launch_full.fp32 = 123456"])
    assert bench.profiled_traffic(w, "fused", "fp32") is None        # taken on other sources
    assert bench.profiled_traffic(wl.euler_3d(), "fused", "fp32_acc64") is None   # no summary


def committed_keys(name):
    path = os.path.join(bench.ROOT, "profiles", f"fused_sweep_{name}.md")
    keys = {}
    with open(path) as f:
        for line in f:
            if line.startswith("bench-key:"):
                k, _, v = line.partition(":")[2].strip().partition("=")
                keys[k.strip()] = v.strip()
    return keys


@pytest.mark.parametrize("w", [wl.acoustics_3d(), wl.elasticity_3d(), wl.euler_3d()])
def test_committed_traffic_against_the_byte_model(w):
    """Each committed full-size traffic figure is the DRAM bytes ncu counted,
    scaled by cells; it must sit below the algorithmic bytes (neighbour face
    reads hit L2) but not far below (that would mean a wrong capture)."""
    keys = committed_keys(w.name)
    full = {k.split(".", 1)[1]: float(v) for k, v in keys.items() if k.startswith("dram_bytes_per_launch_full.")}
    assert full, "no full-size traffic key"
    for prec, traffic in full.items():
        alg = bench.fused_bytes_per_cell(w, prec) * w.cells
        assert 0.6 * alg < traffic < 1.05 * alg, (prec, traffic / alg)
