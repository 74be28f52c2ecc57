"""Measurement models of bench.py against numbers the paper prints."""
import os

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hull_footprint.txt")


def printed_footprints():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                p, r2, r3 = line.split()
                rows.append((int(p), float(r2), float(r3)))
    return rows


def test_hull_footprint_matches_printed_table():
    """Corollary "hull": the ratio reproduces every printed two-decimal value."""
    rows = printed_footprints()
    assert [p for p, _, _ in rows] == list(range(2, 10))
    for p, r2, r3 in rows:
        assert abs(bench.hull_footprint_ratio(2, p) - r2) <= 0.005
        assert abs(bench.hull_footprint_ratio(3, p) - r3) <= 0.005


def test_hull_footprint_bound():
    """The corollary's bound 0.875, reached at d = 2, p = 0."""
    vals = [bench.hull_footprint_ratio(d, p) for d in (2, 3) for p in range(0, 12)]
    assert max(vals) <= 0.875 + 1e-15
    assert abs(bench.hull_footprint_ratio(2, 0) - 0.875) < 1e-15


def test_rerun_bound_balances_the_two_runtimes():
    """Rerun corollary (Sec. 5): at C_rerun equal to the bound, the fused run
    ((C_rerun - 1) T_STP + T_fused) N_fused takes exactly as long as the three
    sweeps T_3steps N_3steps, with N_fused = N_3steps / r; below it, less."""
    for t3, tf, tstp, r in ((32.7, 28.2, 20.2, 1.0), (5.5, 1.65, 1.7, 0.99), (3.0, 2.0, 1.5, 0.9)):
        n3 = 1000.0
        nf = n3 / r
        c = bench.c_rerun_bound(t3, tf, tstp, r)
        fused = ((c - 1.0) * tstp + tf) * nf
        assert abs(fused - t3 * n3) <= 1e-9 * t3 * n3
        assert ((c - 0.01 - 1.0) * tstp + tf) * nf < t3 * n3
