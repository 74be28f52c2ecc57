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
