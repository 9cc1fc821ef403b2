"""The seeded workload generators on the CPU: the serving stream's recipe and the benchmark's
byte accounting helpers."""
from __future__ import annotations

import numpy as np

import bench
import synth


def test_serve_stream_recipe():
    w = synth.WORKLOADS["serve_ba200k"]
    a = synth.serve_stream(w)
    assert a == synth.serve_stream(w)  # seeded
    assert len(a) == 2000 and synth.serve_stream(w, 300) == a[:300]
    t = np.array([q["t"] for q in a])
    assert (np.diff(t) > 0).all()
    assert abs(len(a) / t[-1] - w["rate"]) < 0.1 * w["rate"]  # Poisson arrivals at the rate
    fams = {q["pattern"][0] for q in a}
    assert fams == {"path", "cycle", "grid", "ktree"}
    for q in a:
        nF = q["k"]
        assert 4 <= nF <= 10 and q["trials"] == 1
        pat = synth.make_pattern(q["pattern"])
        assert pat[0] == nF
        if q["pattern"][0] == "grid":
            assert nF in synth.GRID_SHAPES
        if q["pattern"][0] == "ktree":
            assert 1 <= q["pattern"][2] <= min(3, nF - 1)
    # patterns repeat, as a served population would
    assert len({q["pattern"] for q in a}) < 100


def test_percentile_and_entry_bytes():
    xs = list(range(1, 101))
    assert bench.pct(xs, 50) == 50 and bench.pct(xs, 99) == 99 and bench.pct([7], 99) == 7
    assert bench.slot_bytes(2, 8) == 4 * 2 + 2 + 8 and bench.slot_bytes(3, 20) == 12 + 4 + 8
