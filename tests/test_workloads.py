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


def test_traffic_summary_from_an_ncu_listing(tmp_path):
    """The DRAM-traffic summary of a capture: DRAM bytes of each kernel summed by node rule
    (templated, demangled names included), each rule's ratio to the step's algorithmic bytes,
    read back by the bench only while the library's sources are unchanged."""
    import json

    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"')
    rows = [head]

    def add(i, name, rd, wr, ns):
        for m, u, v in (("dram__bytes_read.sum", "Mbyte", rd), ("dram__bytes_write.sum",
                                                                 "Kbyte", wr),
                        ("gpu__time_duration.sum", "nsecond", ns)):
            rows.append(f'"{i}","1","python","h","{name}","1","7","(256, 1, 1)","(10, 1, 1)",'
                        f'"0","10.3","Command line profiler metrics","{m}","{u}","{v}"')

    add(0, "void cc::(anonymous namespace)::color_kernel(int, int)", "1.5", "3,000", "1000")
    add(1, "void cc::(anonymous namespace)::intro_warp_kernel<unsigned long, 1>(cc::X)", "100",
        "50,000", "500000")
    add(2, "void cc::(anonymous namespace)::sweep_pass_kernel<unsigned long, unsigned long, "
        "256, 6, true, false>(cc::SortSpec)", "200", "200,000", "250000")
    add(3, "reduce_write_kernel<unsigned long, 256, false>", "40", "10,000", "50000")
    add(4, "enum_step_kernel", "1", "1", "100")
    csv = tmp_path / "dram.csv"
    csv.write_text("==PROF== Connected\n" + "\n".join(rows) + "\n")
    alg = {"workload": "toy", "trials": 2, "sources": bench.source_hash(), "opts": {"fuse": 0},
           "entries": 1, "groups": {"colour": {"launches": 1, "bytes": 4.5e6},
                                    "introduce": {"launches": 1, "bytes": 75e6},
                                    "forget": {"launches": 2, "bytes": 100e6}}}
    aj = tmp_path / "alg.json"
    aj.write_text(json.dumps(alg))
    path = bench.traffic_summary(str(csv), str(aj), "ncu ... bench.py --capture", str(tmp_path))
    r = bench.traffic_ratios("toy", str(tmp_path))
    assert abs(r["colour"] - 1.0) < 1e-9
    assert abs(r["introduce"] - 2.0) < 1e-9  # 150 MB against 75 MB
    assert abs(r["forget"] - 4.5) < 1e-9  # (400 + 50) MB against 100 MB
    assert "other" not in r
    text = open(path).read()
    assert "sweep_pass_kernel" in text and "bench.py --capture" in text
    # another build's capture is not used
    alg["sources"] = "0" * 16
    aj.write_text(json.dumps(alg))
    bench.traffic_summary(str(csv), str(aj), "x", str(tmp_path))
    assert bench.traffic_ratios("toy", str(tmp_path)) == {}
    # the launch list summary of the same listing: shares per kernel and per node rule
    lp = bench.launch_summary(str(csv), "toy", "ncu ... bench.py", str(tmp_path))
    lines = {ln.split()[0]: ln.split() for ln in open(lp) if not ln.startswith("#")}
    assert lines["forget"][1] == "2" and abs(float(lines["forget"][3]) - 0.3 / 0.8001) < 1e-3
    assert lines["intro_warp_kernel"][1] == "1"


def test_chained_introduce_byte_accounting():
    """A chained launch (two introduces in one pass, timed at the upper node) reads the lower
    introduce's child and writes the upper introduce's entries: the lower table is neither
    written nor read back, so its entries add no bytes."""
    # nodes: (type, child0, child1, vertex, bag): leaf 0, introduce 1 (lower), introduce 2
    nodes = [(0, -1, -1, 0, [0]), (1, 0, -1, 1, [0, 1]), (1, 1, -1, 2, [0, 1, 2])]
    sizes = [10, 1000, 7]
    k = 3
    got = bench.algorithmic_bytes("intro_chain", 2, nodes, sizes, 40, 100, 1, k)
    assert got == 10 * bench.slot_bytes(1, k) + 40 * 5 + 7 * bench.slot_bytes(3, k)
    assert bench.GROUPS["intro_chain"] == "introduce"
    assert bench.kernel_group("void cc::(anonymous namespace)::nb_colour_hist_kernel(x)",
                              False) == "introduce"  # timed with the chained launch
    assert bench.kernel_group("intro_group_warp_kernel<unsigned long, 1, true>", True) == \
        "introduce+forget"


def test_forest_hom_counts_against_brute_force():
    """The host-side counts behind the power-law memory bound: injective homomorphisms of the
    forests on at most four vertices into the subgraph induced by the vertices of degree >= t,
    by brute force over all injective maps; the 4-vertex path's count is a lower bound."""
    import itertools

    g = synth.barabasi_albert(22, 3, 4)
    rp, col = np.asarray(g[0]), np.asarray(g[1])
    n = len(rp) - 1
    deg = np.diff(rp)
    E = {(int(a), int(b)) for a in range(n) for b in col[rp[a]:rp[a + 1]]}
    shapes = {  # (vertices, edges, sorted degrees) -> an edge list on 0..b-1
        (1, 0, (0,)): [], (2, 0, (0, 0)): [], (2, 1, (1, 1)): [(0, 1)],
        (3, 1, (0, 1, 1)): [(0, 1)], (3, 2, (1, 1, 2)): [(0, 1), (1, 2)],
        (4, 2, (0, 1, 1, 2)): [(0, 1), (1, 2)], (4, 2, (1, 1, 1, 1)): [(0, 1), (2, 3)],
        (4, 3, (1, 1, 1, 3)): [(0, 1), (0, 2), (0, 3)],
        (4, 3, (1, 1, 2, 2)): [(0, 1), (1, 2), (2, 3)],
    }
    for t in (1, 4, 6):
        got = bench.tree_hom_counts(rp, col, t)
        vs = [v for v in range(n) if deg[v] >= t]
        for shape, es in shapes.items():
            brute = sum(1 for phi in itertools.permutations(vs, shape[0])
                        if all((phi[a], phi[b]) in E for a, b in es))
            if shape == (4, 3, (1, 1, 2, 2)):
                assert got[shape] <= brute and got[shape] >= 0.5 * brute, (t, shape)
            else:
                assert got[shape] == brute, (t, shape, got[shape], brute)
