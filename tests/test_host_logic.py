"""Host logic of the C library, on the CPU: nice decompositions and CSR validation.

The library's nice-decomposition builder and the oracle's follow the same stated construction
(children in increasing id, each child's subtree followed by forgets then introduces in
increasing vertex order, left-deep joins, leaf bags of size one, empty root) but share no code;
here they must agree node for node, and the library's result must satisfy the definitions of
Section 1.2 on its own.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_pins import check_nice

cc = pytest.importorskip("paper_1908_11248_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()


PATTERNS = [
    synth.path_pattern(1), synth.path_pattern(2), synth.path_pattern(7), synth.cycle_pattern(3),
    synth.cycle_pattern(6), synth.star_pattern(6), synth.clique_pattern(5),
    synth.grid_pattern(2, 4), synth.grid_pattern(3, 3), synth.grid_pattern(4, 2),
    synth.pattern_A(), synth.pattern_B(), synth.pattern_C(), synth.pattern_D(),
] + [synth.random_partial_ktree(n, k, s) for n, k, s in
     [(10, 3, 1), (11, 3, 2), (12, 3, 3), (9, 2, 4), (7, 1, 5), (12, 3, 6), (6, 4, 7)]]


@pytest.mark.parametrize("pi", range(len(PATTERNS)))
def test_nice_decomposition_equals_oracle(pi):
    nF, e, td = PATTERNS[pi]
    nodes, width = cc.cc_nice_decomposition(nF, e, td)
    assert nodes == oracle.nice_td(nF, e, td)
    check_nice(nF, e, td, nodes)
    assert width == max(len(nd[4]) for nd in nodes) - 1 <= max(len(b) for b in td[0]) - 1


@pytest.mark.parametrize("pat,tw", [
    (synth.path_pattern(6), 1), (synth.cycle_pattern(7), 2), (synth.clique_pattern(5), 4),
    (synth.grid_pattern(3, 3), 3), (synth.grid_pattern(2, 5), 2), (synth.star_pattern(6), 1),
    (synth.pattern_A(), 1), (synth.pattern_B(), 2), (synth.pattern_C(), 2),
    (synth.pattern_D(), 2), (synth.grid_pattern(4, 4), 4),
    ((3, np.zeros((0, 2), np.int32), None), 0),
])
def test_minimum_width_decomposition(pat, tw):
    """Table 1 treewidths (P_n, C_n, K_n, S_n: 1, 2, n-1, 1; G_{r,c}: min(r, c)); A-D: 1,2,2,2."""
    nF, e, _ = pat
    nodes, width = cc.cc_nice_decomposition(nF, e, None)
    assert width == tw
    bags = [nd[4] for nd in nodes if nd[4]]
    check_nice(nF, e, (bags, None), nodes)


def test_min_fill_above_twenty_vertices():
    nF, e, _ = synth.random_partial_ktree(24, 3, 11)
    nodes, width = cc.cc_nice_decomposition(nF, e, None)
    assert 3 <= width <= 5
    check_nice(nF, e, ([nd[4] for nd in nodes if nd[4]], None), nodes)


def test_invalid_decompositions():
    nF, e, td = synth.cycle_pattern(5)
    for bad in [([[0, 1, 2], [0, 2, 3]], [1, -1]),                 # vertex 4 missing
                ([[0, 1, 2], [2, 3, 4], [0, 4]], [1, 2, -1]),     # edge 0-4 ... 3-4 uncovered
                ([[0, 1, 2], [0, 2, 3], [0, 3, 4]], [-1, -1, 1]),  # two roots
                ([[0, 1, 2], [], [0, 2, 3, 4]], [1, 2, -1]),      # empty bag
                ([[0, 1, 2], [0, 2, 3, 4]], [1, 0])]:             # cycle in the tree
        with pytest.raises(cc.CCError) as ex:
            cc.cc_nice_decomposition(nF, e, bad)
        assert ex.value.code == cc.CC_EINVAL
    with pytest.raises(cc.CCError):
        cc.cc_nice_decomposition(33, [], None)
    with pytest.raises(cc.CCError):
        cc.cc_nice_decomposition(3, [(0, 0)], None)  # loop


def test_check_graph():
    assert cc.cc_check_graph(*synth.barabasi_albert(300, 3, 1)) == 0
    assert cc.cc_check_graph(*synth.erdos_renyi(100, 0.1, 2)) == 0
    assert cc.cc_check_graph(np.array([0], np.int32), np.zeros(0, np.int32)) == 0  # n = 0
    bad = [
        ([0, 1, 1], [1]),              # asymmetric
        ([0, 1], [0]),                 # self loop
        ([0, 2, 3, 4], [2, 1, 0, 0]),  # unsorted row
        ([0, 2, 3, 4], [1, 1, 0, 0]),  # duplicate
        ([0, 1, 2], [5, 0]),           # out of range
        ([1, 1, 2], [1, 0]),           # row_ptr[0] != 0
        ([0, 2, 1], [1, 0]),           # decreasing row_ptr
    ]
    for rp, col in bad:
        assert cc.cc_check_graph(np.array(rp, np.int32), np.array(col, np.int32)) == cc.CC_EINVAL


def test_solve_trials_count():
    """Repetitions for error bound epsilon: ceil(e^{n_F} ln(1/epsilon)) (Section 2.1), checked on
    values worked out by hand; invalid arguments give -1."""
    assert cc.cc_solve_trials(5, 0.1) == 342      # 148.413 * 2.30259 = 341.74
    assert cc.cc_solve_trials(1, 0.5) == 2        # 2.71828 * 0.69315 = 1.884
    assert cc.cc_solve_trials(8, 0.01) == 13728   # 2980.958 * 4.60517 = 13727.8
    assert cc.cc_solve_trials(0, 0.1) == -1
    assert cc.cc_solve_trials(5, 0.0) == -1
    assert cc.cc_solve_trials(5, 1.0) == -1


def test_width_of_phase_study_patterns():
    """The width the Erdos-Renyi study records for a pattern G(10, q) (the minimum-width
    decomposition the library computes when none is given) is its treewidth, by the subset
    recurrence over elimination orderings, across the q axis."""
    from tests import brute
    import synth

    for iq in range(0, 34, 3):
        _, q, _, pat, _ = synth.er_phase_instance(7, iq)
        nodes, w = cc.cc_nice_decomposition(pat[0], pat[1], None)
        assert w == brute.exact_treewidth(pat[0], pat[1]), q
