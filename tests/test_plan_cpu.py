"""Host logic of the grouped schedule, no GPU needed: the gate groups of
shared-prefix mode (qn_group_plan) and the tile maps of the mixer-block
sweeps (qn_mix_tile_map).

The groups must cover the circuit's gates exactly once and in circuit order:
consecutive phase gates of one layer on at most 10 qubits and at most 12 gates,
each group ending only where the next gate would break a limit or the layer
ends; for n >= 12, consecutive mixer rotations in blocks: qubits 0-7 (the sweep
of the layer's last phase group rotates qubits 0-3 and forms the block's joint),
then four qubits at a time.  A
tile map must be a bijection of the float4-index bits that puts the block's
qubits on its A bits and the next block's qubits on its B bits, which is what
the sweep's register pairs rely on."""
import numpy as np
import pytest

from paper_2210_15874_gb300 import workloads as W

MAX_QUBITS, MAX_GATES, BLOCK, WIDE = 10, 12, 4, 8


@pytest.fixture(scope="module")
def qn():
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


GRAPHS = {
    "n20_3reg_bench": lambda: (20, W.damping_n20().edges, 3),
    "n5_ring": lambda: (5, W.ring_graph(5), 2),
    "n12_3reg": lambda: (12, W.regular_graph(12, 3, 7), 2),
    "n13_4reg": lambda: (13, W.regular_graph(13, 4, 8), 1),
    "n16_5reg": lambda: (16, W.regular_graph(16, 5, 9), 2),
    "n26_3reg": lambda: (26, W.regular_graph(26, 3, 10), 4),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_group_plan_covers_the_circuit(qn, name):
    n, edges, p = GRAPHS[name]()
    E = len(edges)
    plan = qn.group_plan(n, edges, p)
    phase_gate = {}  # gate index -> edge
    for l in range(p):
        for e in range(E):
            phase_gate[n + l * (E + n) + e] = tuple(int(x) for x in edges[e])
    covered = []
    for g in plan:
        gates = list(range(g["first_gate"], g["first_gate"] + g["gates"]))
        covered += gates
        layer = (g["first_gate"] - n) // (E + n)
        assert all((x - n) // (E + n) == layer for x in gates)  # inside one layer
        if g["kind"] == 0:
            assert all(x in phase_gate for x in gates)
            qs = sorted({q for x in gates for q in phase_gate[x]})
            assert qs == g["qubits"]
            assert len(qs) <= MAX_QUBITS and g["gates"] <= MAX_GATES
            # greedy: the next gate of the layer would break a limit
            nxt = g["first_gate"] + g["gates"]
            if nxt in phase_gate:
                grown = set(qs) | set(phase_gate[nxt])
                assert len(grown) > MAX_QUBITS or g["gates"] == MAX_GATES
        else:
            assert n >= 12
            rot = [x - (n + layer * (E + n) + E) for x in gates]  # qubit of each rotation
            assert rot == list(range(rot[0], rot[0] + len(rot))) and rot[0] % BLOCK == 0
            if rot[0] == 0:
                assert len(rot) == WIDE and g["qubits"] == rot
                assert plan[plan.index(g) - 1]["kind"] == 0  # a phase group's sweep starts it
            elif rot[0] == WIDE and n >= 20 and n % BLOCK == 0:
                # qubits 8-15 as one block too: the last phase group's sweep rotates 0-7 whole
                assert len(rot) == WIDE and g["qubits"] == rot
            else:
                assert len(rot) == min(BLOCK, n - rot[0]) and g["qubits"] == rot
    expected = sorted(phase_gate)
    if n >= 12:  # the mixer rotations are grouped too
        expected = sorted(expected + [n + l * (E + n) + E + q for l in range(p) for q in range(n)])
    assert covered == expected  # every grouped gate once, in circuit order


@pytest.mark.parametrize("n", [12, 13, 14, 16, 19, 20, 23, 26, 30])
def test_mix_tile_maps_are_bijections(qn, n):
    for q_lo in range(0, n, BLOCK):
        m = min(BLOCK, n - q_lo)
        m_next = min(BLOCK, n - q_lo - m)
        t = qn.mix_tile_map(n, q_lo, m, m_next)
        bits = t["lane"] + t["a"] + t["b"] + t["tile"]
        assert sorted(bits) == list(range(n - 1))  # every float4-index bit exactly once
        own = [q - 1 for q in range(q_lo, q_lo + m) if q > 0]  # qubit q is f bit q - 1; qubit 0 is in the float4
        assert t["a"][:len(own)] == own
        assert t["b"][:m_next] == [q - 1 for q in range(q_lo + m, q_lo + m + m_next)]
        if q_lo == 0 and m == BLOCK and m_next == BLOCK:
            # the contiguous tile the first block's address-order copies rely on
            assert t["a"] == [0, 1, 2, 7] and t["b"] == [3, 4, 5, 6] and t["lane"] == [8, 9, 10]
        if q_lo >= 8:
            assert t["lane"] == [0, 1, 2]  # neighbouring float4 on neighbouring lanes


def test_plan_and_map_reject_bad_arguments(qn):
    with pytest.raises(qn.QnError, match="QN_EINVAL"):
        qn.group_plan(4, np.array([[0, 4]], dtype=np.int32), 1)
    with pytest.raises(qn.QnError, match="QN_EINVAL"):
        qn.group_plan(4, W.ring_graph(4), -1)
    with pytest.raises(qn.QnError, match="QN_EINVAL"):
        qn.mix_tile_map(11, 0, 4, 4)
    with pytest.raises(qn.QnError, match="QN_EINVAL"):
        qn.mix_tile_map(20, 16, 4, 4)
    assert qn.group_plan(6, W.ring_graph(6), 0) == []


def test_fused_window_schedules(qn):
    """The library's window schedules of the fused layers (qn_fused_windows): every window
    list covers the qubits once in order; the forward one equals the rule the GPU test
    mirrors and the sweep counts the bench's byte figures use; the adjoint's takes qubits
    0-9 and then at most six per window from 12 qubits on (its last window also undoes the
    cost diagonal), qubits 0-3 and then two or three per window below."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from test_gpu_fused import fused_windows

    for n in range(2, 31):
        fw, aw = qn.fused_windows(n), qn.fused_windows(n, reverse=True)
        for w in (fw, aw):
            assert [q for lo, m in w for q in range(lo, lo + m)] == list(range(n)), (n, w)
        assert fw == fused_windows(n), n
        assert len(fw) == bench.fused_window_count(n), n
        if n >= 12:
            assert aw[0] == (0, 10) and all(1 <= m <= 6 for _, m in aw[1:]), (n, aw)
            assert len(aw) == bench.adjoint_window_count(n) == 1 + -(-(n - 10) // 6), n
        else:
            assert aw[0] == (0, min(4, n)) and all(2 <= m <= 3 for _, m in aw[1:]) or n <= 5, (n, aw)
            assert len(aw) + 1 == bench.adjoint_window_count(n), n  # plus the diagonal's sweep
    assert qn.fused_windows(16) == [(0, 12), (12, 4)]
    assert qn.fused_windows(26) == [(0, 12), (12, 7), (19, 7)]
    assert qn.fused_windows(20) == [(0, 8), (8, 6), (14, 6)]
    assert qn.fused_windows(16, reverse=True) == [(0, 10), (10, 6)]
    assert qn.fused_windows(20, reverse=True) == [(0, 10), (10, 5), (15, 5)]
    for bad in (1, 31):
        with pytest.raises(qn.QnError, match="QN_EINVAL"):
            qn.fused_windows(bad)
