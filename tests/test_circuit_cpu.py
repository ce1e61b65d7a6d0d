"""Host-side circuit layer (no GPU): the QuDiet QASM front end (Sec. 4), the
Toffoli decomposition through an elevated carrier (Sec. 3.4), the
logarithmic-depth multi-controlled Toffoli through |d>-level controls
(Sec. 2.1.2, Fig. 1), ket labels (Sec. 3.8-3.9), the measurement flag
(Sec. 3.4) and the moment packing of the paper's execution model (Sec. 3.5).
The library's host code produces gate records; the FP64 oracle executes them
and supplies the expected truth tables."""
import itertools

import numpy as np
import pytest

from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


# The sample program as Sec. 4 prints it, typos included ("X X2 2" names x2 in
# capitals; "CX x1 x1 2" controls and targets the same qudit, while the text
# says the generalized CNOT with +2 acts on x1 and x2).
PAPER_QASM = """.qudit 3
qudit x0 (2)
qudit x1 (3)
qudit x2 (3)
.begin
X x0
H x0
Z x0
X x1
X X2 2
CX x0 x1
CX x1 x1 2
.end
"""


def test_qasm_paper_program_as_printed_is_rejected_at_the_self_targeted_cx():
    with pytest.raises(L.QuditError) as e:
        L.qd_qasm_parse(PAPER_QASM)
    assert e.value.code == -3  # QD_ERR_OVERLAP
    assert e.value.line == 12


def test_qasm_paper_program_read_as_its_text_describes():
    # reading: the last line is "CX x1 x2 2", as the text after the listing says
    dims, gates = L.qd_qasm_parse(PAPER_QASM.replace("CX x1 x1 2", "CX x1 x2 2"))
    assert dims == [2, 3, 3]
    want = [("X", (0,), (), 1), ("H", (0,), (), 0), ("Z", (0,), (), 1), ("X", (1,), (), 1), ("X", (2,), (), 2),
            ("X", (1,), (0,), 1), ("X", (2,), (1,), 2)]
    got = [(g.kind, g.targets, g.controls, g.param) for g in gates]
    assert got == want
    # controls fire on d_c - 1 (the paper's C_{X,d}); -1 encodes that default
    assert all(g.levels in (None, (-1,)) for g in gates)
    # the parsed records evolve |000> exactly like the circuit the text describes
    ref = [wl.Gate("X", (0,), param=1), wl.Gate("H", (0,)), wl.Gate("Z", (0,), param=1), wl.Gate("X", (1,), param=1),
           wl.Gate("X", (2,), param=2), wl.Gate("X", (1,), (0,), (1,), 1), wl.Gate("X", (2,), (1,), (2,), 2)]
    a = qo.run_circuit(dims, gates, mode="dense")
    b = qo.run_circuit(dims, ref, mode="dense")
    assert np.max(np.abs(a - b)) == 0.0


@pytest.mark.parametrize("text,code,line", [
    ("qudit x0 (2)\n.begin\n.end\n", -1, 1),                          # declaration before .qudit
    (".qudit 1\nqudit x0 (2)\n.begin\nY x0\n.end\n", -1, 4),           # unknown gate
    (".qudit 1\nqudit x0 (2)\n.begin\nX y0\n.end\n", -1, 4),           # unknown qudit
    (".qudit 1\nqudit x0 (3)\n.begin\nX x0 3\n.end\n", -1, 4),         # shift = d
    (".qudit 1\nqudit x0 (3)\n.begin\nX x0 0\n.end\n", -1, 4),         # shift 0
    (".qudit 1\nqudit x0 (65)\n.begin\n.end\n", -2, 2),                # dimension above 64
    (".qudit 1\nqudit x0 (1)\n.begin\n.end\n", -2, 2),                 # dimension below 2
    (".qudit 2\nqudit x0 (2)\n.begin\n.end\n", -1, 3),                 # fewer declarations than .qudit
    (".qudit 1\nqudit x0 (2)\nX x0\n.begin\n.end\n", -1, 3),           # gate before .begin
    (".qudit 2\nqudit x0 (2)\nqudit X0 (3)\n.begin\n.end\n", -1, 3),   # names are case-insensitive
    (".qudit 1\nqudit x0 (2)\n.begin\nX x0\n", -1, 0),                 # no .end
])
def test_qasm_errors(text, code, line):
    with pytest.raises(L.QuditError) as e:
        L.qd_qasm_parse(text)
    assert e.value.code == code
    assert e.value.line == line


def test_qasm_comments_blank_lines_and_spacing():
    dims, gates = L.qd_qasm_parse("# header\n.qudit 2\n\nqudit a ( 4 )  // ququart\nqudit B (2)\n.begin\n"
                                  "h A\ncx a b\nz b 3\n.end\n")
    assert dims == [4, 2]
    assert [(g.kind, g.targets, g.controls, g.param) for g in gates] == [
        ("H", (0,), (), 0), ("X", (1,), (0,), 1), ("Z", (1,), (), 3)]


def test_toffoli_records_are_the_papers_three_cx():
    # Sec. 3.4: Toffoli((0,1,2), plus=1) -> cx((0,1), plus=1), cx((1,2), plus=1), cx((0,1), plus=2)
    g = L.qd_toffoli_gates([2, 3, 2], 0, 1, 2, 1)
    assert [(x.kind, x.targets, x.controls, x.levels, x.param) for x in g] == [
        ("X", (1,), (0,), (1,), 1), ("X", (2,), (1,), (2,), 1), ("X", (1,), (0,), (1,), 2)]


def _basis_out(dims, gates, levels):
    psi = qo.run_circuit(dims, gates, init_levels=levels)
    i = int(np.argmax(np.abs(psi)))
    assert abs(abs(psi[i]) - 1.0) <= 1e-12
    return qo.decode(i, dims)


@pytest.mark.parametrize("dims,shift", [([2, 3, 2], 1), ([3, 4, 3], 2), ([2, 5, 4], 3)])
def test_toffoli_truth_table(dims, shift):
    gates = L.qd_toffoli_gates(dims, 0, 1, 2, shift)
    for x0 in range(dims[0]):
        for x1 in range(dims[1] - 1):  # the carrier's logical levels
            for x2 in range(dims[2]):
                got = _basis_out(dims, gates, [x0, x1, x2])
                fire = x0 == dims[0] - 1 and x1 == dims[1] - 2
                assert got == [x0, x1, (x2 + shift) % dims[2] if fire else x2], (x0, x1, x2, got)


def _depth(gates):
    """Layers of a greedy as-soon-as-possible schedule (gates on disjoint qudits share a layer)."""
    last = {}
    depth = 0
    for g in gates:
        qs = list(g.targets) + list(g.controls)
        layer = 1 + max((last.get(q, 0) for q in qs), default=0)
        for q in qs:
            last[q] = layer
        depth = max(depth, layer)
    return depth


@pytest.mark.parametrize("nc", range(1, 9))
def test_mct_tree_truth_table_and_depth(nc):
    # controls are qutrits holding qubit values (active level 1, elevated level 2)
    dims = [3] * nc + [2]
    t = nc
    gates, depth = L.qd_mct_tree_gates(dims, list(range(nc)), t, 1)
    levels = int(np.floor(np.log2(nc)))
    assert depth == 2 * levels + 1
    assert _depth(gates) == depth
    assert len(gates) == 2 * (nc // 2) + 1
    assert all(len(g.controls) <= 2 for g in gates)
    for bits in itertools.product(range(2), repeat=nc):
        for xt in range(2):
            got = _basis_out(dims, gates, list(bits) + [xt])
            fire = all(bits)
            assert got == list(bits) + [(xt + 1) % 2 if fire else xt], (bits, xt, got)


def test_mct_tree_mixed_dims_equals_oracle_multi_controlled_gate():
    # controls of dims 4, 5, 3, 6, 4 active at levels 2, 3, 1, 4, 3 (inner controls
    # need a free level above); the target a qutrit shifted by 2
    dims = [4, 5, 3, 6, 4, 3]
    ctrls = [0, 1, 2, 3, 4]
    lv = [2, 3, 1, 4, 3]
    gates, _ = L.qd_mct_tree_gates(dims, ctrls, 5, 2, lv)
    mct = [wl.Gate("X", (5,), tuple(ctrls), tuple(lv), 2)]
    for xs in itertools.product(*[range(l + 1) for l in lv]):
        for xt in range(3):
            init = list(xs) + [xt]
            assert _basis_out(dims, gates, init) == _basis_out(dims, mct, init), init


def test_mct_tree_needs_a_free_level_on_inner_controls():
    with pytest.raises(L.QuditError) as e:
        # qubits active on |1>: the inner control 0 has no level above it
        L.qd_mct_tree_gates([2, 2, 2, 2], [0, 1, 2], 3, 1, [1, 1, 1])
    assert e.value.code == -2
    # a single control needs none (plain generalized CNOT on its top level)
    gates, depth = L.qd_mct_tree_gates([2, 2], [0], 1, 1, [1])
    assert depth == 1 and [(g.targets, g.controls, g.levels) for g in gates] == [((1,), (0,), (1,))]


def test_ket_labels():
    dims = [2, 3, 3]
    assert L.qd_ket_label(dims, qo.encode([1, 2, 0], dims)) == "|120>"
    assert L.qd_ket_label(dims, 0) == "|000>"
    for i in range(18):
        assert L.qd_ket_label(dims, i) == qo.ket_label(i, dims)
    assert L.qd_ket_label([12, 3], qo.encode([11, 2], [12, 3])) == "|11,2>"
    with pytest.raises(L.QuditError):
        L.qd_ket_label(dims, 18)


@pytest.mark.parametrize("seed", range(4))
def test_moment_packing_is_first_moment_after_last_use(seed):
    rng = np.random.default_rng(50 + seed)
    dims = [int(x) for x in rng.choice([2, 3, 4], size=6)]
    gates = wl.random_circuit(dims, 30, 50 + seed, wl.C0_MIX + ("U2",))
    m, nm = L.qd_moment_packing(dims, gates)
    last = {}
    for g, mg in zip(gates, m):
        qs = list(g.targets) + list(g.controls or ())
        want = 1 + max((last.get(q, -1) for q in qs), default=-1)
        assert mg == want
        for q in qs:
            last[q] = mg
    assert nm == 1 + max(m)


def test_measurement_flag_ends_the_circuit():
    dims, gates = wl.circuit_c0()
    k = 17
    cut = gates[:k] + [wl.Gate("MEASURE", ())] + gates[k:]
    # the oracle: gates after the flag are ignored (Sec. 3.4)
    assert np.max(np.abs(qo.run_circuit(dims, cut, mode="dense") - qo.run_circuit(dims, gates[:k], mode="dense"))) == 0
    # the library's planner and moment packing see only the prefix
    m, nm = L.qd_moment_packing(dims, cut)
    assert all(x == -1 for x in m[k:])
    segs, _ = L.qd_debug_fuse_plan(dims, cut, L.QD_PLAN_NONE)
    assert sum(b - a + 1 for a, b in segs) == sum(1 for x in m[:k] if x >= 0)
