"""Fusion planner pins (host only).

* A fused block applied as one matrix over its qudits acts exactly like its
  gates applied in order (checked with the oracle's index-loop mode).
* The exhaustive planner's optimum equals brute-force enumeration of every
  contiguous segmentation under the same cost model (<= 12 gates).
* Greedy and one-gate-per-launch plans never cost less than the optimum.
"""
import itertools

import numpy as np
import pytest

from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.build import build
from paper_2211_07918_gb300.workloads import Gate


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _acting(g, dims):
    return list(g.controls) + list(g.targets)


def _circuit(rng, dims, n):
    mix = ["X", "Z", "H", "CX", "U1", "U2"]
    gates = []
    while len(gates) < n:
        g = wl.random_gate(rng, dims, mix)
        D = int(np.prod([dims[q] for q in _acting(g, dims)]))
        if D <= 32:
            gates.append(g)
    return gates


@pytest.mark.parametrize("seed", range(12))
def test_block_equals_sequential_gates(seed):
    rng = np.random.default_rng(seed)
    dims = [int(x) for x in rng.choice([2, 3, 4], size=int(rng.integers(3, 6)))]
    gates = _circuit(rng, dims, 8)
    N = qo.register_size(dims)
    for _ in range(6):
        a = int(rng.integers(0, len(gates)))
        b = int(rng.integers(a, min(len(gates), a + 3)))
        qs, M = L.qd_debug_fuse_block(dims, gates, a, b)
        psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        want = qo.run_circuit(dims, gates[a:b + 1], psi0=psi)
        got = qo.loop_apply(psi, dims, Gate("U", tuple(qs), matrix=M))
        assert np.max(np.abs(got - want)) <= 1e-12
        assert np.max(np.abs(M @ M.conj().T - np.eye(M.shape[0]))) <= 1e-12


def _is_diag(g):
    return g.kind in ("Z", "DIAG")


def _range_table(dims, qs):
    return int(np.prod(dims[min(qs):max(qs) + 1]))


def _feasible(gates, dims, a, b, kmax, dmax):
    """The planner's segment forms, restated: a block within the limits; a run
    of diagonal gates whose covering qudit range has at most 2^24 states; a
    dense part (<= kmax qudits, <= 16 states) followed by such a run."""
    if a == b:
        return True
    s = set()
    for g in gates[a:b + 1]:
        s |= set(_acting(g, dims))
    if len(s) <= kmax and int(np.prod([dims[q] for q in s])) <= dmax:
        return True
    if all(_is_diag(g) for g in gates[a:b + 1]):
        return _range_table(dims, s) <= 1 << 24
    k = b
    while k >= a and _is_diag(gates[k]):
        k -= 1
    if k == b:
        return False
    pre = set()
    for g in gates[a:k + 1]:
        pre |= set(_acting(g, dims))
    run = set()
    for g in gates[k + 1:b + 1]:
        run |= set(_acting(g, dims))
    return (len(pre) <= kmax and int(np.prod([dims[q] for q in pre])) <= 16
            and _range_table(dims, run) <= 1 << 24)


@pytest.mark.parametrize("prec", [L.QD_C64, L.QD_C128])
@pytest.mark.parametrize("seed", range(8))
def test_exhaustive_equals_brute_force(seed, prec):
    rng = np.random.default_rng(40 + seed)
    dims = [int(x) for x in rng.choice([2, 3, 4], size=5)] + [3] * 9
    n = int(rng.integers(6, 13))
    gates = _circuit(rng, dims, n)
    # the register's default fusion limits, which qd_debug_segment_cost prices with
    kmax, dmax = 3, (64 if prec == L.QD_C64 else 32)
    cost = {}
    for a in range(n):
        for b in range(a, n):
            if _feasible(gates, dims, a, b, kmax, dmax):
                cost[(a, b)] = L.qd_debug_segment_cost(dims, gates, a, b, prec)
    best = np.inf
    for cuts in itertools.product([0, 1], repeat=n - 1):
        segs, start = [], 0
        for i, c in enumerate(cuts):
            if c:
                segs.append((start, i))
                start = i + 1
        segs.append((start, n - 1))
        if all(s in cost for s in segs):
            best = min(best, sum(cost[s] for s in segs))
    segs, c = L.qd_debug_fuse_plan(dims, gates, L.QD_PLAN_EXHAUSTIVE, prec, kmax, dmax)
    assert c == pytest.approx(best, rel=1e-12)
    _, cg = L.qd_debug_fuse_plan(dims, gates, L.QD_PLAN_GREEDY, prec, kmax, dmax)
    _, cn = L.qd_debug_fuse_plan(dims, gates, L.QD_PLAN_NONE, prec, kmax, dmax)
    assert cg >= c * (1 - 1e-12) and cn >= c * (1 - 1e-12)


@pytest.mark.parametrize("kind", [L.QD_PLAN_NONE, L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE])
def test_segments_cover_gates_in_order(kind):
    dims, gates = wl.circuit_c1(ngates=120)
    segs, _ = L.qd_debug_fuse_plan(dims, gates, kind)
    nxt = 0
    for a, b in segs:
        assert a == nxt and b >= a
        assert _feasible(gates, dims, a, b, 3, 32)
        nxt = b + 1
    assert nxt == len(gates)
    if kind != L.QD_PLAN_NONE:
        assert len(segs) < len(gates)


def test_identity_gates_are_dropped_before_fusion():
    dims = [3, 3]
    gates = [Gate("H", (0,)), Gate("Z", (1,), param=3), Gate("H", (1,))]
    segs, _ = L.qd_debug_fuse_plan(dims, gates, L.QD_PLAN_NONE)
    assert len(segs) == 2


def test_segment_of_permutations_is_costed_as_mono():
    """A fused segment whose gates are all permutations with phases is itself
    one and runs on the mono kernel: the cost model sees a memory-only launch.
    In complex128, where a dense 9 x 9 block is arithmetic-bound, the fused
    [X, CX] segment therefore costs less than the fused [H, CX] one on the
    same two qutrits, and no more than the single-qutrit permutation alone
    (the same pass over the state)."""
    dims = [3] * 16
    mono = [Gate("X", (4,), param=1), Gate("X", (9,), (4,), (2,), 2)]
    dense = [Gate("H", (4,)), Gate("X", (9,), (4,), (2,), 2)]
    c_mono = L.qd_debug_segment_cost(dims, mono, 0, 1, L.QD_C128)
    c_dense = L.qd_debug_segment_cost(dims, dense, 0, 1, L.QD_C128)
    c_single = L.qd_debug_segment_cost(dims, mono, 0, 0, L.QD_C128)
    assert c_mono < c_dense
    assert c_mono <= c_single * 1.0001


def test_diagonal_runs_are_planned_as_single_segments():
    """In the d-ary QFT the controlled phases onto one target (Sec. 2.1.2 phase
    gates, controlled) form a run of diagonal gates; the exhaustive planner
    takes each run, whatever its qudit count, into one segment, alone or
    behind the generalized Hadamard before it, and every segment it returns
    is within the block limits, all-diagonal, or a dense part of at most 3
    qudits and 16 states followed by diagonal gates."""
    dims, gates = wl.circuit_c2(n_qubits=3, n_ququarts=5)
    segs, _ = L.qd_debug_fuse_plan(dims, gates, L.QD_PLAN_EXHAUSTIVE, L.QD_C64, 3, 64)
    assert segs[0][0] == 0 and segs[-1][1] == len(gates) - 1
    assert all(b + 1 == c for (_, b), (c, _) in zip(segs, segs[1:]))
    wide = 0
    for a, b in segs:
        qs = {q for g in gates[a:b + 1] for q in tuple(g.targets) + tuple(g.controls or ())}
        if len(qs) <= 3:
            continue
        wide += 1
        k = b
        while k >= a and gates[k].kind in ("Z", "DIAG"):
            k -= 1
        pre = {q for g in gates[a:k + 1] for q in tuple(g.targets) + tuple(g.controls or ())}
        assert k < b, (a, b)  # a diagonal suffix
        assert len(pre) <= 3 and int(np.prod([dims[q] for q in pre])) <= 16, (a, b)
    assert wide >= 1


def test_segment_forms_enumeration():
    """The kernel forms a planner weighs for one segment (host replay of
    qd_segment_forms): a dense gate on qudits (1, 2) followed by diagonal
    gates on qudits 1..3 is a fused block (CUDA-core kernel; tensor cores
    too for complex64, D = 18 >= 9) or a dense part + diagonal run; a single
    gate has its own kernel only; a run of diagonal gates over many qudits is
    a diagonal run (a mono block too while it fits a block); dense gates
    with no diagonal tail have no dense part + run form.  Feature 10 names
    the form, feature 0 is log2 of its dimension (of the table for a run)."""
    rng = np.random.default_rng(4)
    dims = [2, 3, 3, 2, 4, 3]
    seg = [Gate("U", (1, 2), matrix=wl.haar_unitary(9, rng)), Gate("Z", (1,), param=1),
           Gate("DIAG", (3,), (2,), (2,), matrix=np.exp(2j * np.pi * rng.random(2)))]
    for prec, want in ((L.QD_C64, [L.QD_FORM_BLOCK, L.QD_FORM_BLOCK_TC, L.QD_FORM_DENSE_RUN]),
                       (L.QD_C128, [L.QD_FORM_BLOCK, L.QD_FORM_DENSE_RUN])):
        forms = L.qd_debug_segment_forms(dims, seg, 0, 2, prec)
        assert sorted(k for k, _ in forms) == want
        for k, f in forms:
            assert int(f[10]) == k
            if k in (L.QD_FORM_BLOCK, L.QD_FORM_BLOCK_TC):
                assert abs(f[0] - np.log2(18)) < 1e-6 and f[1] == 3  # qudits 1, 2, 3
            else:
                assert abs(f[0] - np.log2(9)) < 1e-6 and f[1] == 2  # the dense part on 1, 2
    # one gate: its own kernel
    assert [k for k, _ in L.qd_debug_segment_forms(dims, seg[:1], 0, 0)] == [L.QD_FORM_DENSE]
    assert [k for k, _ in L.qd_debug_segment_forms(dims, seg[1:2], 0, 0)] == [L.QD_FORM_MONO]
    # two dense gates, no diagonal tail: blocks only
    two = [Gate("U", (0, 1), matrix=wl.haar_unitary(6, rng)), Gate("U", (1, 4), matrix=wl.haar_unitary(12, rng))]
    assert sorted(k for k, _ in L.qd_debug_segment_forms(dims, two, 0, 1)) == [L.QD_FORM_BLOCK, L.QD_FORM_BLOCK_TC]
    # diagonal gates: over qudits 0..2 (18 states) one permutation-with-phases
    # block; over 0..4 (144 states, beyond the 32 of such a block) one
    # diagonal run whose table has 144 entries
    diag = [Gate("DIAG", (q, q + 1), matrix=np.exp(2j * np.pi * rng.random(dims[q] * dims[q + 1])))
            for q in range(4)]
    forms = L.qd_debug_segment_forms(dims, diag, 0, 1)
    assert [k for k, _ in forms] == [L.QD_FORM_MONO]
    assert abs(forms[0][1][0] - np.log2(18)) < 1e-6 and forms[0][1][1] == 3
    forms = L.qd_debug_segment_forms(dims, diag, 0, 3)
    assert [k for k, _ in forms] == [L.QD_FORM_DIAG_RUN]
    assert abs(forms[0][1][0] - np.log2(144)) < 1e-5 and forms[0][1][1] == 5
