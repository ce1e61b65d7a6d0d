"""GPU tests of the circuit layer through the C ABI: ket readout (Sec. 3.8;
the worked example's printed output, Sec. 3.9), the measurement flag
(Sec. 3.4), the Toffoli and logarithmic-depth MCT decompositions applied to a
register (Sec. 3.4; Sec. 2.1.2 Fig. 1), a QASM program run end to end
(Sec. 4), and the paper's own moment / Kronecker / GEMM-chain execution model
(Sec. 3.5-3.6) against the FP64 oracle."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def _golden_gates(d):
    return [wl.Gate(g["kind"], tuple(g["targets"]), tuple(g.get("controls", ())), None, g.get("param", 0))
            for g in d["gates"]]


@pytest.mark.parametrize("prec,tol", [(L.QD_C128, 1e-15), (L.QD_C64, 1e-7)])
def test_worked_example_ket_output(prec, tol):
    with open(os.path.join(GOLDEN, "worked_example.json")) as f:
        d = json.load(f)
    dims = d["dims"]
    c = L.Circuit(dims)
    c.gates = _golden_gates(d)
    c.measure_all()
    with L.Register(dims, d["init_levels"], prec) as r:
        c.run(r.h)
        assert L.qd_is_measured(r.h)
        amp = L.ket_dict(r.h, dims, L.QD_OUT_AMPLITUDE)
        prob = L.output(r.h, dims, "print", "probability")
        state = L.output(r.h, dims, "state", "amplitude")
    assert sorted(amp) == sorted(d["amplitudes"])
    for k, v in d["amplitudes"].items():
        assert abs(amp[k] - v) <= tol
        assert abs(prob[k] - v * v) <= 2 * tol
    assert state.shape == (18,)


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
@pytest.mark.parametrize("dims", [[3] * 9, [4] * 7 + [2], [5, 3, 2, 4, 3, 7]])
def test_ket_list_matches_oracle(prec, dims):
    """A random state with a third of its entries zeroed: the kept entries,
    their order, and their values equal the oracle's ket dict; a cap below the
    total returns the first cap entries and the full count.  Sizes span many
    4096-amplitude chunks with a ragged last one."""
    rng = np.random.default_rng(sum(dims) + prec)
    N = qo.register_size(dims)
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi[rng.random(N) < 0.33] = 0.0
    psi /= np.linalg.norm(psi)
    psi = psi.astype(np.complex64 if prec == L.QD_C64 else np.complex128)
    ref_state = psi.astype(np.complex128)
    thr = 1e-14 if prec == L.QD_C128 else 1e-12
    with L.Register(dims, None, prec) as r:
        L.qd_set_amplitudes(r.h, psi)
        idx, vals, total = L.qd_ket_list(r.h, L.QD_OUT_AMPLITUDE, thr)
        pidx, pvals, ptotal = L.qd_ket_list(r.h, L.QD_OUT_PROBABILITY, thr)
        cidx, cvals, ctotal = L.qd_ket_list(r.h, L.QD_OUT_AMPLITUDE, thr, cap=1000)
    want = np.nonzero(qo.probabilities(ref_state) > thr)[0]
    assert total == ptotal == ctotal == len(want)
    assert np.array_equal(idx, want) and np.array_equal(pidx, want)
    assert np.max(np.abs(vals - ref_state[want])) == 0.0
    assert np.max(np.abs(pvals - qo.probabilities(ref_state)[want])) <= 1e-15
    assert np.array_equal(cidx, want[:1000]) and np.array_equal(cvals, ref_state[want[:1000]])


def test_ket_list_threshold_and_empty():
    dims = [2, 2, 2]
    with L.Register(dims, None, L.QD_C128) as r:
        idx, vals, total = L.qd_ket_list(r.h, L.QD_OUT_PROBABILITY, 0.5)
        assert total == 1 and list(idx) == [0] and vals[0] == 1.0
        idx, vals, total = L.qd_ket_list(r.h, L.QD_OUT_PROBABILITY, 1.0)
        assert total == 0 and len(idx) == 0


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_measurement_flag(prec):
    dims, gates = wl.circuit_c0()
    k = 23
    ref = qo.run_circuit(dims, gates[:k], mode="dense")
    cut = gates[:k] + [wl.Gate("MEASURE", ())] + gates[k:]
    tol = 1e-12 if prec == L.QD_C128 else 1e-5
    with L.Register(dims, None, prec) as r:
        plan = L.qd_plan_create(r.h, cut, L.QD_PLAN_NONE)
        L.qd_plan_run(plan)
        assert L.qd_is_measured(r.h)
        L.qd_apply_h(r.h, 0)                 # ignored after the flag
        L.qd_run_circuit(r.h, gates[k:])     # ignored
        L.qd_plan_run(plan)                  # ignored
        assert np.max(np.abs(r.amplitudes() - ref)) <= tol
        L.qd_reset(r.h)                      # a new circuit
        assert not L.qd_is_measured(r.h)
        L.qd_plan_run(plan)
        assert np.max(np.abs(r.amplitudes() - ref)) <= tol
        L.qd_reset(r.h)
        L.qd_measure_all(r.h)
        L.qd_apply_x(r.h, 0, 1)
        assert np.max(np.abs(r.amplitudes() - qo.basis_state(dims))) == 0.0


def test_toffoli_and_mct_tree_on_the_register():
    # Toffoli: qubit control, qutrit carrier, qubit target (the paper's mapping)
    dims = [2, 3, 2]
    for x0, x1, x2 in itertools.product(range(2), range(2), range(2)):
        with L.Register(dims, [x0, x1, x2], L.QD_C128) as r:
            L.qd_apply_toffoli(r.h, 0, 1, 2, 1)
            out = r.amplitudes()
        want = qo.basis_state(dims, [x0, x1, (x2 + 1) % 2 if (x0 and x1) else x2])
        assert np.max(np.abs(out - want)) == 0.0
    # MCT over 6 qutrit-held qubits onto a ququart target (shift 3)
    dims = [3] * 6 + [4]
    for bits in itertools.product(range(2), repeat=6):
        for xt in (0, 2):
            with L.Register(dims, list(bits) + [xt], L.QD_C64) as r:
                L.qd_apply_mct_tree(r.h, list(range(6)), 6, 3)
                out = r.amplitudes()
            fire = all(bits)
            want = qo.basis_state(dims, list(bits) + [(xt + 3) % 4 if fire else xt])
            assert np.max(np.abs(out - want)) == 0.0, (bits, xt)


def test_mct_tree_on_superposition_equals_oracle_mct():
    rng = np.random.default_rng(5)
    dims = [3, 3, 3, 3, 3, 2]
    # a superposition inside the logical subspace of the controls (levels 0, 1)
    psi0 = qo.run_circuit(dims, [])
    for q in range(6):
        U = np.eye(dims[q], dtype=np.complex128)
        U[:2, :2] = wl.haar_unitary(2, rng)
        psi0 = qo.run_circuit(dims, [wl.Gate("U", (q,), matrix=U)], psi0=psi0)
    ref = qo.run_circuit(dims, [wl.Gate("X", (5,), tuple(range(5)), (1,) * 5, 1)], psi0=psi0)
    with L.Register(dims, None, L.QD_C128) as r:
        L.qd_set_amplitudes(r.h, psi0)
        L.qd_apply_mct_tree(r.h, list(range(5)), 5, 1, [1] * 5)
        out = r.amplitudes()
    assert np.max(np.abs(out - ref)) <= 1e-14


def test_qasm_program_end_to_end():
    text = (".qudit 4\nqudit a (2)\nqudit b (3)\nqudit c (4)\nqudit d (3)\n.begin\n"
            "H a\nH c\nCX a b\nCX c d 2\nZ b\nX d 1\nH b\nCX b c 3\n.end\n")
    dims, gates = L.qd_qasm_parse(text)
    ref = qo.run_circuit(dims, gates, mode="dense")
    with L.Register(dims, None, L.QD_C128) as r:
        L.qd_run_circuit(r.h, gates)
        assert np.max(np.abs(r.amplitudes() - ref)) <= 1e-12


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
@pytest.mark.parametrize("case", ["c0", "r0", "r1", "r2"])
def test_moment_path_matches_oracle(prec, case):
    if case == "c0":
        dims, gates = wl.circuit_c0()
    else:
        seed = 60 + int(case[1])
        rng = np.random.default_rng(seed)
        dims = [int(x) for x in rng.choice([2, 3, 4], size=int(rng.integers(4, 7)))]
        while qo.register_size(dims) > 1024:
            dims.pop()
        gates = wl.random_circuit(dims, 30, seed, wl.C0_MIX + ("U2",))
    ref = qo.run_circuit(dims, gates, mode="dense")
    _, nm_host = L.qd_moment_packing(dims, gates)
    with L.Register(dims, None, prec) as r:
        nm = L.qd_run_moments(r.h, gates)
        out = r.amplitudes().astype(np.complex128)
    assert nm == nm_host
    err = np.max(np.abs(out - ref))
    # complex128: the GEMM chain sums N products per entry per moment
    assert err <= (1e-12 if prec == L.QD_C128 else 1e-6), err


def test_moment_path_rejects_large_registers():
    with L.Register([2] * 13, None, L.QD_C128) as r:
        with pytest.raises(L.QuditError) as e:
            L.qd_run_moments(r.h, [wl.Gate("H", (0,))])
        assert e.value.code == -2
