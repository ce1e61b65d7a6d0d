"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: values the paper
prints (tests/golden/), closed forms, algebraic identities of the gate
definitions (Sec. 2.1.2), library routines (numpy FFT / Philox), brute force
on tiny inputs, and agreement between its two independent modes.  The
``planted`` tests break a copy of the oracle on purpose and check that a pin
catches it.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import fast as qf
from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.workloads import Gate

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _gate_from_json(g):
    return Gate(g["kind"], tuple(g["targets"]), tuple(g.get("controls", ())),
                tuple(g["levels"]) if g.get("levels") else None, g.get("param", 0))


# ---------------------------------------------------------------- paper values

@pytest.mark.parametrize("mode", ["dense", "loop", "python"])
def test_worked_example(mode):
    gold = _gold("worked_example.json")
    dims = gold["dims"]
    gates = [_gate_from_json(g) for g in gold["gates"]]
    psi = qo.run_circuit(dims, gates, gold["init_levels"], mode=mode)
    kd = qo.ket_dict(psi, dims, "amplitude")
    assert set(kd) == set(gold["amplitudes"])
    for k, v in gold["amplitudes"].items():
        assert abs(kd[k] - v) <= 1e-15
    # everything else is exactly zero
    p = qo.probabilities(psi)
    assert np.count_nonzero(p) == 2


def test_worked_example_c_oracle():
    gold = _gold("worked_example.json")
    dims = gold["dims"]
    gates = [_gate_from_json(g) for g in gold["gates"]]
    psi = qf.run_circuit(dims, gates, gold["init_levels"])
    kd = qo.ket_dict(psi, dims, "amplitude")
    assert set(kd) == set(gold["amplitudes"])
    for k, v in gold["amplitudes"].items():
        assert abs(kd[k] - v) <= 1e-15


def test_f2_matches_paper():
    gold = _gold("f2_matrix.json")
    want = np.array(gold["real"]) + 1j * np.array(gold["imag"])
    assert np.max(np.abs(qo.f_gate(2) - want)) <= 1e-16


def test_cx_block_matrix_matches_paper():
    gold = _gold("cx_d3_blocks.json")
    want = np.array(gold["matrix"], dtype=np.complex128)
    assert np.array_equal(qo.cx_matrix(gold["d"], gold["d"], gold["a"]), want)


def test_register_size_example():
    # Sec. 2.2: a qubit, a qutrit and a ququad give 2*3*4 = 24 entries
    assert qo.register_size([2, 3, 4]) == 24
    assert qo.strides([2, 3, 4]) == [1, 2, 6]


def test_init_state_kron_and_levels():
    # Sec. 3.2 example: dims [4,5,3], init [0,3,2]; Eq. 2 product of columns
    dims, lv = [4, 5, 3], [0, 3, 2]
    a = qo.basis_state(dims, lv)
    b = qo.product_state_kron(dims, lv)
    assert np.array_equal(a, b)
    assert a[0 + 3 * 4 + 2 * 20] == 1.0


# ------------------------------------------------------------------ algebra

DS = [2, 3, 4, 5, 6, 7, 8]


@pytest.mark.parametrize("d", DS)
def test_x_power_d_is_identity(d):
    x = qo.x_gate(d, 1)
    assert np.array_equal(np.linalg.matrix_power(x, d), np.eye(d))
    for a in range(1, d):
        assert np.array_equal(qo.x_gate(d, a), np.linalg.matrix_power(x, a))


@pytest.mark.parametrize("d", DS)
def test_zx_commutation(d):
    w = np.exp(2j * np.pi / d)
    z, x = qo.z_gate(d), qo.x_gate(d)
    assert np.max(np.abs(z @ x - w * (x @ z))) <= 1e-13


@pytest.mark.parametrize("d", DS)
def test_f_is_normalised_dft(d):
    # F_d[j,k] = w^{jk}/sqrt(d) equals sqrt(d) times numpy's inverse DFT matrix
    f = qo.f_gate(d)
    ref = np.fft.ifft(np.eye(d), axis=0) * math.sqrt(d)
    assert np.max(np.abs(f - ref)) <= 1e-13
    assert np.max(np.abs(f @ f.conj().T - np.eye(d))) <= 1e-13
    par = np.zeros((d, d))
    for x in range(d):
        par[(-x) % d, x] = 1
    assert np.max(np.abs(f @ f - par)) <= 1e-13
    xinv = qo.x_gate(d, d - 1)
    assert np.max(np.abs(f @ qo.z_gate(d) @ f.conj().T - xinv)) <= 1e-13


def test_exact_quarter_turns():
    assert np.array_equal(qo.z_gate(2), np.diag([1.0, -1.0]).astype(complex))
    assert np.array_equal(qo.z_gate(4), np.diag([1, 1j, -1, -1j]))


# --------------------------------------------------------- modes agree

def _random_small_case(rng):
    n = int(rng.integers(1, 7))
    dims = [int(x) for x in rng.integers(2, 6, size=n)]
    while qo.register_size(dims) > 2048:
        dims.pop()
    n = len(dims)
    mix = ["X", "Z", "H", "U1"] + (["CX", "U2"] if n >= 2 else [])
    gates = [wl.random_gate(rng, dims, mix) for _ in range(12)]
    if n >= 3:
        # a controlled two-target gate with mixed dims and a three-target gate
        c, t1, t2 = (int(x) for x in rng.choice(n, size=3, replace=False))
        D = dims[t1] * dims[t2]
        gates.append(Gate("U", (t1, t2), (c,), (int(rng.integers(0, dims[c])),),
                          matrix=wl.haar_unitary(D, rng)))
        a, b, e = (int(x) for x in rng.choice(n, size=3, replace=False))
        gates.append(Gate("U", (a, b, e), matrix=wl.haar_unitary(dims[a] * dims[b] * dims[e], rng)))
        gates.append(Gate("DIAG", (b, a), matrix=np.exp(2j * np.pi * rng.random(dims[a] * dims[b]))))
    return dims, gates


@pytest.mark.parametrize("seed", range(12))
def test_loop_equals_dense(seed):
    rng = np.random.default_rng(100 + seed)
    dims, gates = _random_small_case(rng)
    psi0 = rng.standard_normal(qo.register_size(dims)) + 1j * rng.standard_normal(qo.register_size(dims))
    psi0 /= np.sqrt(qo.norm2(psi0))
    a = qo.run_circuit(dims, gates, mode="dense", psi0=psi0)
    b = qo.run_circuit(dims, gates, mode="loop", psi0=psi0)
    c = qf.run_circuit(dims, gates, psi0=psi0)
    assert np.max(np.abs(a - b)) <= 1e-13
    assert np.max(np.abs(a - c)) <= 1e-13
    if qo.register_size(dims) <= 400:
        d = qo.run_circuit(dims, gates, mode="python", psi0=psi0)
        assert np.max(np.abs(a - d)) <= 1e-13


def test_c0_dense_loop_c_agree_and_norm():
    dims, gates = wl.circuit_c0()
    psi_d = qo.basis_state(dims)
    psi_c = qo.basis_state(dims)
    for g in gates:
        psi_d = qo.dense_apply(psi_d, dims, g)
        qf.apply(psi_c, dims, g)
        assert abs(qo.norm2(psi_d) - 1.0) <= 1e-13
        assert np.max(np.abs(psi_d - psi_c)) <= 1e-13


def test_multi_target_order_matters():
    # first-listed target is the most significant local digit: an asymmetric
    # gate on (0,2) and (2,0) must give different states, each equal to the
    # dense definition
    rng = np.random.default_rng(7)
    dims = [2, 3, 4]
    u = wl.haar_unitary(8, rng)
    psi0 = rng.standard_normal(24) + 0j
    ga = Gate("U", (0, 2), matrix=u)
    gb = Gate("U", (2, 0), matrix=u)
    a = qo.loop_apply(psi0, dims, ga)
    b = qo.loop_apply(psi0, dims, gb)
    assert np.max(np.abs(a - b)) > 1e-3
    assert np.max(np.abs(a - qo.dense_apply(psi0, dims, ga))) <= 1e-13
    assert np.max(np.abs(b - qo.dense_apply(psi0, dims, gb))) <= 1e-13


def test_single_qudit_against_brute_force_definition():
    # G on qudit q acts on digit q alone: check every matrix element of U_full
    # by the definition <y|U_full|x> = G[y_q, x_q] * prod_{p != q} delta(y_p, x_p)
    dims = [3, 2, 4]
    rng = np.random.default_rng(3)
    for q in range(3):
        g = wl.haar_unitary(dims[q], rng)
        u = qo.full_unitary(dims, g, [q])
        for x in range(24):
            for y in range(24):
                xs, ys = qo.decode(x, dims), qo.decode(y, dims)
                same = all(xs[p] == ys[p] for p in range(3) if p != q)
                want = g[ys[q], xs[q]] if same else 0
                assert u[y, x] == want


# ------------------------------------------------------ controlled gates

@pytest.mark.parametrize("seed", range(4))
def test_controlled_acts_only_on_level(seed):
    rng = np.random.default_rng(seed)
    dims = [3, 2, 4, 3]
    psi = rng.standard_normal(72) + 1j * rng.standard_normal(72)
    c, t = 3, 2
    lvl = int(rng.integers(0, 3))
    u = wl.haar_unitary(4, rng)
    gc = Gate("U", (t,), (c,), (lvl,), matrix=u)
    out = qo.loop_apply(psi, dims, gc)
    full = qo.loop_apply(psi, dims, Gate("U", (t,), matrix=u))
    digit = (np.arange(72) // qo.strides(dims)[c]) % dims[c]
    off = digit != lvl
    assert np.array_equal(out[off], psi[off])           # bit-identical
    assert np.max(np.abs(out[~off] - full[~off])) <= 1e-15
    assert np.max(np.abs(out - qo.dense_apply(psi, dims, gc))) <= 1e-13


def test_mct_fires_only_when_all_controls_at_top_level():
    dims = [3, 3, 3]
    g = Gate("X", (2,), (0, 1), None, 1)
    for x in range(27):
        psi = np.zeros(27, complex)
        psi[x] = 1
        out = qo.loop_apply(psi, dims, g)
        xs = qo.decode(x, dims)
        ys = list(xs)
        if xs[0] == 2 and xs[1] == 2:
            ys[2] = (xs[2] + 1) % 3
        assert out[qo.encode(ys, dims)] == 1


# --------------------------------------------------------- Toffoli ladders

def test_paper_toffoli_decomposition_truth_table():
    # Sec. 3.4: Toffoli((0,1,2), plus=1) = cx((0,1),+1), cx((1,2),+1),
    # cx((0,1),+2) with qudit 1 an intermediate qutrit; controls fire at d-1
    dims = [2, 3, 2]
    gates = [Gate("X", (1,), (0,), None, 1), Gate("X", (2,), (1,), None, 1), Gate("X", (1,), (0,), None, 2)]
    for a, b, c in itertools.product([0, 1], repeat=3):
        psi = qo.run_circuit(dims, gates, [a, b, c])
        out = qo.decode(int(np.argmax(np.abs(psi))), dims)
        assert out == [a, b, c ^ (a & b)]
        assert abs(abs(psi[qo.encode(out, dims)]) - 1) < 1e-15


def test_ququart_toffoli_rung_truth_table():
    # the ladder rung: controls qubit 0 and ququart 2 (binary use), target qubit 1
    dims = [2, 2, 4]
    gates = wl.toffoli_rung(0, 2, 1, 4)
    for a, b, c in itertools.product([0, 1], repeat=3):
        psi = qo.run_circuit(dims, gates, [a, c, b])
        out = qo.decode(int(np.argmax(np.abs(psi))), dims)
        assert out == [a, c ^ (a & b), b]


# ----------------------------------------------------------------- QFT

@pytest.mark.parametrize("nq", [1, 2, 3, 4])
def test_qft_closed_form(nq):
    # d=4 QFT on nq ququarts after 2 qubits: with output digits reversed, the
    # ququart amplitudes equal sqrt(M) * ifft(input) (normalised DFT, w=+)
    rng = np.random.default_rng(nq)
    dims = [2, 2] + [4] * nq
    M = 4 ** nq
    psi0 = rng.standard_normal(4 * M) + 1j * rng.standard_normal(4 * M)
    gates = wl.qft_gates(list(range(2, 2 + nq)), 4)
    out = qo.run_circuit(dims, gates, mode="loop", psi0=psi0)
    for low in range(4):
        x_in = psi0[low::4]
        y = out[low::4]
        rev = np.empty(M, dtype=np.int64)
        for k in range(M):
            ds = [(k // 4 ** i) % 4 for i in range(nq)]
            rev[k] = sum(dd * 4 ** (nq - 1 - i) for i, dd in enumerate(ds))
        want = np.fft.ifft(x_in) * math.sqrt(M)
        assert np.max(np.abs(y[rev] - want)) <= 1e-12


# ------------------------------------------------------------ readout

def test_marginals_and_cdf():
    rng = np.random.default_rng(5)
    dims = [3, 2, 5]
    psi = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    p = qo.probabilities(psi)
    for q in range(3):
        m = qo.marginal(psi, dims, q)
        brute = np.zeros(dims[q])
        for i in range(30):
            brute[qo.decode(i, dims)[q]] += abs(psi[i]) ** 2
        assert np.max(np.abs(m - brute)) <= 1e-13
    c = qo.cdf(psi)
    assert abs(c[-1] - qo.norm2(psi)) <= 1e-12
    assert np.all(np.diff(c) >= 0)
    assert abs(c[7] - sum(p[:8])) <= 1e-13


def test_sampling_fixed_u_exact():
    # probabilities 1/4 (exact in binary): CDF = [.25, .25, .5, .75, 1]
    psi = np.array([0.5, 0.0, 0.5, 0.5, 0.5]) + 0j
    c = qo.cdf(psi)
    u = np.array([0.0, 0.2, 0.25, 0.26, 0.5, 0.74, 0.75, 0.99])
    got = qo.sample_from_cdf(c, u)
    # smallest i with CDF_i > u*total; the zero-probability index 1 is never
    # drawn and a u on a boundary goes to the next index
    assert list(got) == [0, 0, 2, 2, 3, 3, 4, 4]


def test_philox_matches_numpy():
    # numpy's Philox bit generator is Philox4x64-10 and pre-increments its
    # counter: its first block for counter c is our block for c+1
    for key, ctr in [((0, 0), 0), ((7, 9), 5), ((2**63 + 11, 3), 2**40)]:
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([ctr, 0, 0, 0], dtype=np.uint64))
        want = [int(x) for x in bg.random_raw(4)]
        assert qo.philox4x64([ctr + 1, 0, 0, 0], key) == want


def test_sampling_chi2():
    rng = np.random.default_rng(11)
    dims = [3, 3, 2]
    psi = rng.standard_normal(18) + 1j * rng.standard_normal(18)
    psi /= np.sqrt(qo.norm2(psi))
    shots = 20000
    s = qo.sample(psi, seed=1234, shots=shots)
    counts = np.bincount(s, minlength=18)
    exp = qo.probabilities(psi) * shots
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 45.0  # 17 dof, p ~ 3e-4


# --------------------------------------------------------- planted mistakes

def test_planted_transposed_operand_is_caught(monkeypatch):
    # a loop mode that applies G^T instead of G must fail the dense agreement
    real = qo.target_matrix

    def transposed(gate, dims):
        return real(gate, dims).T

    rng = np.random.default_rng(1)
    dims, gates = [3, 3, 2], [Gate("U", (1,), matrix=wl.haar_unitary(3, rng))]
    psi0 = rng.standard_normal(18) + 0j
    good = qo.run_circuit(dims, gates, mode="dense", psi0=psi0)
    monkeypatch.setattr(qo, "target_matrix", transposed)
    bad = qo.run_circuit(dims, gates, mode="loop", psi0=psi0)
    assert np.max(np.abs(good - bad)) > 1e-3


def test_planted_msb_convention_is_caught(monkeypatch):
    # building U_full with qudit 0 as the MSB must break the worked example
    gold = _gold("worked_example.json")
    dims = gold["dims"]
    gates = [_gate_from_json(g) for g in gold["gates"]]

    def msb_strides(ds):
        out, s = [0] * len(ds), 1
        for q in range(len(ds) - 1, -1, -1):
            out[q] = s
            s *= ds[q]
        return out

    monkeypatch.setattr(qo, "strides", msb_strides)
    psi = qo.run_circuit(dims, gates, gold["init_levels"], mode="loop")
    assert set(qo.ket_dict(psi, dims)) != set(gold["amplitudes"])


def test_planted_control_on_wrong_level_is_caught():
    # a CX firing on level 0 instead of d-1 fails the paper's truth table
    dims = [2, 3, 2]
    gates = [Gate("X", (1,), (0,), (0,), 1), Gate("X", (2,), (1,), (0,), 1), Gate("X", (1,), (0,), (0,), 2)]
    psi = qo.run_circuit(dims, gates, [1, 1, 0])
    out = qo.decode(int(np.argmax(np.abs(psi))), dims)
    assert out != [1, 1, 1]
