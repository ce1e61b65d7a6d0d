"""Seeded synthetic workloads: gate records and circuits.

This module is the only code shared by the CUDA path's tests and benchmark
and by the FP64 oracle, and it holds none of the method's arithmetic: it
draws gate *descriptions* (kind, acting qudits, shift, control levels) and the
random matrices of user-defined gates, which both sides receive as data.  The
named gates (X, Z, H) are built independently by each side from their
definitions.

The paper's own benchmark circuits (RevLib netlists, the algorithm circuits of
its Tables 1-3) are not available here; these seeded circuits stand in for
them with the shapes the paper works with: random circuits over the
generalized gate set, a d-ary QFT, and Toffoli ladders decomposed through an
elevated intermediate level (Sec. 2.1.2, Fig. 1; Sec. 3.4 Toffoli example).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np


@dataclass
class Gate:
    """One gate of a circuit.

    kind     "X" (shift ``param``), "Z" (power ``param``), "H" (generalized
             Hadamard F_d), "U" (dense D x D ``matrix``), "DIAG" (D diagonal
             entries in ``matrix``)
    targets  acting qudits; the first listed is the most significant digit of
             the gate's local index
    controls control qudits (may be empty)
    levels   the level each control must hold for the gate to act; None means
             d_c - 1 for every control (the paper's C_{X,d} convention)
    """
    kind: str
    targets: tuple
    controls: tuple = ()
    levels: Optional[tuple] = None
    param: int = 0
    matrix: Optional[np.ndarray] = field(default=None, repr=False)


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random d x d unitary: QR of a complex Ginibre matrix with the
    phases of R's diagonal moved into Q (Mezzadri 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return np.ascontiguousarray(q * ph[None, :], dtype=np.complex128)


def _cx(rng, dims, c, t):
    return Gate("X", (t,), (c,), (int(rng.integers(0, dims[c])),), int(rng.integers(1, dims[t])))


def random_gate(rng: np.random.Generator, dims: Sequence[int], mix: Sequence[str]) -> Gate:
    """One gate drawn uniformly from ``mix`` on uniformly drawn qudits.

    mix entries: "X" (shift a uniform in [1, d-1]), "Z" (power 1), "H",
    "CX" (distinct control/target, control level uniform in [0, d_c), shift
    uniform in [1, d_t-1]), "U1" (Haar single-qudit), "U2" (Haar two-qudit on
    a distinct ordered pair)."""
    n = len(dims)
    kind = mix[int(rng.integers(0, len(mix)))]
    q = int(rng.integers(0, n))
    if kind == "X":
        return Gate("X", (q,), param=int(rng.integers(1, dims[q])))
    if kind == "Z":
        return Gate("Z", (q,), param=1)
    if kind == "H":
        return Gate("H", (q,))
    if kind == "U1":
        return Gate("U", (q,), matrix=haar_unitary(dims[q], rng))
    if kind in ("CX", "U2"):
        c, t = (int(x) for x in rng.choice(n, size=2, replace=False))
        if kind == "CX":
            return _cx(rng, dims, c, t)
        return Gate("U", (c, t), matrix=haar_unitary(dims[c] * dims[t], rng))
    raise ValueError(kind)


C0_MIX = ("X", "Z", "H", "CX", "U1")


def random_circuit(dims: Sequence[int], ngates: int, seed: int, mix: Sequence[str] = C0_MIX) -> list:
    rng = np.random.default_rng(seed)
    return [random_gate(rng, dims, mix) for _ in range(ngates)]


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

C0_DIMS = (3, 3, 3, 3, 2, 2)


def circuit_c0(seed: int = 0, ngates: int = 40):
    """Tiny register [3,3,3,3,2,2] (324 amplitudes), 40 gates uniform over
    X shift, Z clock, F_d, controlled-X on a random level, Haar-1."""
    return list(C0_DIMS), random_circuit(C0_DIMS, ngates, seed, C0_MIX)


def circuit_c1(seed: int = 1, n: int = 14, ngates: int = 500, d: int = 3):
    """n qutrits, ``ngates`` gates: 40% Haar single-qutrit, 30% F_3, 30%
    controlled-X_3 on random distinct control/target pairs and random control
    levels, in a seeded random order."""
    rng = np.random.default_rng(seed)
    dims = [d] * n
    n_u = (ngates * 4) // 10
    n_h = (ngates * 3) // 10
    kinds = ["U1"] * n_u + ["H"] * n_h + ["CX"] * (ngates - n_u - n_h)
    order = rng.permutation(len(kinds))
    gates = []
    for k in order:
        gates.append(random_gate(rng, dims, [kinds[k]]))
    return dims, gates


def qft_phase_diag(x_weight_denominator: int, dc: int, dt: int) -> np.ndarray:
    """Diagonal of the QFT's controlled phase between a control digit x_c
    and a target digit x_t: exp(2 pi i x_c x_t / den), over the local index
    (control most significant).  This is a user-supplied gate matrix."""
    v = np.empty(dc * dt, dtype=np.complex128)
    for xc in range(dc):
        for xt in range(dt):
            m = (xc * xt) % x_weight_denominator
            t = 2.0 * math.pi * m / x_weight_denominator
            v[xc * dt + xt] = complex(math.cos(t), math.sin(t))
    return v


def qft_gates(qudits: Sequence[int], d: int) -> list:
    """d-ary QFT on ``qudits`` (listed least significant first).

    Reading (the paper cites the d-ary QFT without defining it): for i from
    the most significant qudit down, apply F_d on qudit i, then for every
    lower j a controlled phase exp(2 pi i x_j x_i / d^(i-j+1)); no final
    digit reversal, so the output frequency digits come out reversed."""
    gates = []
    n = len(qudits)
    for i in range(n - 1, -1, -1):
        gates.append(Gate("H", (qudits[i],)))
        for j in range(i - 1, -1, -1):
            den = d ** (i - j + 1)
            gates.append(Gate("DIAG", (qudits[j], qudits[i]), matrix=qft_phase_diag(den, d, d)))
    return gates


def toffoli_rung(c1: int, carrier: int, target: int, d_carrier: int, elevated: int = 2) -> list:
    """Toffoli(c1, carrier -> target) through an elevated carrier level.

    Following the paper's Toffoli decomposition into three CX gates
    (Sec. 3.4) and the |d>-level activation of Fig. 1: raise the carrier by
    one when c1 = 1, flip the target when the carrier is at the elevated
    level, then lower the carrier again (shift d_carrier - 1 is the inverse
    of +1 mod d_carrier)."""
    return [
        Gate("X", (carrier,), (c1,), (1,), 1),
        Gate("X", (target,), (carrier,), (elevated,), 1),
        Gate("X", (carrier,), (c1,), (1,), d_carrier - 1),
    ]


C2_DIMS = tuple([2] * 8 + [4] * 12)


def circuit_c2(seed: int = 2, n_qubits: int = 8, n_ququarts: int = 12, rungs: Optional[int] = None):
    """Hybrid register of qubits followed by ququarts: a seeded Haar layer on
    every qudit, a d=4 QFT on the ququarts, then a ladder of Toffoli rungs
    whose controls are qubit r and ququart r and whose target is qubit r+1."""
    rng = np.random.default_rng(seed)
    dims = [2] * n_qubits + [4] * n_ququarts
    gates = [Gate("U", (q,), matrix=haar_unitary(dims[q], rng)) for q in range(len(dims))]
    gates += qft_gates(list(range(n_qubits, n_qubits + n_ququarts)), 4)
    if rungs is None:
        rungs = min(n_qubits - 1, n_ququarts)
    for r in range(rungs):
        gates += toffoli_rung(r, n_qubits + r, r + 1, 4)
    return dims, gates


C3_MAX_TOTAL = 5 ** 12


def batch_c3(seed: int = 1000, count: int = 256, ngates: int = 200, nmin: int = 6, nmax: int = 12,
             dim_choices=(2, 3, 4, 5), max_total: int = C3_MAX_TOTAL):
    """``count`` independent circuits: circuit c draws n in [nmin, nmax] and
    dims uniformly from ``dim_choices`` with seed ``seed + c``; if the running
    amplitude total would pass ``max_total`` the circuit is redrawn with seed
    seed + c + count*k.  Gates: the C0 mix plus two-qudit Haar."""
    out, total = [], 0
    mix = C0_MIX + ("U2",)
    for c in range(count):
        k = 0
        while True:
            rng = np.random.default_rng(seed + c + count * k)
            n = int(rng.integers(nmin, nmax + 1))
            dims = [int(x) for x in rng.choice(dim_choices, size=n)]
            N = int(np.prod(dims))
            if total + N <= max_total or k > 64:
                break
            k += 1
        total += N
        out.append((dims, [random_gate(rng, dims, mix) for _ in range(ngates)]))
    return out


C4_DIMS = tuple([3] * 18 + [2] * 4)


def circuit_c4(seed: int = 4000, ngates: int = 1000):
    dims = list(C4_DIMS)
    return dims, random_circuit(dims, ngates, seed, C0_MIX + ("U2",))


def worked_example():
    """The paper's worked example (Sec. 3.9): dims [2,3,3], start |000>,
    F on qudit 0, then CX_{+2} with control qudit 0 and target qudit 1."""
    return [2, 3, 3], [Gate("H", (0,)), Gate("X", (1,), (0,), None, 2)]


def amplitude_updates(dims: Sequence[int], gates: Sequence[Gate]) -> int:
    """Number of original gates times N (the amp-updates/s numerator)."""
    return len(gates) * int(np.prod(dims))
