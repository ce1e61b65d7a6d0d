"""FP64 CPU oracle for generalized qudit gates on mixed-radix registers.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library; the two meet only through the seeded circuit descriptions
produced by ``paper_2211_07918_gb300.workloads``.

What it computes (QuDiet, arXiv 2211.07918):

* A register is a list of qudit dimensions d_0..d_{n-1}; the state has
  N = prod d_q amplitudes (Sec. 2.2).  The first qudit is the least
  significant digit (Sec. 3.2, description of ``qregs``), so the flat index is
  i = sum_q x_q s_q with s_q = prod_{p<q} d_p.
* Each qudit starts in a computational basis level, |0> by default
  (Sec. 3.2 ``init_states``; Sec. 2.2 "circuits on qudits ... start in |0>").
* Gates (Sec. 2.1.2): the generalized NOT X^d_{+a}|x> = |(x+a) mod d>,
  1 <= a <= d-1; the phase-shift gate Z_d = diag(1, w, ..., w^{d-1}) with
  w = exp(2 pi i / d); the generalized Hadamard F_d[j,k] = w^{jk}/sqrt(d);
  the generalized CNOT / INCREMENT C_{X,d}, block-diagonal with X^d_{+a} in the
  block of control level d-1; the multi-controlled Toffoli C^n_{X,d} that fires
  when every control is at level d-1; user-defined k-qudit matrices
  (Sec. 3.4, "User Defined Gate").
* The evolution is psi <- U_full psi, U_full the gate padded with identities
  by Kronecker products (Sec. 3.5 and 3.6, the Moment and OperatorFlow
  evaluation), starting from the InitState product vector (Sec. 3.3, Eq. 2).

Two independent evaluation modes:

``dense`` builds U_full explicitly (the paper's own definition) and is only
usable for N <= ~4096.  ``loop`` walks the basis index space by digit decode
and applies the gate matrix once per group of D = prod_t d_t amplitudes.

Readings of points the paper leaves open are documented at each function; the
list is repeated in the repository's design notes.
"""
from __future__ import annotations

import math
from typing import Iterable, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Register geometry (Sec. 2.2, Sec. 3.2)
# ---------------------------------------------------------------------------


def register_size(dims: Sequence[int]) -> int:
    """N = prod of the qudit dimensions (Sec. 2.2: (2,3,4) gives 24 entries)."""
    n = 1
    for d in dims:
        n *= int(d)
    return n


def strides(dims: Sequence[int]) -> list[int]:
    """s_q = prod_{p<q} d_p: qudit 0 is the least significant digit (Sec. 3.2)."""
    out, s = [], 1
    for d in dims:
        out.append(s)
        s *= int(d)
    return out


def decode(i: int, dims: Sequence[int]) -> list[int]:
    """Digits (x_0..x_{n-1}) of basis index i by repeated div/mod, qudit 0 first."""
    xs = []
    for d in dims:
        xs.append(i % d)
        i //= d
    return xs


def encode(xs: Sequence[int], dims: Sequence[int]) -> int:
    """Inverse of :func:`decode`."""
    i = 0
    for x, s in zip(xs, strides(dims)):
        i += int(x) * s
    return i


def ket_label(i: int, dims: Sequence[int]) -> str:
    """Ket string of basis index i.

    Reading: the printed label lists qudit 0 first.  The worked example of
    Sec. 3.9 (dims [2,3,3], F on qudit 0 then CX_{+2} from qudit 0 to 1)
    prints |120> for (x_0, x_1, x_2) = (1, 2, 0)."""
    return "|" + "".join(str(x) for x in decode(i, dims)) + ">"


def basis_state(dims: Sequence[int], levels: Sequence[int] | None = None) -> np.ndarray:
    """Product state |l_0 ... l_{n-1}> (Sec. 3.2 ``init_states``, default all 0)."""
    n = register_size(dims)
    psi = np.zeros(n, dtype=np.complex128)
    if levels is None:
        levels = [0] * len(dims)
    for l, d in zip(levels, dims):
        if not 0 <= l < d:
            raise ValueError("init level out of range")
    psi[encode(levels, dims)] = 1.0
    return psi


def product_state_kron(dims: Sequence[int], levels: Sequence[int] | None = None) -> np.ndarray:
    """The same product state built as the Kronecker product of per-qudit
    column vectors (Sec. 3.3, Eq. 2), in the LSB-first digit order: the
    Kronecker chain runs from the last qudit (most significant) to qudit 0."""
    if levels is None:
        levels = [0] * len(dims)
    v = np.ones(1, dtype=np.complex128)
    for d, l in zip(dims, levels):
        e = np.zeros(d, dtype=np.complex128)
        e[l] = 1.0
        v = np.kron(e, v)
    return v


# ---------------------------------------------------------------------------
# Gate definitions (Sec. 2.1.2)
# ---------------------------------------------------------------------------


def omega_power(d: int, m: int) -> complex:
    """w^m with w = exp(2 pi i / d) (Sec. 2.1.2, phase-shift gate).

    The exponent is reduced mod d first; quarter turns are returned exactly
    (1, i, -1, -i) so that Z_2 = diag(1, -1) and F_2 have no rounding in
    their zero parts."""
    m %= d
    if (4 * m) % d == 0:
        return [1.0 + 0j, 1j, -1.0 + 0j, -1j][(4 * m) // d]
    t = 2.0 * math.pi * m / d
    return complex(math.cos(t), math.sin(t))


def x_gate(d: int, a: int = 1) -> np.ndarray:
    """Generalized NOT X^d_{+a}: column x has its 1 in row (x+a) mod d (Sec. 2.1.2)."""
    if not 1 <= a <= d - 1:
        raise ValueError("shift a must satisfy 1 <= a <= d-1")
    m = np.zeros((d, d), dtype=np.complex128)
    for x in range(d):
        m[(x + a) % d, x] = 1.0
    return m


def z_gate(d: int, p: int = 1) -> np.ndarray:
    """Z_d^p = diag(w^{p j}) (Sec. 2.1.2; powers p != 1 are this build's
    extension, Z_d itself is p = 1)."""
    return np.diag([omega_power(d, p * j) for j in range(d)]).astype(np.complex128)


def f_gate(d: int) -> np.ndarray:
    """Generalized Hadamard F_d[j,k] = w^{jk} / sqrt(d) (Sec. 2.1.2)."""
    s = 1.0 / math.sqrt(d)
    return np.array([[omega_power(d, j * k) * s for k in range(d)] for j in range(d)],
                    dtype=np.complex128)


def controlled_matrix(ctrl_dims: Sequence[int], levels: Sequence[int], g: np.ndarray) -> np.ndarray:
    """Block-diagonal controlled gate on (controls..., targets...).

    The controls are the most significant local digits, listed first; the
    matrix is the identity except the diagonal block at the control
    combination ``levels``, which is ``g``.  With one control of dimension d
    at level d-1 this is C_{X,d} of Sec. 2.1.2 (X in the last block); with
    n-1 controls at d-1 it is the multi-controlled Toffoli C^n_{X,d}."""
    D = g.shape[0]
    C = register_size(ctrl_dims)
    m = np.eye(C * D, dtype=np.complex128)
    # local control index with the first control most significant
    c = 0
    for l, d in zip(levels, ctrl_dims):
        c = c * d + int(l)
    m[c * D:(c + 1) * D, c * D:(c + 1) * D] = g
    return m


def cx_matrix(dc: int, dt: int, a: int = 1, level: int | None = None) -> np.ndarray:
    """C_{X,d}: |x>|y> -> |x>|(y+a) mod d_t> iff x = level (default d_c - 1).

    Reading: the garbled text formula of Sec. 2.1.2 is read through its block
    matrix (X^d_{+a} in the last block) and the worked example, where a qubit
    control fires on |1>.  The control may have a dimension different from
    the target's (Fig. 2 caption, CX^3_{+2} with a qubit control)."""
    if level is None:
        level = dc - 1
    return controlled_matrix([dc], [level], x_gate(dt, a))


# ---------------------------------------------------------------------------
# Gate records -> (matrix over acting qudits, acting list)
# ---------------------------------------------------------------------------


def _levels(gate, dims):
    ctrls = list(getattr(gate, "controls", ()) or ())
    lv = getattr(gate, "levels", None)
    if lv is None:
        lv = [None] * len(ctrls)
    out = []
    for c, l in zip(ctrls, lv):
        out.append(dims[c] - 1 if (l is None or l < 0) else int(l))
    return ctrls, out


def target_matrix(gate, dims: Sequence[int]) -> np.ndarray:
    """The uncontrolled D x D matrix of a gate record over its targets.

    Gate records carry ``kind`` in {"X", "Z", "H", "U", "DIAG"}, ``targets``
    (first listed = most significant local digit), optional ``controls`` and
    ``levels``, ``param`` (X shift a or Z power p) and ``matrix`` (U: D x D;
    DIAG: the D diagonal entries)."""
    tg = list(gate.targets)
    kind = gate.kind
    if kind == "X":
        (t,) = tg
        return x_gate(dims[t], int(gate.param))
    if kind == "Z":
        (t,) = tg
        return z_gate(dims[t], int(gate.param))
    if kind == "H":
        (t,) = tg
        return f_gate(dims[t])
    D = register_size([dims[t] for t in tg])
    if kind == "U":
        m = np.asarray(gate.matrix, dtype=np.complex128).reshape(D, D)
        return m
    if kind == "DIAG":
        v = np.asarray(gate.matrix, dtype=np.complex128).reshape(D)
        return np.diag(v)
    raise ValueError(f"unknown gate kind {kind!r}")


def acting_matrix(gate, dims: Sequence[int]):
    """(matrix over controls+targets, acting list) for the dense mode."""
    g = target_matrix(gate, dims)
    ctrls, lv = _levels(gate, dims)
    if not ctrls:
        return g, list(gate.targets)
    return controlled_matrix([dims[c] for c in ctrls], lv, g), ctrls + list(gate.targets)


# ---------------------------------------------------------------------------
# Mode 1: dense Kronecker (the paper's own definition, Sec. 3.5-3.6)
# ---------------------------------------------------------------------------


def embed_single(dims: Sequence[int], q: int, g: np.ndarray) -> np.ndarray:
    """I (x) ... (x) G (x) ... (x) I with G on qudit q.

    With qudit 0 least significant, the Kronecker chain is written from the
    last qudit down to qudit 0 (np.kron(A, B) puts A's index in the more
    significant position)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for p in range(len(dims) - 1, -1, -1):
        f = g if p == q else np.eye(dims[p], dtype=np.complex128)
        m = np.kron(m, f)
    return m


def permutation_matrix(dims: Sequence[int], acting: Sequence[int]) -> np.ndarray:
    """Explicit permutation P with (P psi)[pi(i)] = psi[i], where pi moves the
    acting qudits, in the listed order (first = most significant), above all
    other qudits, which keep their relative order below them."""
    n = register_size(dims)
    rest = [q for q in range(len(dims)) if q not in acting]
    order_ls = rest + list(reversed(list(acting)))  # new digit order, LSB first
    new_dims = [dims[q] for q in order_ls]
    P = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        xs = decode(i, dims)
        j = encode([xs[q] for q in order_ls], new_dims)
        P[j, i] = 1.0
    return P


def full_unitary(dims: Sequence[int], g: np.ndarray, acting: Sequence[int]) -> np.ndarray:
    """U_full for a gate matrix over the acting qudits (first listed most
    significant): embed_single for one qudit, else P^T (G (x) I_rest) P."""
    acting = list(acting)
    if len(set(acting)) != len(acting):
        raise ValueError("acting qudits must be distinct")
    if len(acting) == 1:
        return embed_single(dims, acting[0], g)
    rest_n = register_size([dims[q] for q in range(len(dims)) if q not in acting])
    P = permutation_matrix(dims, acting)
    return P.T @ np.kron(g, np.eye(rest_n, dtype=np.complex128)) @ P


def dense_apply(psi: np.ndarray, dims: Sequence[int], gate) -> np.ndarray:
    g, acting = acting_matrix(gate, dims)
    return full_unitary(dims, g, acting) @ psi


# ---------------------------------------------------------------------------
# Mode 2: index loop
# ---------------------------------------------------------------------------


def local_offsets(dims: Sequence[int], targets: Sequence[int]) -> np.ndarray:
    """Flat offsets sum_t x_t s_t for every local index j of the targets,
    j = sum_m x_{t_m} prod_{m'>m} d_{t_{m'}} (first target most significant)."""
    s = strides(dims)
    offs = [0]
    for t in targets:
        offs = [o + x * s[t] for o in offs for x in range(dims[t])]
    return np.array(offs, dtype=np.int64)


def group_bases(dims: Sequence[int], targets: Sequence[int], controls: Sequence[int] = (),
                levels: Sequence[int] = ()) -> np.ndarray:
    """All basis indices whose target digits are 0 and whose control digits
    equal their levels: one per group of amplitudes the gate mixes."""
    n = register_size(dims)
    i = np.arange(n, dtype=np.int64)
    keep = np.ones(n, dtype=bool)
    s = strides(dims)
    for t in targets:
        keep &= (i // s[t]) % dims[t] == 0
    for c, l in zip(controls, levels):
        keep &= (i // s[c]) % dims[c] == l
    return i[keep]


def loop_apply(psi: np.ndarray, dims: Sequence[int], gate) -> np.ndarray:
    """Index-loop apply, vectorised over groups: gather the D amplitudes of
    every group, multiply by the D x D matrix in FP64, scatter back."""
    g = target_matrix(gate, dims)
    ctrls, lv = _levels(gate, dims)
    tg = list(gate.targets)
    _check_acting(dims, tg, ctrls, lv)
    bases = group_bases(dims, tg, ctrls, lv)
    offs = local_offsets(dims, tg)
    idx = bases[None, :] + offs[:, None]          # D x G
    out = psi.copy()
    out[idx] = g @ psi[idx]
    return out


def loop_apply_python(psi: np.ndarray, dims: Sequence[int], gate) -> np.ndarray:
    """Pure-Python index loop (tiny registers only): for every basis index,
    decode its digits; if it is a group base, gather, multiply, scatter."""
    g = target_matrix(gate, dims)
    ctrls, lv = _levels(gate, dims)
    tg = list(gate.targets)
    out = psi.copy()
    n = register_size(dims)
    D = g.shape[0]
    for i in range(n):
        xs = decode(i, dims)
        if any(xs[t] != 0 for t in tg):
            continue
        if any(xs[c] != l for c, l in zip(ctrls, lv)):
            continue
        members = []
        for j in range(D):
            # local digits of j, first target most significant
            rem, ys = j, list(xs)
            for t in reversed(tg):
                ys[t] = rem % dims[t]
                rem //= dims[t]
            members.append(encode(ys, dims))
        v = [psi[m] for m in members]
        for r in range(D):
            acc = 0j
            for c in range(D):
                acc += g[r, c] * v[c]
            out[members[r]] = acc
    return out


def _check_acting(dims, targets, controls, levels):
    n = len(dims)
    act = list(targets) + list(controls)
    if len(set(act)) != len(act) or any(not 0 <= q < n for q in act):
        raise ValueError("targets/controls must be distinct qudits of the register")
    for c, l in zip(controls, levels):
        if not 0 <= l < dims[c]:
            raise ValueError("control level out of range")


def run_circuit(dims: Sequence[int], gates: Iterable, init_levels=None, mode: str = "loop",
                psi0: np.ndarray | None = None) -> np.ndarray:
    """Evolve the initial product state through a gate list in the given mode.

    A record of kind "MEASURE" is the paper's Measurement Gate: it has no
    unitary, marks the end of the circuit, and every gate after it is ignored
    (Sec. 3.4, "Measurement Gate"; Sec. 3.6, measure_all)."""
    psi = basis_state(dims, init_levels) if psi0 is None else np.array(psi0, dtype=np.complex128)
    step = {"loop": loop_apply, "dense": dense_apply, "python": loop_apply_python}[mode]
    for g in gates:
        if getattr(g, "kind", None) == "MEASURE":
            break
        psi = step(psi, dims, g)
    return psi


# ---------------------------------------------------------------------------
# Readout (Sec. 3.8: probabilities or amplitudes of the basis states)
# ---------------------------------------------------------------------------


def norm2(psi: np.ndarray) -> float:
    """sum_i |psi_i|^2 in FP64 (Eq. 1 normalisation)."""
    return float(np.sum(psi.real * psi.real + psi.imag * psi.imag))


def probabilities(psi: np.ndarray) -> np.ndarray:
    """p_i = |psi_i|^2 in FP64."""
    return psi.real * psi.real + psi.imag * psi.imag


def marginal(psi: np.ndarray, dims: Sequence[int], q: int) -> np.ndarray:
    """P(x_q = v) for v < d_q: the measurement distribution of one qudit in
    the computational basis (Sec. 2.2)."""
    p = probabilities(psi)
    digit = (np.arange(len(p)) // strides(dims)[q]) % dims[q]
    return np.bincount(digit, weights=p, minlength=dims[q])


def cdf(psi: np.ndarray) -> np.ndarray:
    """Inclusive prefix sum of the probabilities, left to right."""
    return np.cumsum(probabilities(psi))


def sample_from_cdf(c: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Reading of measurement sampling: shot s returns the smallest index i
    with CDF_i > u_s * CDF_{N-1} (ties to the lower index)."""
    total = c[-1]
    return np.searchsorted(c, np.asarray(u, dtype=np.float64) * total, side="right")


def ket_dict(psi: np.ndarray, dims: Sequence[int], method: str = "amplitude",
             threshold: float = 1e-14) -> dict:
    """{ket label: value} of the basis states whose probability exceeds
    ``threshold`` (Sec. 3.8 OutputMethod: probability or amplitude)."""
    p = probabilities(psi)
    out = {}
    for i in np.nonzero(p > threshold)[0]:
        out[ket_label(int(i), dims)] = complex(psi[i]) if method == "amplitude" else float(p[i])
    return out


def fidelity(ref: np.ndarray, psi: np.ndarray, normalise: bool = False) -> float:
    """|<ref|psi>|^2 in FP64; optionally divided by both squared norms."""
    ref = np.asarray(ref, dtype=np.complex128)
    psi = np.asarray(psi, dtype=np.complex128)
    f = abs(np.vdot(ref, psi)) ** 2
    if normalise:
        f /= norm2(ref) * norm2(psi)
    return float(f)


# ---------------------------------------------------------------------------
# Counter-based generator for sampling: Philox4x64-10 (Salmon, Moraes, Dror,
# Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011)
# ---------------------------------------------------------------------------

_M64 = (1 << 64) - 1
_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox4x64(counter: Sequence[int], key: Sequence[int], rounds: int = 10) -> list[int]:
    """One Philox4x64 block: 10 rounds of two 64x64->128 multiplies with the
    published multipliers and Weyl key schedule."""
    c = [int(x) & _M64 for x in counter]
    k = [int(x) & _M64 for x in key]
    for _ in range(rounds):
        p0 = _PHILOX_M[0] * c[0]
        p1 = _PHILOX_M[1] * c[2]
        c = [(p1 >> 64) ^ c[1] ^ k[0], p1 & _M64, (p0 >> 64) ^ c[3] ^ k[1], p0 & _M64]
        k = [(k[0] + _PHILOX_W[0]) & _M64, (k[1] + _PHILOX_W[1]) & _M64]
    return c


def shot_uniforms(seed: int, shots: int) -> np.ndarray:
    """u_s in [0, 1) for shot s: the top 53 bits of word 0 of
    Philox4x64-10(counter=(s, 0, 0, 0), key=(seed, 0)), times 2^-53."""
    out = np.empty(shots, dtype=np.float64)
    for s in range(shots):
        w = philox4x64([s, 0, 0, 0], [seed, 0])[0]
        out[s] = (w >> 11) * (1.0 / 9007199254740992.0)
    return out


def sample(psi: np.ndarray, seed: int, shots: int) -> np.ndarray:
    return sample_from_cdf(cdf(psi), shot_uniforms(seed, shots))
