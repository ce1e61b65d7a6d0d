"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: complex128 <= 1e-12 max-abs per amplitude; complex64 <= 1e-5
max-abs and fidelity >= 1 - 1e-6.  Integer results (sampled indices) are
exact except where u * total lands within rounding of a CDF boundary.
"""
import json
import os

import numpy as np
import pytest

from oracle import fast as qf
from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

TOL128 = 1e-12
TOL64 = 1e-5
FID64 = 1 - 1e-6
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def run_gpu(dims, gates, prec, init=None, psi0=None, plan=L.QD_PLAN_NONE, tile_stride=None, index64=False):
    with L.Register(dims, init, prec, tile_stride=tile_stride) as r:
        if index64:
            L.qd_set_tuning(r.h, L.QD_TUNE_INDEX64, 1)
        if psi0 is not None:
            L.qd_set_amplitudes(r.h, psi0)
        r.run(gates, plan)
        assert L.qd_sync(r.h) == 0
        return r.amplitudes().astype(np.complex128)


def check(psi, ref, prec):
    err = np.max(np.abs(psi - ref))
    if prec == L.QD_C128:
        assert err <= TOL128, err
    else:
        assert err <= TOL64, err
        assert qo.fidelity(ref, psi) >= FID64 * qo.norm2(ref) ** 2


def rand_state(rng, N):
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return v / np.sqrt(qo.norm2(v))


# --------------------------------------------------------------- paper example

@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_worked_example(prec):
    with open(os.path.join(GOLD, "worked_example.json")) as f:
        gold = json.load(f)
    dims = gold["dims"]
    gates = [Gate(g["kind"], tuple(g["targets"]), tuple(g.get("controls", ())), None, g.get("param", 0))
             for g in gold["gates"]]
    psi = run_gpu(dims, gates, prec, gold["init_levels"])
    kd = qo.ket_dict(psi, dims)
    assert set(kd) == set(gold["amplitudes"])
    tol = 1e-15 if prec == L.QD_C128 else 1e-7
    for k, v in gold["amplitudes"].items():
        assert abs(kd[k] - v) <= tol


def test_named_gate_calls():
    # qd_apply_h / qd_apply_cx / qd_apply_x / qd_apply_z / qd_apply_mct against the oracle
    dims = [2, 3, 4, 3]
    with L.Register(dims, None, L.QD_C128) as r:
        L.qd_apply_h(r.h, 0)
        L.qd_apply_h(r.h, 2)
        L.qd_apply_cx(r.h, 0, 1, 2)
        L.qd_apply_x(r.h, 3, 2)
        L.qd_apply_z(r.h, 2, 3)
        L.qd_apply_cx(r.h, 2, 3, 1, 1)
        L.qd_apply_mct(r.h, [0, 1], 3, 1, [1, 2])
        psi = r.amplitudes()
    gates = [Gate("H", (0,)), Gate("H", (2,)), Gate("X", (1,), (0,), None, 2), Gate("X", (3,), param=2),
             Gate("Z", (2,), param=3), Gate("X", (3,), (2,), (1,), 1), Gate("X", (3,), (0, 1), (1, 2), 1)]
    ref = qo.run_circuit(dims, gates, mode="dense")
    check(psi, ref, L.QD_C128)


# ------------------------------------------------------------------ C0 config

@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_c0_full_state_vs_dense_oracle(prec):
    dims, gates = wl.circuit_c0()
    ref = qo.run_circuit(dims, gates, mode="dense")
    psi = run_gpu(dims, gates, prec)
    check(psi, ref, prec)


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_c0_per_gate_and_norm(prec):
    dims, gates = wl.circuit_c0()
    ref = qo.basis_state(dims)
    with L.Register(dims, None, prec) as r:
        for g in gates:
            L.qd_apply_gate(r.h, g)
            ref = qo.loop_apply(ref, dims, g)
            psi = r.amplitudes().astype(np.complex128)
            check(psi, ref, prec)
            nrm = L.qd_norm(r.h)
            assert abs(nrm - 1.0) <= (1e-13 if prec == L.QD_C128 else 2e-6)


# ------------------------------------------------- random sweep of geometries

def _random_case(rng, nmax=8, Nmax=60000, pow2=False):
    n = int(rng.integers(1, nmax + 1))
    dims = ([int(x) for x in rng.choice([2, 4], size=n)] if pow2
            else [int(x) for x in rng.integers(2, 8, size=n)])
    while qo.register_size(dims) > Nmax:
        dims.pop()
    n = len(dims)
    gates = []
    for _ in range(16):
        k = int(rng.integers(1, min(3, n) + 1))
        acting = [int(x) for x in rng.choice(n, size=min(n, k + int(rng.integers(0, 3))), replace=False)]
        t, c = acting[:k], acting[k:]
        D = int(np.prod([dims[q] for q in t]))
        while D > 32:
            t = t[:-1]
            D = int(np.prod([dims[q] for q in t]))
        lv = tuple(int(rng.integers(0, dims[q])) for q in c)
        kind = rng.integers(0, 5)
        if kind == 0:
            g = Gate("U", tuple(t), tuple(c), lv, matrix=wl.haar_unitary(D, rng))
        elif kind == 1:
            g = Gate("DIAG", tuple(t), tuple(c), lv, matrix=np.exp(2j * np.pi * rng.random(D)))
        elif kind == 2:
            g = Gate("X", (t[0],), tuple(c), lv, int(rng.integers(1, dims[t[0]])))
        elif kind == 3:
            g = Gate("H", (t[0],), tuple(c), lv)
        else:
            perm = rng.permutation(D)
            m = np.zeros((D, D), complex)
            m[np.arange(D), perm] = np.exp(2j * np.pi * rng.random(D))
            g = Gate("U", tuple(t), tuple(c), lv, matrix=m)
        gates.append(g)
    return dims, gates


@pytest.mark.parametrize("tile_stride", [0, 32, 100000])
@pytest.mark.parametrize("seed", range(24))
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_random_geometry_sweep(seed, prec, tile_stride):
    rng = np.random.default_rng(500 + seed)
    dims, gates = _random_case(rng)
    psi0 = rand_state(rng, qo.register_size(dims))
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    psi = run_gpu(dims, gates, prec, psi0=psi0, tile_stride=tile_stride)
    check(psi, ref, prec)


@pytest.mark.parametrize("tile_stride", [0, 32])
@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_random_geometry_sweep_index64(seed, prec, tile_stride):
    """The 64-bit index kernels (those of registers of >= 2^31 amplitudes,
    power-of-two divisors as shifts) forced on small registers, so that
    every amplitude is compared with the oracle; seeds 700+ draw dims in
    {2, 4} half of the time (all strides powers of two)."""
    rng = np.random.default_rng(700 + seed)
    dims, gates = _random_case(rng, pow2=seed % 2 == 0)
    psi0 = rand_state(rng, qo.register_size(dims))
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    psi = run_gpu(dims, gates, prec, psi0=psi0, tile_stride=tile_stride, index64=True)
    check(psi, ref, prec)


@pytest.mark.parametrize("index64", [False, True])
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_dense_gates_on_the_lowest_qudits(prec, index64):
    """Dense gates whose group is D consecutive amplitudes (targets = the
    lowest qudits, in any listed order, D even: the complex64 kernels move
    16-byte amplitude pairs) with and without controls above them; every
    amplitude against the oracle."""
    rng = np.random.default_rng(61)
    dims = [2, 4, 2, 3, 2, 5, 2]
    N = qo.register_size(dims)
    gates = []
    for t in [(0,), (1, 0), (0, 1), (2, 1, 0), (1, 2, 0), (0, 2, 1)]:
        D = int(np.prod([dims[q] for q in t]))
        gates.append(Gate("U", t, matrix=wl.haar_unitary(D, rng)))
        gates.append(Gate("U", t, (4, 5), (1, 3), matrix=wl.haar_unitary(D, rng)))
    gates.append(Gate("U", (1,), matrix=wl.haar_unitary(4, rng)))       # stride 2: not contiguous
    gates.append(Gate("U", (0, 2), matrix=wl.haar_unitary(4, rng)))     # offsets 0, 1, 8, 9
    psi0 = rand_state(rng, N)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    psi = run_gpu(dims, gates, prec, psi0=psi0, index64=index64)
    check(psi, ref, prec)


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_controlled_leaves_other_levels_bit_identical(prec):
    rng = np.random.default_rng(9)
    dims = [3, 2, 5, 3, 4, 3]
    N = qo.register_size(dims)
    psi0 = rand_state(rng, N)
    dt = np.complex128 if prec == L.QD_C128 else np.complex64
    for c, t in [(0, 4), (4, 0), (3, 1), (5, 2)]:
        lvl = int(rng.integers(0, dims[c]))
        g = Gate("U", (t,), (c,), (lvl,), matrix=wl.haar_unitary(dims[t], rng))
        with L.Register(dims, None, prec) as r:
            L.qd_set_amplitudes(r.h, psi0.astype(dt))
            before = r.amplitudes().copy()
            L.qd_apply_gate(r.h, g)
            after = r.amplitudes()
        digit = (np.arange(N) // qo.strides(dims)[c]) % dims[c]
        assert np.array_equal(after[digit != lvl].view(np.uint8), before[digit != lvl].view(np.uint8))
        check(after.astype(np.complex128), qo.loop_apply(before.astype(np.complex128), dims, g), prec)


@pytest.mark.parametrize("tile_stride", [0, 32])
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_large_dims_and_three_targets(prec, tile_stride):
    rng = np.random.default_rng(21)
    dims = [31, 2, 17, 3]
    N = qo.register_size(dims)
    psi0 = rand_state(rng, N)
    gates = [Gate("U", (0,), matrix=wl.haar_unitary(31, rng)),
             Gate("U", (2,), (0,), (30,), matrix=wl.haar_unitary(17, rng)),
             Gate("U", (1, 3), matrix=wl.haar_unitary(6, rng)),
             Gate("H", (3,), (0, 2), (3, 16)),
             Gate("U", (3, 1), (2,), (5,), matrix=wl.haar_unitary(6, rng))]
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    check(run_gpu(dims, gates, prec, psi0=psi0, tile_stride=tile_stride), ref, prec)


def test_single_qudit_register_and_d64():
    for d in (2, 7, 32):
        rng = np.random.default_rng(d)
        u = wl.haar_unitary(d, rng)
        g = [Gate("U", (0,), matrix=u)]
        psi0 = rand_state(rng, d)
        check(run_gpu([d], g, L.QD_C128, psi0=psi0), qo.loop_apply(psi0, [d], g[0]), L.QD_C128)
    # a d=64 qudit can be held and measured; a one-qudit gate on it exceeds QD_MAX_D
    with L.Register([64, 2], [63, 1], L.QD_C64) as r:
        p = L.qd_probabilities(r.h)
        assert p[63 + 64] == 1.0
        with pytest.raises(L.QuditError) as e:
            L.qd_apply_h(r.h, 0)
        assert e.value.code == -2


def test_identity_gate_is_noop():
    dims = [3, 3]
    with L.Register(dims, [1, 2], L.QD_C128) as r:
        L.qd_apply(r.h, np.eye(3), [0])
        L.qd_apply_z(r.h, 1, 3)   # Z_3^3 = I
        psi = r.amplitudes()
    assert psi[1 + 2 * 3] == 1.0 and np.count_nonzero(psi) == 1


# ----------------------------------------------------------------- C1 config

@pytest.fixture(scope="module")
def c1_reference():
    dims, gates = wl.circuit_c1()
    return dims, gates, qf.run_circuit(dims, gates)


@pytest.mark.parametrize("tile_stride", [0, 32])
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_c1_full_size(prec, tile_stride, c1_reference):
    dims, gates, ref = c1_reference
    psi = run_gpu(dims, gates, prec, tile_stride=tile_stride)
    check(psi, ref, prec)


# ------------------------------------------------------------------ readouts

@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_readouts(prec):
    rng = np.random.default_rng(3)
    dims = [3, 4, 2, 5, 3, 7, 3]
    N = qo.register_size(dims)
    psi0 = rand_state(rng, N) * 1.3
    dt = np.complex128 if prec == L.QD_C128 else np.complex64
    psi0 = psi0.astype(dt)
    ref = psi0.astype(np.complex128)
    with L.Register(dims, None, prec) as r:
        L.qd_set_amplitudes(r.h, psi0)
        assert abs(L.qd_norm(r.h) - qo.norm2(ref)) <= 1e-13
        p = L.qd_probabilities(r.h)
        assert np.max(np.abs(p - qo.probabilities(ref))) <= 1e-15
        for q in range(len(dims)):
            m = L.qd_marginal(r.h, q, dims[q])
            assert np.max(np.abs(m - qo.marginal(ref, dims, q))) <= 1e-13
        c = L.qd_cdf(r.h)
        assert np.max(np.abs(c - qo.cdf(ref))) <= 1e-12
        u = np.concatenate([rng.random(5000), [0.0, 0.5, 0.999999999]])
        s = L.qd_sample_u(r.h, u)
        s2 = L.qd_sample(r.h, 1234, 4000)
    want = qo.sample_from_cdf(qo.cdf(ref), u)
    _check_samples(s, want, u, qo.cdf(ref))
    u2 = qo.shot_uniforms(1234, 4000)
    _check_samples(s2, qo.sample_from_cdf(qo.cdf(ref), u2), u2, qo.cdf(ref))


def _check_samples(got, want, u, cdf):
    bad = np.nonzero(got != want)[0]
    total = cdf[-1]
    for i in bad:
        # a mismatch is allowed only where u*total is within rounding of the boundary
        t = u[i] * total
        b = cdf[min(got[i], want[i])]
        assert abs(t - b) <= 1e-12 * total, (i, got[i], want[i])
    assert len(bad) <= max(1, len(u) // 1000)


@pytest.mark.parametrize("pa,pb", [(L.QD_C64, L.QD_C128), (L.QD_C128, L.QD_C128), (L.QD_C64, L.QD_C64)])
def test_overlap(pa, pb):
    rng = np.random.default_rng(8)
    dims = [3, 5, 4, 7]
    N = qo.register_size(dims)
    a = rand_state(rng, N)
    b = rand_state(rng, N)
    with L.Register(dims, None, pa) as ra, L.Register(dims, None, pb) as rb:
        L.qd_set_amplitudes(ra.h, a)
        L.qd_set_amplitudes(rb.h, b)
        got = L.qd_overlap(ra.h, rb.h)
        aa = ra.amplitudes().astype(np.complex128)
        bb = rb.amplitudes().astype(np.complex128)
    assert abs(got - np.vdot(aa, bb)) <= 1e-13


def test_reset_and_torch_buffer():
    torch = pytest.importorskip("torch")
    dims = [3, 5, 2]
    N = 30
    buf = torch.zeros(N, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    h = L.qd_create(dims, [2, 1, 1], L.QD_C64, buf.data_ptr(), buf.numel() * 8, stream)
    try:
        L.qd_sync(h)
        idx = 2 + 1 * 3 + 1 * 15
        assert buf[idx].item() == 1 and int((buf != 0).sum()) == 1
        L.qd_apply_h(h, 1)
        L.qd_reset(h, [0, 0, 0])
        L.qd_sync(h)
        assert buf[0].item() == 1 and int((buf != 0).sum()) == 1
    finally:
        L.qd_destroy(h)


def test_plan_reuse_matches_single_run():
    dims, gates = wl.circuit_c0(seed=5)
    with L.Register(dims, None, L.QD_C128) as r:
        plan = L.qd_plan_create(r.h, gates)
        info = L.qd_plan_info(plan)
        assert 0 < info["launches"] <= len(gates)
        L.qd_plan_run(plan)
        L.qd_reset(r.h)
        L.qd_plan_run(plan)
        L.qd_plan_destroy(plan)
        psi = r.amplitudes()
    check(psi, qo.run_circuit(dims, gates, mode="dense"), L.QD_C128)
