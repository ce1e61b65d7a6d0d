"""Parity at the full sizes the benchmark times (2^32 and 6.2e9 amplitudes),
where no oracle can hold the state: properties that hold at any size, on the
same kernels and plans the benchmark runs.  The per-gate paths they compare
against are pinned to the oracle amplitude by amplitude at smaller sizes
(tests/test_gpu_parity.py).

* QFT + Toffoli ladder on [2]*8 + [4]*12 (2^32 amplitudes): the fused
  complex64 plan chosen with the learned cost model against the per-gate
  complex128 path: fidelity >= 1 - 1e-6 and both norms within 1e-6 of 1.
* 1,000-gate circuit on [3]*18 + [2]*4 (6.2e9 amplitudes): the learned plan
  against per-gate complex64 kernels, same bars."""
import numpy as np
import pytest

from paper_2211_07918_gb300 import costmodel as cm
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def _run_plan(reg, gates, kind, model=None):
    if model is not None:
        L.qd_set_cost_model(reg, model)
    plan = L.qd_plan_create(reg, gates, kind)
    try:
        L.qd_plan_run(plan)
        assert L.qd_sync(reg) == 0
        return L.qd_plan_info(plan)
    finally:
        L.qd_plan_destroy(plan)


def test_qft_ladder_2_32_fused_vs_complex128():
    dims, gates = wl.circuit_c2()
    assert int(np.prod(dims)) == 2 ** 32
    model = cm.load()
    try:
        with L.Register(dims, None, L.QD_C64) as f, L.Register(dims, None, L.QD_C128) as r:
            info = _run_plan(f.h, gates, L.QD_PLAN_LEARNED, model)
            assert info["launches"] < len(gates)  # the plan fused some gates
            _run_plan(r.h, gates, L.QD_PLAN_NONE)
            ov = L.qd_overlap(r.h, f.h)
            assert abs(ov) ** 2 >= 1 - 1e-6
            assert abs(L.qd_norm(f.h) - 1.0) <= 1e-6
            assert abs(L.qd_norm(r.h) - 1.0) <= 1e-12
    finally:
        L.qd_model_destroy(model)


def test_learned_plan_6e9_vs_per_gate():
    dims, gates = wl.circuit_c4()
    assert int(np.prod(dims)) == 6_198_727_824
    model = cm.load()
    try:
        with L.Register(dims, None, L.QD_C64) as f, L.Register(dims, None, L.QD_C64) as r:
            _run_plan(f.h, gates, L.QD_PLAN_LEARNED, model)
            _run_plan(r.h, gates, L.QD_PLAN_NONE)
            ov = L.qd_overlap(r.h, f.h)
            assert abs(ov) ** 2 >= 1 - 1e-6
            assert abs(L.qd_norm(f.h) - 1.0) <= 1e-6
            assert abs(L.qd_norm(r.h) - 1.0) <= 1e-6
    finally:
        L.qd_model_destroy(model)


def _factor_circuit(dims, rng):
    """A Haar layer on every qudit, then 2-qudit gates (Haar, controlled
    shift, diagonal) on disjoint pairs, several of them on qudits whose
    strides exceed 2^31: the final state is a product of 1- and 2-qudit
    factors, so the oracle can give any amplitude exactly."""
    n = len(dims)
    gates = [wl.Gate("U", (q,), matrix=wl.haar_unitary(dims[q], rng)) for q in range(n)]
    pairs = [(n - 1, n - 2), (0, n - 3), (5, n - 5), (9, 3), (n - 4, 12)]
    for k, (a, b) in enumerate(pairs):
        if k % 3 == 0:
            gates.append(wl.Gate("U", (a, b), matrix=wl.haar_unitary(dims[a] * dims[b], rng)))
        elif k % 3 == 1:
            gates.append(wl.Gate("X", (b,), (a,), (int(rng.integers(0, dims[a])),), int(rng.integers(1, dims[b]))))
        else:
            gates.append(wl.Gate("DIAG", (a, b), matrix=np.exp(1j * rng.uniform(0, 6, dims[a] * dims[b]))))
    factors = [sorted(p) for p in pairs]
    paired = {q for p in pairs for q in p}
    factors += [[q] for q in range(n) if q not in paired]
    return gates, factors


def _factor_states(dims, gates, factors):
    """Oracle state of every factor (qudits ascending, as in the register)."""
    from oracle import fast as qf
    out = []
    for f in factors:
        pos = {q: i for i, q in enumerate(f)}
        sub = [wl.Gate(g.kind, tuple(pos[t] for t in g.targets), tuple(pos[c] for c in (g.controls or ())),
                       g.levels, g.param, g.matrix)
               for g in gates if set(g.targets) | set(g.controls or ()) <= set(f)]
        out.append(qf.run_circuit([dims[q] for q in f], sub))
    return out


def _amplitude(i, dims, factors, states):
    digits = []
    for d in dims:
        digits.append(i % d)
        i //= d
    amp = 1.0 + 0j
    for f, st in zip(factors, states):
        j, s = 0, 1
        for q in f:
            j += digits[q] * s
            s *= dims[q]
        amp *= st[j]
    return amp


@pytest.mark.parametrize("index64", [False, True])
@pytest.mark.parametrize("plan_kind", [L.QD_PLAN_NONE, L.QD_PLAN_GREEDY])
def test_sampled_amplitudes_2_32_vs_oracle(plan_kind, index64):
    """2^32 amplitudes (the QFT + ladder register: every dimension a power of
    two, so the gate kernels keep 32-bit indices up to 2^32 - 1; index64
    forces the 64-bit kernels) against the oracle on 4,096 sampled
    amplitudes of a product-of-factors state: the estimated squared error
    norm N * mean |psi_i - ref_i|^2 stays within the complex64 fidelity bar
    (1e-6)."""
    torch = pytest.importorskip("torch")
    dims, _ = wl.circuit_c2()
    N = int(np.prod(dims))
    rng = np.random.default_rng(2032)
    gates, factors = _factor_circuit(dims, rng)
    states = _factor_states(dims, gates, factors)
    buf = torch.zeros(N, dtype=torch.complex64, device="cuda")
    h = L.qd_create(dims, None, L.QD_C64, buf.data_ptr(), buf.numel() * 8, 0)
    try:
        if index64:
            L.qd_set_tuning(h, L.QD_TUNE_INDEX64, 1)
        plan = L.qd_plan_create(h, gates, plan_kind)
        L.qd_plan_run(plan)
        assert L.qd_sync(h) == 0
        L.qd_plan_destroy(plan)
        idx = np.unique(np.concatenate([rng.integers(0, N, size=4000, dtype=np.int64),
                                        [0, N - 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, N // 3]]))
        got = buf[torch.from_numpy(idx).to("cuda")].cpu().numpy().astype(np.complex128)
        ref = np.array([_amplitude(int(i), dims, factors, states) for i in idx])
        err2 = float(np.mean(np.abs(got - ref) ** 2)) * N
        assert err2 <= 1e-6, err2
        # the samples see the state (|a|^2 of a product state is heavy-tailed: a loose band)
        assert 0.2 <= float(np.mean(np.abs(ref) ** 2)) * N <= 5.0
    finally:
        L.qd_destroy(h)
        del buf
        torch.cuda.empty_cache()
