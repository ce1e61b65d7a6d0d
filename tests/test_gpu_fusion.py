"""GPU parity of fused plans: the state after a greedy or exhaustive fused
plan equals the FP64 oracle's gate-by-gate result (complex128 <= 1e-12,
complex64 <= 1e-5 with fidelity >= 1 - 1e-6)."""
import numpy as np
import pytest

from oracle import fast as qf
from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def _run(dims, gates, prec, kind, psi0=None, kmax=None, dmax=None, tc_min_d=None, index64=False):
    with L.Register(dims, None, prec) as r:
        if index64:
            L.qd_set_tuning(r.h, L.QD_TUNE_INDEX64, 1)
        if tc_min_d:
            L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, tc_min_d)
        if kmax:
            L.qd_set_tuning(r.h, L.QD_TUNE_FUSE_KMAX, kmax)
        if dmax:
            L.qd_set_tuning(r.h, L.QD_TUNE_FUSE_DMAX, dmax)
        if psi0 is not None:
            L.qd_set_amplitudes(r.h, psi0)
        plan = L.qd_plan_create(r.h, gates, kind)
        info = L.qd_plan_info(plan)
        L.qd_plan_run(plan)
        L.qd_sync(r.h)
        L.qd_plan_destroy(plan)
        return r.amplitudes().astype(np.complex128), info


def _check(psi, ref, prec):
    err = np.max(np.abs(psi - ref))
    if prec == L.QD_C128:
        assert err <= 1e-12, err
    else:
        assert err <= 1e-5, err
        assert qo.fidelity(ref, psi) >= (1 - 1e-6) * qo.norm2(ref) ** 2


@pytest.mark.parametrize("kind", [L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE])
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_fused_c0(prec, kind):
    dims, gates = wl.circuit_c0()
    ref = qo.run_circuit(dims, gates, mode="dense")
    psi, info = _run(dims, gates, prec, kind)
    _check(psi, ref, prec)


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_fused_random(seed, prec):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(3, 9))
    dims = [int(x) for x in rng.choice([2, 3, 4, 5], size=n)]
    while qo.register_size(dims) > 50000:
        dims.pop()
    gates = wl.random_circuit(dims, 30, 900 + seed, wl.C0_MIX + ("U2",))
    gates = [g for g in gates if np.prod([dims[q] for q in g.targets]) <= 32]
    N = qo.register_size(dims)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    for kind in (L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE):
        psi, info = _run(dims, gates, prec, kind, psi0=psi0)
        _check(psi, ref, prec)
    # a larger fusion limit (4 qudits, D <= 32) exercises bigger blocks
    psi, info = _run(dims, gates, prec, L.QD_PLAN_GREEDY, psi0=psi0, kmax=4, dmax=32)
    _check(psi, ref, prec)


@pytest.fixture(scope="module")
def c1_ref():
    dims, gates = wl.circuit_c1()
    return dims, gates, qf.run_circuit(dims, gates)


@pytest.mark.parametrize("kind", [L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE])
@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_fused_c1_full_size(prec, kind, c1_ref):
    dims, gates, ref = c1_ref
    psi, info = _run(dims, gates, prec, kind)
    assert info["blocks"] > 0 and info["launches"] < len(gates)
    _check(psi, ref, prec)


def _kclasses(dims, gates, prec, kind, kmax=3, dmax=None, tc_min_d=None):
    with L.Register(dims, None, prec) as r:
        if tc_min_d:
            L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, tc_min_d)
        L.qd_set_tuning(r.h, L.QD_TUNE_FUSE_KMAX, kmax)
        if dmax:
            L.qd_set_tuning(r.h, L.QD_TUNE_FUSE_DMAX, dmax)
        plan = L.qd_plan_create(r.h, gates, kind)
        _, _, kc = L.qd_plan_timings(plan, with_times=False)
        L.qd_plan_destroy(plan)
    return [L.kclass_name(int(c)) for c in kc]


def test_tensor_block_d64():
    # two dense two-qudit gates on (0,1) and (1,2) of three ququarts fuse into
    # one D = 64 block, which runs on the tensor cores
    rng = np.random.default_rng(3)
    dims = [4, 4, 4, 2, 3]
    gates = [wl.Gate("U", (0, 1), matrix=wl.haar_unitary(16, rng)),
             wl.Gate("U", (2, 1), matrix=wl.haar_unitary(16, rng))]
    names = _kclasses(dims, gates, L.QD_C64, L.QD_PLAN_GREEDY, 3, 64)
    assert names == ["tensor_block_D64"], names
    N = qo.register_size(dims)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qo.run_circuit(dims, gates, psi0=psi0)
    psi, info = _run(dims, gates, L.QD_C64, L.QD_PLAN_GREEDY, psi0=psi0, kmax=3, dmax=64)
    assert info["blocks"] == 1
    _check(psi, ref, L.QD_C64)


@pytest.mark.parametrize("seed", range(8))
def test_tensor_blocks_random(seed):
    rng = np.random.default_rng(1200 + seed)
    n = int(rng.integers(4, 9))
    dims = [int(x) for x in rng.choice([2, 3, 4], size=n)]
    while qo.register_size(dims) > 200000:
        dims.pop()
    gates = wl.random_circuit(dims, 40, 1200 + seed, wl.C0_MIX + ("U2",))
    N = qo.register_size(dims)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    # default routing (the cost model picks per block), every block of D >= 9
    # on the tensor cores, and every block of D <= 32 on the CUDA cores
    for tc_min_d in (None, 9, 65):
        for kind in (L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE):
            psi, info = _run(dims, gates, L.QD_C64, kind, psi0=psi0, kmax=3, dmax=64, tc_min_d=tc_min_d)
            _check(psi, ref, L.QD_C64)


def test_block_routing_threshold():
    """Fused complex64 blocks below the threshold run on the CUDA-core dense
    kernels, at or above it on the tensor cores; above 32 always on the
    tensor cores; with threshold 0 the plan's cost model picks."""
    rng = np.random.default_rng(8)
    dims = [3, 3, 2, 4, 4, 4]
    g27 = [wl.Gate("U", (0,), matrix=wl.haar_unitary(3, rng)), wl.Gate("U", (1,), matrix=wl.haar_unitary(3, rng)),
           wl.Gate("U", (0, 2), matrix=wl.haar_unitary(6, rng))]  # qudits {0,1,2}: D = 18
    g64 = [wl.Gate("U", (3, 4), matrix=wl.haar_unitary(16, rng)), wl.Gate("U", (5, 4), matrix=wl.haar_unitary(16, rng))]
    segs = [(0, 2)]
    with L.Register(dims, None, L.QD_C64) as r:
        for tc, want18 in ((None, None), (9, "tensor_block_D18"), (19, "dense_direct_D18"),
                           (18, "tensor_block_D18"), (65, "dense_direct_D18"), (0, None)):
            if tc is not None:
                L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, tc)
            plan = L.qd_plan_create_segmented(r.h, g27, segs)
            names = [L.kclass_name(int(c)) for c in L.qd_plan_timings(plan, with_times=False)[2]]
            L.qd_plan_destroy(plan)
            if want18 is None:  # the cost model picks one of the two dense kernels
                assert names in (["tensor_block_D18"], ["dense_direct_D18"]), (tc, names)
            else:
                assert names == [want18], (tc, names)
            plan = L.qd_plan_create_segmented(r.h, g64, [(0, 1)])
            names = [L.kclass_name(int(c)) for c in L.qd_plan_timings(plan, with_times=False)[2]]
            L.qd_plan_destroy(plan)
            assert names == ["tensor_block_D64"], (tc, names)
        with pytest.raises(L.QuditError):
            L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, 8)
        with pytest.raises(L.QuditError):
            L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, -1)
        with pytest.raises(L.QuditError):
            L.qd_set_tuning(r.h, L.QD_TUNE_TC_MIN_D, 66)


@pytest.mark.parametrize("dims", [[4] * 13, [2] * 6 + [3] * 12])
def test_tensor_blocks_many_tiles_per_cta(dims):
    """Fused blocks on a register large enough that every CTA of the
    tensor-core kernel runs tens of tiles, so that each pipeline barrier goes
    through many phases: the fused complex64 state against the per-gate
    complex64 state (each already pinned to the oracle) on the device."""
    rng = np.random.default_rng(31)
    n = len(dims)
    gates = []
    for _ in range(24):
        qs = [int(x) for x in rng.choice(n, size=3, replace=False)]
        D = int(np.prod([dims[q] for q in qs]))
        if D > 64:
            qs = qs[:2]
            D = int(np.prod([dims[q] for q in qs]))
        a, b = qs[0], qs[1]
        gates.append(wl.Gate("U", (a, b), matrix=wl.haar_unitary(dims[a] * dims[b], rng)))
        if len(qs) == 3:
            c = qs[2]
            gates.append(wl.Gate("U", (b, c), matrix=wl.haar_unitary(dims[b] * dims[c], rng)))
    with L.Register(dims, None, L.QD_C64) as fused, L.Register(dims, None, L.QD_C64) as ref:
        L.qd_set_tuning(fused.h, L.QD_TUNE_TC_MIN_D, 9)  # every dense block of D >= 9 on the tensor cores
        plan = L.qd_plan_create(fused.h, gates, L.QD_PLAN_EXHAUSTIVE)
        classes = {L.kclass_name(int(c)) for c in L.qd_plan_timings(plan, with_times=False)[2]}
        L.qd_plan_run(plan)
        assert L.qd_sync(fused.h) == 0
        L.qd_plan_destroy(plan)
        L.qd_run_circuit(ref.h, gates, L.QD_PLAN_NONE)
        assert L.qd_sync(ref.h) == 0
        ov = L.qd_overlap(ref.h, fused.h)
        assert abs(ov) ** 2 >= 1 - 1e-6
        assert abs(L.qd_norm(fused.h) - 1.0) <= 1e-6
        assert any(c.startswith("tensor_block") for c in classes), classes


@pytest.mark.parametrize("kind", [L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE])
def test_fused_permutation_blocks_run_as_mono(kind):
    """A fused block of permutations with phases (shifts, clocks, controlled
    shifts) is itself one: in complex64 it runs on the mono kernel, also at
    D >= 9 where a dense block would go to the tensor cores."""
    rng = np.random.default_rng(404)
    dims = [3, 3, 2, 3, 3, 2, 3]
    gates = []
    for _ in range(60):
        t = int(rng.integers(0, len(dims)))
        sub = int(rng.integers(0, 3))
        if sub == 0:
            gates.append(wl.Gate("X", (t,), param=int(rng.integers(1, dims[t]))))
        elif sub == 1:
            gates.append(wl.Gate("Z", (t,), param=1))
        else:
            c = int(rng.choice([q for q in range(len(dims)) if q != t]))
            gates.append(wl.Gate("X", (t,), (c,), (int(rng.integers(0, dims[c])),), int(rng.integers(1, dims[t]))))
    ref = qf.run_circuit(dims, gates)
    psi, info = _run(dims, gates, L.QD_C64, kind, tc_min_d=9)
    _check(psi, ref, L.QD_C64)
    assert info["blocks"] > 0
    classes = _kclasses(dims, gates, L.QD_C64, kind, tc_min_d=9)
    assert not any(c.startswith("tensor_block") for c in classes), classes
    assert any(c.startswith("mono") and int(c.split("_D")[1]) >= 9 for c in classes), classes


def _diag_heavy_circuit(dims, ngates, seed):
    """Runs of diagonal gates (Z powers, random-phase diagonals on one or two
    qudits, controlled phases) between dense and permutation gates."""
    rng = np.random.default_rng(seed)
    n = len(dims)
    gates = []
    for _ in range(ngates):
        r = rng.random()
        if r < 0.12:
            q = int(rng.integers(0, n))
            gates.append(wl.Gate("U", (q,), matrix=wl.haar_unitary(dims[q], rng)))
        elif r < 0.18:
            q = int(rng.integers(0, n))
            gates.append(wl.Gate("X", (q,), param=int(rng.integers(1, dims[q]))))
        elif r < 0.4:
            q = int(rng.integers(0, n))
            gates.append(wl.Gate("Z", (q,), param=int(rng.integers(1, dims[q]))))
        elif r < 0.7:
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            D = dims[a] * dims[b]
            gates.append(wl.Gate("DIAG", (a, b), matrix=np.exp(2j * np.pi * rng.random(D))))
        else:
            c, t = (int(x) for x in rng.choice(n, size=2, replace=False))
            gates.append(wl.Gate("DIAG", (t,), (c,), (int(rng.integers(0, dims[c])),),
                                 matrix=np.exp(2j * np.pi * rng.random(dims[t]))))
    return gates


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
@pytest.mark.parametrize("case", ["qft", "diag0", "diag1"])
def test_diagonal_runs_match_oracle(prec, case):
    """Runs of consecutive diagonal gates beyond the block limits become one
    table launch each (covered range starting at qudit 0 included, tables of
    ragged mixed-radix size); the fused state equals the oracle's."""
    if case == "qft":
        dims, gates = wl.circuit_c2(n_qubits=3, n_ququarts=5)
    else:
        rng = np.random.default_rng(700 + int(case[-1]))
        dims = [int(x) for x in rng.choice([2, 3, 4, 5], size=7)]
        while qo.register_size(dims) > 40000:
            dims.pop()
        gates = _diag_heavy_circuit(dims, 60, 700 + int(case[-1]))
    N = qo.register_size(dims)
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    seen = set()
    for kind in (L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE):
        psi, info = _run(dims, gates, prec, kind, psi0=psi0, kmax=3, dmax=64 if prec == L.QD_C64 else 32)
        _check(psi, ref, prec)
        seen.update(c.split("_D")[0] for c in _kclasses(dims, gates, prec, kind, 3,
                                                      64 if prec == L.QD_C64 else 32))
    assert "diag_table" in seen or "dense_table" in seen, seen
    if case == "qft":  # F_d followed by its run of controlled phases: one launch
        assert "dense_table" in seen, seen


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
@pytest.mark.parametrize("dense", ["U1", "U2", "X"])
def test_dense_part_with_diagonal_run_explicit(prec, dense):
    """A dense gate (one or two qudits, or a permutation taken as dense)
    followed by diagonal gates spanning most of the register, planned as one
    explicit segment: one dense launch with the run's table as epilogue; the
    state equals the oracle's, on a table range that starts at qudit 0 and on
    one that starts higher up."""
    rng = np.random.default_rng(77)
    dims = [2, 3, 4, 3, 2, 4, 3]
    N = qo.register_size(dims)
    for lo in (0, 2):
        first = {"U1": wl.Gate("U", (3,), matrix=wl.haar_unitary(3, rng)),
                 "U2": wl.Gate("U", (3, 4), matrix=wl.haar_unitary(6, rng)),
                 "X": wl.Gate("X", (5,), param=3)}[dense]
        run = [wl.Gate("Z", (lo,), param=1),
               wl.Gate("DIAG", (6, lo + 1), matrix=np.exp(2j * np.pi * rng.random(dims[6] * dims[lo + 1]))),
               wl.Gate("DIAG", (4,), (lo,), (1,), matrix=np.exp(2j * np.pi * rng.random(dims[4]))),
               wl.Gate("Z", (5,), param=2)]
        gates = [first] + run
        psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        psi0 /= np.linalg.norm(psi0)
        ref = qo.run_circuit(dims, gates, psi0=psi0)
        with L.Register(dims, None, prec) as r:
            L.qd_set_amplitudes(r.h, psi0)
            plan = L.qd_plan_create_segmented(r.h, gates, [(0, len(gates) - 1)])
            names = [L.kclass_name(int(c)) for c in L.qd_plan_timings(plan, with_times=False)[2]]
            L.qd_plan_run(plan)
            L.qd_sync(r.h)
            L.qd_plan_destroy(plan)
            psi = r.amplitudes().astype(np.complex128)
        assert len(names) == 1 and names[0].startswith("dense_table"), names
        _check(psi, ref, prec)


@pytest.mark.parametrize("prec", [L.QD_C128, L.QD_C64])
def test_every_kernel_form_of_a_segment(prec):
    """One segment with several feasible forms (a dense gate on qudits 1, 2
    followed by diagonal gates on qudits 1..3: a fused block -- on either
    block kernel for complex64 -- or a dense part + run).  Each form, forced
    through qd_plan_create_forms, runs as that kernel class and gives the
    oracle's state; a form that is not feasible is refused."""
    rng = np.random.default_rng(91)
    dims = [2, 3, 3, 2, 4, 3]
    N = qo.register_size(dims)
    gates = [wl.Gate("U", (1, 2), matrix=wl.haar_unitary(9, rng)),
             wl.Gate("Z", (1,), param=1),
             wl.Gate("DIAG", (3,), (2,), (2,), matrix=np.exp(2j * np.pi * rng.random(2)))]
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qo.run_circuit(dims, gates, psi0=psi0)
    with L.Register(dims, None, prec) as r:
        forms = L.qd_segment_forms(r.h, gates, 0, len(gates) - 1)
        kinds = sorted(k for k, _ in forms)
        want = [L.QD_FORM_BLOCK] + ([L.QD_FORM_BLOCK_TC] if prec == L.QD_C64 else []) + [L.QD_FORM_DENSE_RUN]
        assert kinds == want, kinds
        feat = L.qd_segment_features(r.h, gates, 0, len(gates) - 1)
        assert int(feat[10]) in kinds
        # a count query (no arrays)
        import ctypes
        n = ctypes.c_int32(-1)
        ga = L.GateArray(gates)
        assert L.load().qd_segment_forms(ctypes.c_void_p(r.h), ga.ptr, ga.n, 0, len(gates) - 1, None, None, 0,
                                         ctypes.byref(n)) == 0
        assert n.value == len(forms)
        for k, f in forms:
            assert int(f[10]) == k
            L.qd_set_amplitudes(r.h, psi0)
            plan = L.qd_plan_create_segmented(r.h, gates, [(0, len(gates) - 1)], [k])
            names = [L.kclass_name(int(c)) for c in L.qd_plan_timings(plan, with_times=False)[2]]
            L.qd_plan_run(plan)
            L.qd_sync(r.h)
            L.qd_plan_destroy(plan)
            assert len(names) == 1, names
            _check(r.amplitudes().astype(np.complex128), ref, prec)
        with pytest.raises(L.QuditError):
            L.qd_plan_create_segmented(r.h, gates, [(0, len(gates) - 1)], [L.QD_FORM_DIAG_RUN])  # not all diagonal


@pytest.mark.parametrize("seed", range(6))
def test_fused_plans_on_64bit_index_kernels(seed):
    """Fused plans (blocks on both dense kernels, diagonal runs, dense parts
    with a run, mono blocks) with the 64-bit index kernels forced on small
    registers; even seeds use qubits and ququarts only (every stride a power
    of two, every division a shift), odd seeds dims 2..5.  Every amplitude
    against the oracle."""
    rng = np.random.default_rng(1500 + seed)
    n = int(rng.integers(5, 9))
    dims = [int(x) for x in rng.choice([2, 4] if seed % 2 == 0 else [2, 3, 4, 5], size=n)]
    while qo.register_size(dims) > 120000:
        dims.pop()
    gates = wl.random_circuit(dims, 40, 1500 + seed, wl.C0_MIX + ("U2",))
    gates += _diag_heavy_circuit(dims, 20, 1500 + seed)
    gates = [g for g in gates if np.prod([dims[q] for q in g.targets]) <= 32]
    N = qo.register_size(dims)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    for prec in (L.QD_C128, L.QD_C64):
        for kind in (L.QD_PLAN_NONE, L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE):
            for tc_min_d in ((None, 9, 65) if prec == L.QD_C64 and kind == L.QD_PLAN_EXHAUSTIVE else (None,)):
                psi, info = _run(dims, gates, prec, kind, psi0=psi0, kmax=3,
                                 dmax=64 if prec == L.QD_C64 else 32, tc_min_d=tc_min_d, index64=True)
                _check(psi, ref, prec)


def test_qft_runs_on_64bit_index_kernels():
    """The QFT + ladder shape (F_d followed by its run of controlled phases:
    dense part + run launches, tables from qudit 8 up) on 3 qubits + 5
    ququarts with the 64-bit index kernels forced."""
    dims, gates = wl.circuit_c2(n_qubits=3, n_ququarts=5)
    N = qo.register_size(dims)
    rng = np.random.default_rng(4)
    psi0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    psi0 /= np.linalg.norm(psi0)
    ref = qf.run_circuit(dims, gates, psi0=psi0)
    for prec in (L.QD_C128, L.QD_C64):
        for kind in (L.QD_PLAN_GREEDY, L.QD_PLAN_EXHAUSTIVE):
            psi, info = _run(dims, gates, prec, kind, psi0=psi0, kmax=3, dmax=64 if prec == L.QD_C64 else 32,
                             index64=True)
            _check(psi, ref, prec)
