"""GPU parity of batched persistent execution (many independent circuits in
one launch) against the FP64 oracle, circuit by circuit.

Each circuit starts from |0...0> on its own register; the library returns the
complex64 amplitudes and the FP64 probabilities of every register.  Bars:
amplitudes <= 1e-5 max-abs and fidelity >= 1 - 1e-6 (the complex64 bar of the
per-gate kernels); probabilities <= 2e-5 max-abs, since
| |a|^2 - |b|^2 | <= (|a| + |b|) |a - b| <= 2 |a - b| for amplitudes of
modulus <= 1.
"""
import numpy as np
import pytest

from oracle import fast as qf
from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.workloads import Gate

pytestmark = pytest.mark.gpu

TOL64 = 1e-5
FID64 = 1 - 1e-6
TOLP = 2e-5
MIX = wl.C0_MIX + ("U2",)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def mixed_batch(seed, count, ngates, nmin=2, nmax=7, dims=(2, 3, 4, 5)):
    out = []
    for c in range(count):
        rng = np.random.default_rng(seed + c)
        n = int(rng.integers(nmin, nmax + 1))
        d = [int(x) for x in rng.choice(dims, size=n)]
        out.append((d, [wl.random_gate(rng, d, MIX) for _ in range(ngates)]))
    return out


def run_batch(circuits, tune=(), stream=0, runs=1):
    b = L.qd_batch_create([d for d, _ in circuits], stream)
    try:
        for key, val in tune:
            L.qd_batch_tune(b, key, val)
        for c, (_, gates) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, gates)
        for _ in range(runs):
            L.qd_batch_run(b)
        info = L.qd_batch_info(b, with_error=True)
        amps, probs = [], []
        for c, (d, _) in enumerate(circuits):
            N = int(np.prod(d))
            amps.append(L.qd_batch_get_amplitudes(b, c, N).astype(np.complex128))
            probs.append(L.qd_batch_probabilities(b, c, N))
        return amps, probs, info
    finally:
        L.qd_batch_destroy(b)


def check_circuit(dims, gates, psi, p):
    ref = qf.run_circuit(dims, gates)
    err = float(np.max(np.abs(psi - ref)))
    assert err <= TOL64, err
    assert qo.fidelity(ref, psi) >= FID64
    assert float(np.max(np.abs(p - qo.probabilities(ref)))) <= TOLP


# Register sizes span 4 .. 5^7 = 78,125 amplitudes: with the default limit of
# 6,144 amplitudes in shared memory, both whole-register items and tiled
# segments run.
@pytest.mark.parametrize("tune", [
    (),
    ((L.QD_BATCH_SMALL_AMPS, 0),),                                  # every circuit tiled
    ((L.QD_BATCH_SMALL_AMPS, 0), (L.QD_BATCH_TILE_AMPS, 100)),      # small tiles, one gate each
    ((L.QD_BATCH_SMALL_AMPS, 24576), (L.QD_BATCH_CTAS_PER_SM, 1)),  # mostly whole registers
    ((L.QD_BATCH_TILE_AMPS, 24576), (L.QD_BATCH_CTAS_PER_SM, 3)),   # largest tiles
    ((L.QD_BATCH_SMALL_AMPS, 0), (L.QD_BATCH_TILE_AMPS, 600), (L.QD_BATCH_TILES_PER_ITEM, 3),
     (L.QD_BATCH_GROUP_AMPS, 1)),                                    # several tiles per item, no groups
], ids=["default", "all_tiled", "tile100", "smem_1cta", "big_tiles", "multi_tile_items"])
def test_batch_vs_oracle(tune):
    circuits = mixed_batch(9100, 24, 40)
    amps, probs, info = run_batch(circuits, tune)
    assert info["device_error"] == 0
    for (d, g), psi, p in zip(circuits, amps, probs):
        check_circuit(d, g, psi, p)


def test_batch_long_circuits_many_chunks():
    # 300 gates on whole-register segments: each segment's descriptors span
    # several shared-memory chunks, loaded one after another
    circuits = mixed_batch(9300, 16, 300, nmin=3, nmax=6)
    for tune in ((), ((L.QD_BATCH_SMALL_AMPS, 0), (L.QD_BATCH_TILE_AMPS, 512), (L.QD_BATCH_TILES_PER_ITEM, 2))):
        amps, probs, info = run_batch(circuits, tune)
        assert info["device_error"] == 0
        for (d, g), psi, p in zip(circuits, amps, probs):
            check_circuit(d, g, psi, p)


def test_batch_long_circuit_precision():
    # 1000 gates, two thirds dense: the FP32 hi + lo coefficient split must
    # keep the norm (a lost lo part drifts it coherently by ~1.5e-9 per gate)
    mix = ("H", "U1", "U2", "X", "CX", "U1")
    circuits = []
    for c in range(6):
        rng = np.random.default_rng(9500 + c)
        d = [int(x) for x in rng.choice((2, 3, 4, 5), size=5)]
        circuits.append((d, [wl.random_gate(rng, d, mix) for _ in range(1000)]))
    for tune in ((), ((L.QD_BATCH_SMALL_AMPS, 0), (L.QD_BATCH_TILE_AMPS, 128))):
        amps, probs, info = run_batch(circuits, tune)
        assert info["device_error"] == 0
        for (d, g), psi, p in zip(circuits, amps, probs):
            assert abs(float(np.sum(p)) - 1.0) <= 1e-6
            check_circuit(d, g, psi, p)


def test_batch_autotune_keeps_results():
    circuits = mixed_batch(9400, 12, 40, nmin=4, nmax=9)
    b = L.qd_batch_create([d for d, _ in circuits])
    try:
        for c, (_, g) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, g)
        best = L.qd_batch_autotune(b, 1)
        assert best["tile_amps"] in (2048, 4096, 6144, 8192) and best["kernel_ms"] > 0
        L.qd_batch_run(b)
        assert L.qd_batch_info(b, with_error=True)["device_error"] == 0
        for c, (d, g) in enumerate(circuits):
            N = int(np.prod(d))
            check_circuit(d, g, L.qd_batch_get_amplitudes(b, c, N).astype(np.complex128),
                          L.qd_batch_probabilities(b, c, N))
    finally:
        L.qd_batch_destroy(b)


def test_batch_graph_replay_on_stream():
    torch = pytest.importorskip("torch")
    circuits = mixed_batch(9200, 12, 30, nmin=3, nmax=8)
    s = torch.cuda.Stream()
    amps1, probs1, info = run_batch(circuits, stream=s.cuda_stream, runs=1)
    amps3, probs3, info3 = run_batch(circuits, stream=s.cuda_stream, runs=3)
    assert info["device_error"] == 0 and info3["device_error"] == 0
    for (d, g), a1, a3, p1, p3 in zip(circuits, amps1, amps3, probs1, probs3):
        # every run restarts from |0...0>: replaying the graph changes nothing
        assert np.array_equal(a1, a3) and np.array_equal(p1, p3)
        check_circuit(d, g, a3, p3)


def test_batch_edge_cases():
    # empty circuits, a one-qudit register, a gate whose control level is
    # never occupied, and set_circuit replacing an earlier gate list
    circuits = [
        ([3, 2], []),
        ([5], [Gate("H", (0,))]),
        ([2, 3, 4], [Gate("X", (2,), (0,), (1,), 1)]),  # control qudit 0 stays at level 0
        ([4, 4, 4, 4, 4, 4, 4], [Gate("H", (q,)) for q in range(7)] + [Gate("Z", (3,), param=1)]),
    ]
    b = L.qd_batch_create([d for d, _ in circuits])
    try:
        L.qd_batch_set_circuit(b, 1, [Gate("X", (0,), param=2)])
        for c, (_, g) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, g)
        L.qd_batch_run(b)
        assert L.qd_batch_info(b, with_error=True)["device_error"] == 0
        for c, (d, g) in enumerate(circuits):
            N = int(np.prod(d))
            check_circuit(d, g, L.qd_batch_get_amplitudes(b, c, N).astype(np.complex128),
                          L.qd_batch_probabilities(b, c, N))
    finally:
        L.qd_batch_destroy(b)


def test_batch_rejections():
    with pytest.raises(L.QuditError) as e:
        L.qd_batch_create([[2] * 31])  # 2^31 amplitudes
    assert e.value.code == -2
    with pytest.raises(L.QuditError):
        L.qd_batch_create([[3, 1]])
    b = L.qd_batch_create([[6, 6], [2, 2], [64, 64, 8]])
    try:
        rng = np.random.default_rng(5)
        with pytest.raises(L.QuditError) as e:  # D = 36 > 25
            L.qd_batch_set_circuit(b, 0, [Gate("U", (0, 1), matrix=wl.haar_unitary(36, rng))])
        assert e.value.code == -2
        with pytest.raises(L.QuditError) as e:  # acting qudits span 32768 amplitudes
            L.qd_batch_set_circuit(b, 2, [Gate("X", (2,), (0, 1), (1, 1), 1)])
        assert e.value.code == -8
        with pytest.raises(L.QuditError):
            L.qd_batch_set_circuit(b, 3, [])
        with pytest.raises(L.QuditError):
            L.qd_batch_set_circuit(b, 1, [Gate("X", (0,), (0,), (1,), 1)])  # control == target
        with pytest.raises(L.QuditError):
            L.qd_batch_tune(b, 99, 1)
        with pytest.raises(L.QuditError):
            L.qd_batch_tune(b, L.QD_BATCH_TILE_AMPS, 1 << 20)
    finally:
        L.qd_batch_destroy(b)


def test_batch_c3_full():
    """The full batching workload (256 circuits, 6-12 qudits of dims 2..5,
    200 gates each, ~2.4e8 amplitudes in total): every register's FP64
    probabilities sum to 1, and every circuit of at most 2e5 amplitudes
    matches the oracle amplitude by amplitude."""
    circuits = wl.batch_c3()
    amps_needed = {c for c, (d, _) in enumerate(circuits) if int(np.prod(d)) <= 200_000}
    assert len(amps_needed) >= 16
    b = L.qd_batch_create([d for d, _ in circuits])
    try:
        for c, (_, g) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, g)
        L.qd_batch_run(b)
        info = L.qd_batch_info(b, with_error=True)
        assert info["device_error"] == 0
        assert info["total"] == sum(int(np.prod(d)) for d, _ in circuits)
        for c, (d, g) in enumerate(circuits):
            N = int(np.prod(d))
            p = L.qd_batch_probabilities(b, c, N)
            assert abs(float(np.sum(p)) - 1.0) <= 1e-5, (c, float(np.sum(p)))
            if c in amps_needed:
                check_circuit(d, g, L.qd_batch_get_amplitudes(b, c, N).astype(np.complex128), p)
    finally:
        L.qd_batch_destroy(b)


@pytest.mark.parametrize("stream_kind", ["legacy", "captured"])
def test_bounded_wait_expires_and_next_run_is_clean(stream_kind):
    """A work item of a later segment waits (bounded) on its circuit's
    completion counter.  With a poll limit of 0 every item whose segment
    dependencies are not complete at its first look gives up: it skips its
    tiles, the kernel still finishes, and the run reports error word 2 as
    QD_ERR_TIMEOUT.  Back at the default limit the next run is clean and its
    states match the oracle."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4242)
    dims = [3] * 12 + [2] * 2  # 2.1e6 amplitudes: thousands of 256-amplitude tiles per segment
    gates = []
    for a, b in [(0, 13), (6, 12), (3, 9), (1, 10), (2, 11), (4, 8), (5, 7), (0, 6)]:
        # two-qudit gates on far-apart qudits: with 256-amplitude tiles every
        # gate or two starts a new segment, whose items wait on the previous one
        gates.append(wl.Gate("U", (a, b), matrix=wl.haar_unitary(dims[a] * dims[b], rng)))
    circuits = [(dims, gates), ([2, 3, 2], [wl.Gate("H", (1,))])]
    stream = torch.cuda.Stream().cuda_stream if stream_kind == "captured" else 0
    b = L.qd_batch_create([d for d, _ in circuits], stream)
    try:
        L.qd_batch_tune(b, L.QD_BATCH_TILE_AMPS, 256)
        for c, (_, g) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, g)
        assert L.qd_batch_info(b)["items"] > 4 * (int(np.prod(dims)) // 256)  # several segments
        L.qd_batch_tune(b, L.QD_BATCH_POLL_LIMIT, 0)
        L.qd_batch_run(b)
        with pytest.raises(L.QuditError) as e:
            L.qd_batch_sync(b)
        assert e.value.code == -6 and e.value.device_error == 2
        assert L.qd_batch_info(b, with_error=True)["device_error"] == 2
        L.qd_batch_tune(b, L.QD_BATCH_POLL_LIMIT, 1 << 22)
        L.qd_batch_run(b)
        assert L.qd_batch_sync(b) == 0
        N = int(np.prod(dims))
        got = L.qd_batch_get_amplitudes(b, 0, N).astype(np.complex128)
    finally:
        L.qd_batch_destroy(b)
    ref = qf.run_circuit(dims, gates)
    assert np.max(np.abs(got - ref)) <= TOL64
    small = L.qd_batch_create([[2]], 0)
    try:
        with pytest.raises(L.QuditError):
            L.qd_batch_tune(small, L.QD_BATCH_POLL_LIMIT, -1)
    finally:
        L.qd_batch_destroy(small)
