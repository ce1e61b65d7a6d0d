"""Batched execution, host side (no GPU): the library's encoding of a batch
(segments of gates on shared-memory tiles, run tables, tile-local gate
geometry, work-queue order) replayed on the host in FP64 with the kernel's
index arithmetic, against the FP64 oracle circuit by circuit.

The replay also checks, item by item, that every item's dependencies are
queued before it (the persistent schedule cannot deadlock), that every tile
index stays inside its register, that each segment's tiles cover the
register exactly once, and that every gate index stays inside its tile.
"""
import numpy as np
import pytest

from oracle import fast as qf
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.workloads import Gate

MIX = wl.C0_MIX + ("U2",)
TOL = 1e-10  # FP64 replay; coefficients are FP32 hi + lo pairs (relative error ~2^-48)


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


def check(circuits, **tune):
    states, info = L.qd_debug_batch_emulate(circuits, **tune)
    assert info["errors"] == 0, info
    for (d, g), psi in zip(circuits, states):
        ref = qf.run_circuit(d, g)
        assert float(np.max(np.abs(psi - ref))) <= TOL
    return info


@pytest.mark.parametrize("tune", [
    {},
    {"small_amps": 0},
    {"small_amps": 0, "tile_amps": 100},
    {"small_amps": 0, "tile_amps": 25},
    {"small_amps": 24576},
    {"small_amps": 0, "tile_amps": 600, "tiles_per_item": 3},
    {"small_amps": 0, "group_amps": 1},
    {"small_amps": 0, "tile_amps": 24576, "group_amps": 1 << 30},
], ids=["default", "all_tiled", "tile100", "tile25", "all_smem", "3_tiles_per_item", "no_groups", "big_tiles"])
def test_replay_matches_oracle(tune):
    info = check(mixed_batch(4100, 20, 40, nmin=2, nmax=8), **tune)
    assert info["segments"] >= 20


def test_segments_cut_passes():
    # with tiles of a few qudits, a segment holds several gates: fewer passes
    circuits = mixed_batch(4200, 6, 60, nmin=7, nmax=8)
    info = check(circuits, small_amps=0, tile_amps=4096)
    assert info["segments"] < 6 * 60 / 2
    # a tile just big enough for one gate: one pass per gate (or fewer)
    info1 = check(circuits, small_amps=0, tile_amps=25)
    assert info["segments"] < info1["segments"] <= 6 * 60


def test_controls_and_odd_dims():
    # multi-controlled gates, non-default control levels, dims outside 2..5,
    # diagonal gates and a 3-qudit dense gate
    rng = np.random.default_rng(77)
    d = [3, 7, 2, 6, 2, 3]
    gates = [Gate("H", (1,)), Gate("H", (3,)), Gate("H", (0,)),
             Gate("X", (1,), (0, 2), (1, 1), 3),
             Gate("X", (5,), (1, 3, 4), (2, 5, 0), 2),
             Gate("U", (2, 4), (0,), (2,), matrix=wl.haar_unitary(4, rng)),
             Gate("U", (0, 2, 4), matrix=wl.haar_unitary(12, rng)),
             Gate("DIAG", (3,), matrix=np.exp(1j * rng.uniform(0, 6, 6))),
             Gate("Z", (1,), param=3), Gate("U", (1, 2), matrix=wl.haar_unitary(14, rng))]
    circuits = [(d, gates), ([5, 5], [Gate("U", (0, 1), matrix=wl.haar_unitary(25, rng))]), ([2], [])]
    for tune in ({}, {"small_amps": 0, "tile_amps": 64}, {"small_amps": 0, "tile_amps": 2000}):
        check(circuits, **tune)


def test_c3_encoding_covers_workload():
    """The full batching workload's encoding: no replay of the large
    circuits (too slow here), but every small one replayed and checked."""
    circuits = [c for c in wl.batch_c3() if int(np.prod(c[0])) <= 4000][:24]
    assert len(circuits) >= 10
    check(circuits)
    check(circuits, small_amps=0, tile_amps=512)


def test_rejections():
    with pytest.raises(L.QuditError):
        L.qd_debug_batch_emulate([([2] * 31, [])])
    rng = np.random.default_rng(3)
    with pytest.raises(L.QuditError):  # D = 36 > 25
        L.qd_debug_batch_emulate([([6, 6], [Gate("U", (0, 1), matrix=wl.haar_unitary(36, rng))])])
    with pytest.raises(L.QuditError):  # acting qudits span 64 * 64 * 8 > 24576 amplitudes
        L.qd_debug_batch_emulate([([64, 64, 8], [Gate("X", (2,), (0, 1), (1, 1), 1)])])
