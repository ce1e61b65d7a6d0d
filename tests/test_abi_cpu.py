"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every declared entry point, argument validation rejects bad input
before touching a device, and the planner's index arithmetic (replayed on the
host through qd_debug_gate_members) enumerates exactly the groups the oracle
defines."""
import os
import re

import numpy as np
import pytest

from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl
from paper_2211_07918_gb300.build import build
from paper_2211_07918_gb300.workloads import Gate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def _declared():
    names = set()
    for h in ("qudit.h", "qudit_debug.h"):
        with open(os.path.join(ROOT, "include", h)) as f:
            txt = f.read()
        names |= set(re.findall(r"^\s*(?:int|const char \*)\s*(qd_\w+)\(", txt, re.M))
    return names


def test_exports_every_declared_symbol():
    lib = L.load()
    names = _declared()
    assert len(names) >= 28
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers every declared call under the same name
    for n in names:
        assert hasattr(L, n), n


def test_strerror():
    assert L.qd_strerror(0) == "ok"
    assert "overlap" in L.qd_strerror(-3)


@pytest.mark.parametrize("dims,prec,code", [
    ([1, 3], L.QD_C64, -2), ([65], L.QD_C64, -2), ([3, 3], 7, -1), ([], L.QD_C64, -1),
    ([2] * 41, L.QD_C64, -2),
])
def test_create_rejects_bad_arguments(dims, prec, code):
    with pytest.raises(L.QuditError) as e:
        L.qd_create(dims, None, prec)
    assert e.value.code == code


def test_create_rejects_bad_init_level():
    with pytest.raises(L.QuditError) as e:
        L.qd_create([3, 3], [0, 3])
    assert e.value.code == -1


def test_null_register_is_rejected():
    with pytest.raises(L.QuditError) as e:
        L.qd_apply_h(0, 0)
    assert e.value.code == -1


# ---------------------------------------------------------------- planner

def _oracle_groups(dims, gate):
    ctrls, lv = qo._levels(gate, dims)
    bases = qo.group_bases(dims, list(gate.targets), ctrls, lv)
    offs = qo.local_offsets(dims, list(gate.targets))
    return {tuple(int(b + o) for o in offs) for b in bases}


def _check_gate(dims, gate, expect_mode=None, tile_stride=32):
    mem, info = L.qd_debug_gate_members(dims, gate, tile_stride=tile_stride)
    assert info["noop"] == 0
    got = {tuple(int(x) for x in row) for row in mem}
    assert len(got) == mem.shape[0]            # no group emitted twice
    assert got == _oracle_groups(dims, gate)   # exactly the oracle's groups, members in local order
    if expect_mode is not None:
        assert info["mode"] == expect_mode
    return info


@pytest.mark.parametrize("tile_stride", [0, 32, 1000])
@pytest.mark.parametrize("seed", range(40))
def test_planner_groups_match_oracle(seed, tile_stride):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    dims = [int(x) for x in rng.choice([2, 3, 4, 5, 7], size=n)]
    while qo.register_size(dims) > 20000:
        dims.pop()
    n = len(dims)
    k = int(rng.integers(1, min(3, n) + 1))
    acting = [int(x) for x in rng.choice(n, size=min(n, k + int(rng.integers(0, 3))), replace=False)]
    targets, controls = acting[:k], acting[k:]
    D = int(np.prod([dims[t] for t in targets]))
    if D > 32:
        targets = targets[:1]
        D = dims[targets[0]]
    levels = tuple(int(rng.integers(0, dims[c])) for c in controls)
    g = Gate("U", tuple(targets), tuple(controls), levels, matrix=wl.haar_unitary(D, rng))
    _check_gate(dims, g, tile_stride=tile_stride)


def test_direct_and_tile_modes_are_both_exercised():
    dims = [3] * 9
    # target stride 3^8 -> direct; target stride 1 -> tile
    rng = np.random.default_rng(0)
    u = wl.haar_unitary(3, rng)
    assert _check_gate(dims, Gate("U", (8,), matrix=u), expect_mode=0)["mode"] == 0
    assert _check_gate(dims, Gate("U", (0,), matrix=u), expect_mode=1)["mode"] == 1
    assert _check_gate(dims, Gate("U", (0,), matrix=u), expect_mode=0, tile_stride=0)["mode"] == 0
    # low control with high target also takes the tile path
    _check_gate(dims, Gate("X", (7,), (0,), (1,), 2), expect_mode=1)
    # a two-qudit gate spanning low and high qudits
    _check_gate(dims, Gate("U", (1, 6), matrix=wl.haar_unitary(9, rng)), expect_mode=1)
    _check_gate(dims, Gate("U", (6, 1), matrix=wl.haar_unitary(9, rng)), expect_mode=1)


def test_classification():
    dims = [3, 4, 5]
    _, i = L.qd_debug_gate_members(dims, Gate("X", (1,), param=1))
    assert i["kind"] == 1 and i["active"] == 0b1111
    _, i = L.qd_debug_gate_members(dims, Gate("Z", (2,), param=1))
    assert i["kind"] == 1 and i["active"] == 0b11110   # level 0 has lambda = 1
    _, i = L.qd_debug_gate_members(dims, Gate("H", (0,)))
    assert i["kind"] == 0
    _, i = L.qd_debug_gate_members(dims, Gate("U", (0,), matrix=np.eye(3)))
    assert i["noop"] == 1
    _, i = L.qd_debug_gate_members(dims, Gate("Z", (1,), param=4))  # Z_4^4 = I
    assert i["noop"] == 1


@pytest.mark.parametrize("gate,code", [
    (Gate("X", (0,), param=0), -1), (Gate("X", (0,), param=3), -1), (Gate("X", (0,), (0,), None, 1), -3),
    (Gate("U", (0, 0), matrix=np.eye(9)), -3), (Gate("X", (3,), param=1), -1),
    (Gate("X", (1,), (0,), (5,), 1), -1),
    (Gate("U", (1, 2), matrix=np.eye(48)), -2),
])
def test_gate_validation(gate, code):
    with pytest.raises(L.QuditError) as e:
        L.qd_debug_gate_members([3, 4, 12], gate)
    assert e.value.code == code
