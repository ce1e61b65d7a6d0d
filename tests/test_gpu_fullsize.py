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
