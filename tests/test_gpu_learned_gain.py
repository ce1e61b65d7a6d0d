"""What the trained cost model gains: on evaluation circuits (10 active qudits of
dims 2..4, 40 gates, among spectator qudits so that the register holds
5e7-7e7 amplitudes), the plan chosen with the learned model runs faster on the
GPU than the greedy plan of the analytic model (the method without the
network).  Uses the weights trained on this GPU type and shipped with the
package."""
import os

import numpy as np
import pytest

from paper_2211_07918_gb300 import costmodel as cm
from paper_2211_07918_gb300 import qudit as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


def test_learned_plan_beats_greedy_plan():
    if not os.path.exists(cm.DEFAULT_WEIGHTS):
        pytest.skip("no trained weights shipped")
    m = cm.load()
    try:
        rows = cm.evaluate(m, n_circuits=2, seed=7002, measured=False, reps=5)
    finally:
        L.qd_model_destroy(m)
    learned = sum(r["learned"] for r in rows)
    greedy = sum(r["greedy"] for r in rows)
    per_gate = sum(r["per_gate"] for r in rows)
    assert learned < greedy, rows
    assert learned < per_gate, rows
