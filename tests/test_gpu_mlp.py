"""GPU checks of the learned cost model: the library's forward and backward
kernels against the FP64 reference network, training, and learned plans."""
import numpy as np
import pytest

from oracle import fast as qf
from oracle import mlp_oracle as mo
from oracle import qudit_oracle as qo
from paper_2211_07918_gb300 import qudit as L
from paper_2211_07918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_07918_gb300.build import build
    build()
    L.load()


@pytest.fixture()
def model():
    m = L.qd_model_create()
    yield m
    L.qd_model_destroy(m)


@pytest.mark.parametrize("n", [1, 31, 257])
def test_forward_and_gradient_match_fp64_reference(model, n):
    rng = np.random.default_rng(n)
    p = (rng.standard_normal(mo.NPARAM) * 0.2).astype(np.float32)
    L.qd_model_set(model, p)
    X = rng.standard_normal((n, mo.IN)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    y_ref, _ = mo.forward(p.astype(np.float64), X.astype(np.float64))
    y32 = L.qd_model_forward_raw(model, X)
    assert np.max(np.abs(y32 - y_ref)) <= 1e-4 * max(1.0, np.max(np.abs(y_ref)))
    y16 = L.qd_model_forward_raw(model, X, fp16=True)
    assert np.max(np.abs(y16 - y_ref)) <= 2e-2 * max(1.0, np.max(np.abs(y_ref)))
    loss, g = L.qd_model_grad_raw(model, X, t)
    loss_ref, g_ref = mo.grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, loss_ref)
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)


def test_training_fits_a_smooth_target(model):
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(4000, 12)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 3]).astype(np.float32)
    loss = L.qd_model_train(model, X, y, epochs=40, batch=128, lr=3e-3, seed=1)
    assert loss < 0.05  # normalised MSE
    pred = L.qd_model_predict(model, X[:500])
    assert np.sqrt(np.mean((pred - y[:500]) ** 2)) < 0.25 * np.std(y)


def test_learned_plan_is_correct(model):
    # any segmentation the learned planner picks must give the oracle's state
    rng = np.random.default_rng(2)
    L.qd_model_set(model, (rng.standard_normal(mo.NPARAM) * 0.1).astype(np.float32))
    dims = [3, 2, 4, 3, 2, 3]
    gates = wl.random_circuit(dims, 30, 11, wl.C0_MIX + ("U2",))
    ref = qf.run_circuit(dims, gates)
    for prec, tol in ((L.QD_C128, 1e-12), (L.QD_C64, 1e-5)):
        with L.Register(dims, None, prec) as r:
            L.qd_set_cost_model(r.h, model)
            plan = L.qd_plan_create(r.h, gates, L.QD_PLAN_LEARNED)
            L.qd_plan_run(plan)
            L.qd_plan_destroy(plan)
            psi = r.amplitudes().astype(np.complex128)
        assert np.max(np.abs(psi - ref)) <= tol


def test_segment_features_match_planner_features():
    dims = [3] * 6 + [2] * 3
    gates = wl.random_circuit(dims, 10, 3, wl.C0_MIX + ("U2",))
    with L.Register(dims, None, L.QD_C64) as r:
        f = L.qd_segment_features(r.h, gates, 0, 0)
    assert f[8] == pytest.approx(np.log2(qo.register_size(dims)), abs=1e-5)
    assert f[9] == 0.0
