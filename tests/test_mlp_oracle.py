"""Pins of the FP64 reference network used to check the learned cost model's
kernels: back-propagated gradients equal central finite differences."""
import numpy as np
import pytest

from oracle import mlp_oracle as mo


@pytest.mark.parametrize("seed", range(3))
def test_backprop_equals_finite_differences(seed):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mo.NPARAM) * 0.3
    X = rng.standard_normal((17, mo.IN))
    t = rng.standard_normal(17)
    _, g = mo.grad(p, X, t)
    idx = rng.choice(mo.NPARAM, size=60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(mo.NPARAM)
        e[k] = h
        fd = (mo.loss(p + e, X, t) - mo.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8, (k, fd, g[k])


def test_parameter_count_matches_library_layout():
    assert mo.NPARAM == 9217


def test_planted_wrong_relu_derivative_is_caught(monkeypatch):
    # a backward pass that forgets the ReLU mask must disagree with the differences
    rng = np.random.default_rng(9)
    p = rng.standard_normal(mo.NPARAM) * 0.3
    X = rng.standard_normal((9, mo.IN))
    t = rng.standard_normal(9)
    w = mo.unpack(p)
    y, (Xc, z1, a1, z2, a2, z3, a3) = mo.forward(p, X)
    gy = 2.0 * (y - t) / len(t)
    d3_no_mask = np.outer(gy, w["W4"])
    gW3_bad = a2.T @ d3_no_mask
    _, g = mo.grad(p, X, t)
    o = mo.IN * mo.H + mo.H + mo.H * mo.H + mo.H
    assert np.max(np.abs(gW3_bad.reshape(-1) - g[o:o + mo.H * mo.H])) > 1e-6


# ---------------------------------------------------------------------------
# Pins of the forward pass that do not go through mo.forward: a hand-set
# network whose output is written down in closed form, and a per-neuron scalar
# loop (plain Python, no matrix products) on random networks.

def _hand_network():
    """W1 copies the 12 inputs into hidden units 0..11, b1 = 1/4 everywhere;
    W2 = 2 I, b2 = -1/2; W3 = I, b3 = +1 on unit 0 and -3 on unit 40 (a unit
    whose input is 0, so a missing ReLU on layer 3 would leak -3);
    W4[j] = j + 1; b4 = 1/8."""
    w = {name: np.zeros(shp) for name, shp in mo.SIZES}
    for i in range(mo.IN):
        w["W1"][i, i] = 1.0
    w["b1"][:] = 0.25
    w["W2"][:] = 2.0 * np.eye(mo.H)
    w["b2"][:] = -0.5
    w["W3"][:] = np.eye(mo.H)
    w["b3"][0] = 1.0
    w["b3"][40] = -3.0
    w["W4"][:] = np.arange(1, mo.H + 1, dtype=np.float64)
    w["b4"][0] = 0.125
    return np.concatenate([w[name].reshape(-1) for name, _ in mo.SIZES])


# Inputs and the closed-form output of the hand network, unit by unit:
#   layer 1: z1_j = x_j + 1/4 (j < 12), 1/4 (j >= 12); x_1 = -2 clips to 0.
#   layer 2: z2_j = 2 a1_j - 1/2; units 1 and 12..63 give -1/2 and clip to 0.
#   layer 3: a3_j = max(a2_j + b3_j, 0): unit 0 gains +1, unit 40 stays 0.
#   output:  y = sum_j (j + 1) a3_j + 1/8.
_X_HAND = np.array([1.0, -2.0, 3.0, 0.5, -0.125, 0.0, 2.0, -1.0, 0.75, 4.0, -0.25, 1.5])


def _closed_form_y(x):
    y = 0.125
    for j in range(mo.IN):
        a1 = max(x[j] + 0.25, 0.0)
        a2 = max(2.0 * a1 - 0.5, 0.0)
        a3 = a2 + (1.0 if j == 0 else 0.0)
        y += (j + 1) * max(a3, 0.0)
    return y


def test_closed_form_values_are_the_hand_computed_numbers():
    # the unit-by-unit formula above, evaluated by hand for _X_HAND:
    # a2 = [2, 0, 6, 1, 0, 0, 4, 0, 1.5, 8, 0, 3]; unit 0 adds 1 -> a3_0 = 3
    a3 = [3.0, 0, 6.0, 1.0, 0, 0, 4.0, 0, 1.5, 8.0, 0, 3.0]
    want = 0.125 + sum((j + 1) * v for j, v in enumerate(a3))
    assert want == 0.125 + 3 + 18 + 4 + 28 + 13.5 + 80 + 36
    assert _closed_form_y(_X_HAND) == want


def _check_forward_closed_form(forward):
    p = _hand_network()
    X = np.stack([_X_HAND, -_X_HAND, np.zeros(mo.IN)])
    y, _ = forward(p, X)
    want = np.array([_closed_form_y(x) for x in X])
    assert np.max(np.abs(np.asarray(y) - want)) <= 1e-12, (y, want)


def test_forward_matches_closed_form_network():
    _check_forward_closed_form(mo.forward)


def _scalar_forward(p, x):
    """The network one neuron at a time, with Python floats."""
    w = mo.unpack(p)
    a = [float(v) for v in x]
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        Wm, bv = w[W], w[b]
        a = [max(sum(a[i] * float(Wm[i, j]) for i in range(len(a))) + float(bv[j]), 0.0) for j in range(mo.H)]
    return sum(a[j] * float(w["W4"][j]) for j in range(mo.H)) + float(w["b4"][0])


@pytest.mark.parametrize("seed", range(2))
def test_forward_matches_scalar_loop(seed):
    rng = np.random.default_rng(100 + seed)
    p = rng.standard_normal(mo.NPARAM) * 0.4
    X = rng.standard_normal((5, mo.IN))
    y, _ = mo.forward(p, X)
    for n in range(len(X)):
        assert abs(y[n] - _scalar_forward(p, X[n])) <= 1e-12 * max(1.0, abs(y[n]))


def _forward_missing_relu3(p, X):
    w = mo.unpack(p)
    a1 = np.maximum(X @ w["W1"] + w["b1"], 0)
    a2 = np.maximum(a1 @ w["W2"] + w["b2"], 0)
    a3 = a2 @ w["W3"] + w["b3"]
    return a3 @ w["W4"] + w["b4"][0], None


def _forward_bias_twice(p, X):
    w = mo.unpack(p)
    a1 = np.maximum(X @ w["W1"] + 2 * w["b1"], 0)
    a2 = np.maximum(a1 @ w["W2"] + w["b2"], 0)
    a3 = np.maximum(a2 @ w["W3"] + w["b3"], 0)
    return a3 @ w["W4"] + w["b4"][0], None


@pytest.mark.parametrize("planted", [_forward_missing_relu3, _forward_bias_twice])
def test_planted_forward_mistakes_are_caught(planted):
    with pytest.raises(AssertionError):
        _check_forward_closed_form(planted)
