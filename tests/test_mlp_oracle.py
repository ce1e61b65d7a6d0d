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
