"""FP64 reference of the learned cost model's network (TEST INFRASTRUCTURE ONLY).

A multilayer perceptron 12 -> 64 -> 64 -> 64 -> 1 with ReLU hidden units and
a mean-squared-error loss, written out with numpy in FP64, with the same flat
parameter layout as the library: W1 (12x64, row = input), b1, W2 (64x64), b2,
W3 (64x64), b3, W4 (64), b4.  Gradients by the chain rule.  Pinned in the
tests without going through this module's own arithmetic: the forward pass by
a hand-set network whose output is written down in closed form (with a
negative pre-activation on every layer that must clip) and by a per-neuron
scalar loop; the gradients by central finite differences of that pinned
forward pass.  The paper has no learned component; this is
the checker of the library's own forward and backward kernels.
"""
from __future__ import annotations

import numpy as np

IN, H = 12, 64
SIZES = [("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("W4", (H,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp)
        o += n
    return out


def forward(p, X):
    """y[n] and the cached pre-activations."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"] + w["b1"]
    a1 = np.maximum(z1, 0)
    z2 = a1 @ w["W2"] + w["b2"]
    a2 = np.maximum(z2, 0)
    z3 = a2 @ w["W3"] + w["b3"]
    a3 = np.maximum(z3, 0)
    y = a3 @ w["W4"] + w["b4"][0]
    return y, (X, z1, a1, z2, a2, z3, a3)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, X, t):
    """(loss, dloss/dp) of the mean squared error, by back-propagation."""
    w = unpack(p)
    y, (X, z1, a1, z2, a2, z3, a3) = forward(p, X)
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    gy = 2.0 * (y - t) / n
    g = {}
    g["W4"] = a3.T @ gy
    g["b4"] = np.array([gy.sum()])
    d3 = np.outer(gy, w["W4"]) * (z3 > 0)
    g["W3"] = a2.T @ d3
    g["b3"] = d3.sum(0)
    d2 = (d3 @ w["W3"].T) * (z2 > 0)
    g["W2"] = a1.T @ d2
    g["b2"] = d2.sum(0)
    d1 = (d2 @ w["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ d1
    g["b1"] = d1.sum(0)
    flat = np.concatenate([g[name].reshape(-1) for name, _ in SIZES])
    return float(np.mean((y - t) ** 2)), flat
