"""Pins of the FP64 oracle of the warm-start network (CPU)."""
import types

import numpy as np

from oracle import mlp_oracle as mo


def _problem(seed, T=24):
    rng = np.random.default_rng(seed)
    layers = []
    for i in range(4):
        q, p = mo.DIMS[i], mo.DIMS[i + 1]
        layers.append((rng.normal(0, np.sqrt(2.0 / q), (p, q)), rng.normal(0, 0.1, p)))
    theta = mo.pack(layers)
    x = np.zeros((T, 16))
    x[:, :4] = rng.normal(0, 1, (T, 4))
    target = rng.normal(0, 1, (T, 16))
    mask = (rng.random((T, 16)) < 0.7).astype(np.float64)
    return theta, x, target, mask


def _fd_check(module, seed=3, n=60, h=1e-4):
    theta, x, target, mask = _problem(seed)
    loss, g = module.loss_and_grad(theta, x, target, mask)
    rng = np.random.default_rng(seed + 100)
    idx = rng.choice(theta.size, size=n, replace=False)
    worst = 0.0
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (module.loss_and_grad(tp, x, target, mask)[0] - module.loss_and_grad(tm, x, target, mask)[0]) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / max(1e-8, abs(fd) + abs(g[i])))
    return worst


def test_pack_roundtrip():
    theta, *_ = _problem(1)
    assert np.array_equal(mo.pack(mo.unpack(theta)), theta)
    assert theta.size == sum(mo.DIMS[i] * mo.DIMS[i + 1] + mo.DIMS[i + 1] for i in range(4))


def test_gradient_matches_central_differences():
    assert _fd_check(mo) < 1e-6


def test_finite_differences_catch_a_dropped_relu_mask():
    src = open(mo.__file__).read()
    bad = src.replace("dz = dh * (h_prev > 0.0)", "dz = dh")
    assert bad != src
    mutant = types.ModuleType("mlp_mutant")
    exec(compile(bad, "mlp_mutant", "exec"), mutant.__dict__)
    assert _fd_check(mutant) > 1e-3


def test_single_active_path_closed_form():
    """One input feature routed through one unit per layer, everything else
    zero: out[0] = w4 * w3 * w2 * w1 * x (all factors positive), so the loss
    and its gradient with respect to each of the four weights are written out
    by hand."""
    layers = [(np.zeros((mo.DIMS[i + 1], mo.DIMS[i])), np.zeros(mo.DIMS[i + 1])) for i in range(4)]
    w = [0.7, 1.3, 0.9, 1.1]
    for i in range(4):
        layers[i][0][0, 0] = w[i]
    theta = mo.pack(layers)
    x = np.zeros((1, 16))
    x[0, 0] = 2.0
    target = np.zeros((1, 16))
    target[0, 0] = 1.0
    mask = np.zeros((1, 16))
    mask[0, 0] = 1.0
    loss, g = mo.loss_and_grad(theta, x, target, mask)
    prod = np.prod(w) * 2.0
    assert abs(loss - (prod - 1.0) ** 2) < 1e-12
    gl = mo.unpack(g)
    for i in range(4):
        expect = 2.0 * (prod - 1.0) * prod / w[i]
        assert abs(gl[i][0][0, 0] - expect) < 1e-9
        others = gl[i][0].copy()
        others[0, 0] = 0.0
        assert np.all(others == 0.0)
