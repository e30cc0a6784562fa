"""Pins of the FP64 reference MLP: parameter count, and gradients against central finite
differences of its own loss (so a wrong transpose, a dropped SiLU derivative or a missing
1/n fails here before any GPU comparison)."""
import numpy as np

from oracle import mlp


def _net(seed=3):
    rng = np.random.default_rng(seed)
    flat = np.empty(mlp.N_PARAMS)
    off = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        fan_in = shape[0] if len(shape) == 2 else 256
        flat[off:off + n] = rng.uniform(-1, 1, n) / np.sqrt(fan_in) * (0.3 if name[0] == "b" else 1)
        off += n
    x = rng.uniform(-1, 1, (9, 4))
    t = np.zeros((9, 8))
    t[:, 0] = rng.integers(0, 2, 9)
    t[:, 1:4] = rng.normal(size=(9, 3))
    t[:, 4] = rng.integers(0, 2, 9)
    t[:, 5] = rng.integers(0, 2, 9)
    return flat, x, t


def test_parameter_count_matches_the_architecture():
    assert mlp.N_PARAMS == 199684


def test_gradients_match_finite_differences():
    flat, x, t = _net()
    g = mlp.gradients(flat, x, t)
    rng = np.random.default_rng(5)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    idx = np.concatenate([rng.integers(offs[k], offs[k + 1], 4) for k in range(len(mlp.SHAPES))])
    for i in idx:
        e = np.zeros_like(flat)
        h = 1e-6
        e[i] = h
        fd = (mlp.loss(flat + e, x, t) - mlp.loss(flat - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_zero_masks_remove_regression_terms():
    flat, x, t = _net()
    t2 = t.copy()
    t2[:, 4:6] = 0
    t3 = t2.copy()
    t3[:, 1:4] += 100.0
    assert mlp.loss(flat, x, t2) == mlp.loss(flat, x, t3)
