"""Pins of the MLP oracle: the analytic gradient equals central finite
differences in float64, and bf16 rounding matches the IEEE definition on
hand-picked values."""
import numpy as np

from oracle import mlp


def _params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, mlp.P)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(37, mlp.F))
    t = rng.normal(size=37)
    p = _params(1)
    g = mlp.gradient(p, x, t)
    eps = 1e-6
    idx = np.concatenate([np.arange(0, 40), rng.choice(mlp.P, 300, replace=False), [mlp.P - 1]])
    for i in idx:
        e = np.zeros(mlp.P)
        e[i] = eps
        fd = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_matches_explicit_loops():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4, mlp.F))
    p = _params(2)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    for s in range(4):
        h1 = [max(0.0, b1[o] + sum(W1[o, f] * x[s, f] for f in range(mlp.F))) for o in range(mlp.H)]
        h2 = [max(0.0, b2[o] + sum(W2[o, j] * h1[j] for j in range(mlp.H))) for o in range(mlp.H)]
        y = b3 + sum(w3[o] * h2[o] for o in range(mlp.H))
        assert abs(y - mlp.forward(p, x[s:s + 1])[0]) < 1e-9


def test_bf16_round():
    vals = np.array([1.0, 1.00390625, 1.005859375, -2.5, 3.0e-3, 65504.0], np.float32)
    got = mlp.bf16_round(vals)
    # 1.00390625 = 1 + 2^-8 is exactly halfway between bf16 1.0 and 1.0078125: ties to even -> 1.0
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0078125 and got[3] == -2.5
    assert abs(got[4] - 3.0e-3) < 3.0e-3 * 2 ** -8 and got[5] == 65536.0
