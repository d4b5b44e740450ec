"""Pins of the reference MLP (learned lambda_0 predictor): gradients against central finite
differences, bfloat16 rounding against its definition."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(seed=3) * 0.5
    x = rng.normal(size=(7, mlp.NIN))
    y = rng.normal(size=7)
    L, g = mlp.loss_grad(theta, x, y)
    idx = rng.choice(mlp.NPARAM, size=40, replace=False)
    idx = np.concatenate([idx, [0, 8 * 256 + 3, mlp.NPARAM - 1, mlp.NPARAM - 2]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_grad(theta + e, x, y)[0] - mlp.loss_grad(theta - e, x, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 3 * 2.0 ** -8, -2.5, 3e-30])
    r = mlp.bf16(vals)
    # 8 significant bits: ties to even at 1 + 2^-8, round up just above the tie
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2.0 ** -7 and r[3] == 1.0 + 2.0 ** -6
    assert r[4] == -2.5
    assert abs(r[5] - 3e-30) / 3e-30 <= 2 ** -8


def test_pack_roundtrip():
    theta = mlp.init_params(seed=1)
    assert np.array_equal(mlp.pack(mlp.unpack(theta)), theta)
    assert theta.size == mlp.NPARAM == 8 * 256 + 256 + 256 * 256 + 256 + 256 + 1
