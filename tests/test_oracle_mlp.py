"""Pins of the reference MLP (learned lambda_0 predictor): gradients against central finite
differences, network, loss and gradient against torch.nn with autograd (FP64), bfloat16
rounding against its definition and against torch's conversion."""
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


def _torch_net(theta):
    import torch
    p = mlp.unpack(theta)
    net = torch.nn.Sequential(torch.nn.Linear(mlp.NIN, mlp.NH), torch.nn.ReLU(),
                              torch.nn.Linear(mlp.NH, mlp.NH), torch.nn.ReLU(),
                              torch.nn.Linear(mlp.NH, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"].T.copy()))
        net[0].bias.copy_(torch.from_numpy(p["b1"]))
        net[2].weight.copy_(torch.from_numpy(p["W2"].T.copy()))
        net[2].bias.copy_(torch.from_numpy(p["b2"]))
        net[4].weight.copy_(torch.from_numpy(p["W3"][None, :].copy()))
        net[4].bias.copy_(torch.from_numpy(p["b3"]))
    return net


def test_forward_loss_gradient_match_torch_autograd():
    """The network, the loss and its gradient against torch.nn layers with autograd in FP64
    (an implementation that shares nothing with the oracle's numpy code)."""
    import torch
    rng = np.random.default_rng(5)
    theta = mlp.init_params(seed=7)
    theta[-(mlp.NH + 1):] = rng.normal(size=mlp.NH + 1) * 0.1    # W3, b3 nonzero
    theta[mlp.NIN * mlp.NH: mlp.NIN * mlp.NH + mlp.NH] = rng.normal(size=mlp.NH) * 0.1   # b1
    x = rng.normal(size=(33, mlp.NIN))
    y = rng.normal(size=33)
    out, _ = mlp.forward(theta, x)
    L, g = mlp.loss_grad(theta, x, y)
    net = _torch_net(theta)
    tx, ty = torch.from_numpy(x), torch.from_numpy(y)
    tout = net(tx)[:, 0]
    tL = 0.5 * ((tout - ty) ** 2).mean()
    tL.backward()
    assert np.allclose(out, tout.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert abs(L - tL.item()) <= 1e-13 * abs(L)
    tg = mlp.pack({"W1": net[0].weight.grad.numpy().T, "b1": net[0].bias.grad.numpy(),
                   "W2": net[2].weight.grad.numpy().T, "b2": net[2].bias.grad.numpy(),
                   "W3": net[4].weight.grad.numpy()[0], "b3": net[4].bias.grad.numpy()})
    assert np.allclose(g, tg, rtol=1e-11, atol=1e-14)


def test_bf16_matches_torch_bfloat16():
    """Round to nearest even on bfloat16 against torch's float32 -> bfloat16 conversion,
    on random values and on exact ties."""
    import torch
    rng = np.random.default_rng(11)
    ties = 1.0 + (2 * np.arange(127) + 1) * 2.0 ** -8        # halfway between bf16 neighbours
    v = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-20, 20, size=4000),
                        ties, -ties * 2.0 ** 5])
    v = v.astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(v), ref)
