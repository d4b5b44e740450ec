"""Reference MLP for the learned initial guess (test infrastructure; see ``oracle/__init__``).

Not in the paper: the learned lambda_0 predictor is one of the systems patterns of this
project.  Network: x (8) -> ReLU(x W1 + b1) (256) -> ReLU(h1 W2 + b2) (256) -> h2 W3 + b3 (1),
mean-squared-error loss L = mean((out - y)^2) / 2 ... computed here in FP64.

``bf16_points=True`` rounds the operands of the two 256-wide products (h1 and W2 in the
forward pass; the gradient d2 and W2, h1 and d2 in the backward pass) to bfloat16 with
round-to-nearest-even, which is where the GPU feeds its tensor cores; everything else stays
FP64.  Pinned by tests/test_oracle_mlp.py against central finite differences (FP64 mode), against
torch.nn layers with autograd (FP64) and, for the rounding, against torch's bfloat16 conversion.

Parameter vector layout (shared by both sides, as the ABI's flat parameter array):
W1 [8 x 256] row-major, b1 [256], W2 [256 x 256] row-major, b2 [256], W3 [256], b3 [1].
"""
import numpy as np

NIN, NH = 8, 256
SIZES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o: o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def bf16(a):
    """Round to bfloat16 (round to nearest even) and return as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, x, bf16_points=False):
    p = unpack(theta)
    q = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    z1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = q(h1) @ q(p["W2"]) + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"] + p["b3"][0]
    return out, (x, z1, h1, z2, h2)


def loss_grad(theta, x, y, bf16_points=False):
    """L = sum((out - y)^2) / (2 m) and its gradient with respect to theta."""
    p = unpack(theta)
    q = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    m = x.shape[0]
    out, (x, z1, h1, z2, h2) = forward(theta, x, bf16_points)
    d_out = (out - y) / m
    L = 0.5 * np.sum((out - y) ** 2) / m
    g = {"W3": h2.T @ d_out, "b3": np.array([d_out.sum()])}
    d2 = np.outer(d_out, p["W3"]) * (z2 > 0)
    g["W2"] = q(h1).T @ q(d2)
    g["b2"] = d2.sum(axis=0)
    d1 = (q(d2) @ q(p["W2"]).T) * (z1 > 0)
    g["W1"] = x.T @ d1
    g["b1"] = d1.sum(axis=0)
    return L, pack(g)


def init_params(seed=0):
    """He-uniform W1 and W2 from a counter-based SplitMix64 stream (same published definition
    as the library's: value i of stream seed -> uniform in (0, 1]); W3 and the biases zero."""
    from paper_2509_06673_gb300.workloads import uniform01
    u = uniform01(seed, np.arange(NPARAM, dtype=np.uint64))
    theta = np.zeros(NPARAM)
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name in ("W1", "W2"):
            fan_in = shape[0]
            lim = np.sqrt(6.0 / fan_in)
            theta[o: o + n] = (2.0 * u[o: o + n] - 1.0) * lim
        o += n
    return theta
