"""CPU reference of the constraint-ordering network -- TEST INFRASTRUCTURE.

float64 numpy forward and backward of the 16 -> 64 -> 64 -> 1 ReLU
perceptron, with optional BF16 rounding (round to nearest, ties to even) at
exactly the points where the GPU kernels round: the input X, W1 and W2, the
first hidden activation before the second product, and the operands of the
backward products (dZ2, dZ1).  With quantize=False it is the plain
real-arithmetic network, which the tests pin against central finite
differences.
"""
import numpy as np

IN, HID = 16, 64
SIZES = [("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(x):
    """Round float values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, quantize=True):
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    P = unpack(p)
    xb = q(X)
    z1 = xb @ q(P["W1"]) + P["b1"]
    h1 = np.maximum(z1, 0.0)
    h1b = q(h1)
    z2 = h1b @ q(P["W2"]) + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (xb, z1, h1b, z2, h2)


def gradient(p, X, T, quantize=True):
    """Gradient of 0.5 * mean((y - T)^2) and the loss."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    P = unpack(p)
    y, (xb, z1, h1b, z2, h2) = forward(p, X, quantize)
    B = X.shape[0]
    dy = (y - T) / B
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = dy[:, None] * P["w3"][None, :] * (z2 > 0)
    dz2b = q(dz2)
    g["W2"] = h1b.T @ dz2b
    g["b2"] = dz2.sum(0)
    dz1 = (dz2b @ q(P["W2"]).T) * (z1 > 0)
    dz1b = q(dz1)
    g["W1"] = xb.T @ dz1b
    g["b1"] = dz1.sum(0)
    loss = 0.5 * np.mean((y - T) ** 2)
    return pack(g), loss
