"""Plain float64 reference of the depth-predictor MLP (numpy).

TEST INFRASTRUCTURE ONLY (see oracle/hc_oracle.c).  The model, loss and
optimiser have textbook definitions; nothing here is shared with the CUDA
path:
  x^ = (x - mu) * isd;  h1 = relu(x^ W1 + b1);  h2 = relu(h1 W2 + b2);
  y = h2 . W3 + b3;     loss = mean((y - t)^2)
  Adam (Kingma and Ba, ICLR 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
The parameter vector uses the layout of hc_mlp: W1[in][h1], b1, W2[h1][h2],
b2, W3[h2], b3.
"""
import numpy as np


def sizes(n_in, h1, h2):
    return [("W1", (n_in, h1)), ("b1", (h1,)), ("W2", (h1, h2)), ("b2", (h2,)), ("W3", (h2,)),
            ("b3", ())]


def unpack(theta, n_in, h1, h2):
    out, o = {}, 0
    for name, shp in sizes(n_in, h1, h2):
        cnt = int(np.prod(shp)) if shp else 1
        out[name] = theta[o:o + cnt].reshape(shp) if shp else theta[o]
        o += cnt
    return out


def pack(P, n_in, h1, h2):
    return np.concatenate([np.atleast_1d(np.asarray(P[name], np.float64)).ravel()
                           for name, _ in sizes(n_in, h1, h2)])


def count(n_in, h1, h2):
    return n_in * h1 + h1 + h1 * h2 + h2 + h2 + 1


def init(seed, n_in, h1, h2):
    """He-style initialisation (scaled Gaussian weights, zero biases)."""
    rng = np.random.default_rng(seed)
    P = {"W1": rng.normal(0, np.sqrt(2.0 / n_in), (n_in, h1)), "b1": np.zeros(h1),
         "W2": rng.normal(0, np.sqrt(2.0 / h1), (h1, h2)), "b2": np.zeros(h2),
         "W3": rng.normal(0, np.sqrt(1.0 / h2), (h2,)), "b3": 0.0}
    return pack(P, n_in, h1, h2)


def forward(theta, mu, isd, X, n_in, h1, h2):
    P = unpack(np.asarray(theta, np.float64), n_in, h1, h2)
    xn = (np.asarray(X, np.float64) - mu) * isd
    z1 = xn @ P["W1"] + P["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ P["W2"] + P["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ P["W3"] + P["b3"]
    return y, (xn, z1, a1, z2, a2)


def loss(theta, mu, isd, X, T, n_in, h1, h2):
    y, _ = forward(theta, mu, isd, X, n_in, h1, h2)
    return float(np.mean((y - T) ** 2))


def gradients(theta, mu, isd, X, T, n_in, h1, h2):
    """Analytic backpropagation of the mean squared error."""
    P = unpack(np.asarray(theta, np.float64), n_in, h1, h2)
    y, (xn, z1, a1, z2, a2) = forward(theta, mu, isd, X, n_in, h1, h2)
    n = X.shape[0]
    dy = 2.0 * (y - T) / n
    g = {"W3": a2.T @ dy, "b3": dy.sum()}
    d2 = np.outer(dy, P["W3"]) * (z2 > 0)
    g["W2"] = a1.T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ P["W2"].T) * (z1 > 0)
    g["W1"] = xn.T @ d1
    g["b1"] = d1.sum(axis=0)
    return pack(g, n_in, h1, h2), float(np.mean((y - T) ** 2))


def adam_step(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def to_bf16(x):
    """Round float values to bfloat16 (nearest, ties to even), as float64."""
    f = np.asarray(x, np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, mu, isd, X, n_in, h1, h2):
    """Inference with every layer's inputs and the weights rounded to
    bfloat16 and sums kept in float64 (the GPU accumulates in float32)."""
    P = unpack(np.asarray(theta, np.float64), n_in, h1, h2)
    xn = to_bf16(((np.asarray(X, np.float32) - mu.astype(np.float32)) * isd.astype(np.float32)))
    a1 = to_bf16(np.maximum(xn @ to_bf16(P["W1"]) + P["b1"].astype(np.float32), 0.0))
    a2 = to_bf16(np.maximum(a1 @ to_bf16(P["W2"]) + P["b2"].astype(np.float32), 0.0))
    return a2 @ to_bf16(P["W3"]) + np.float32(P["b3"])


def _fma32(a, b, c):
    """a * b + c rounded once to float32 for float32 a, b, c: the product is
    exact in float64 (24 + 24 significant bits); the float64 sum can round
    once before the float32 rounding, which differs from a true fused
    multiply-add only when that sum is inexact and lands on a float32 tie."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(np.float32)


def forward_bf16_gpu_order(theta, mu, isd, X, n_in, h1, h2, lanes=32):
    """Inference with every layer's inputs and the weights rounded to
    bfloat16 and float32 sums taken in a fixed order: each hidden unit's sum
    as a chain of fused multiply-adds over its inputs in index order, the
    bias added after the chain, ReLU, then rounding to bfloat16; the output
    as per-lane chains (lane l takes units l, l + lanes, ...) combined by a
    butterfly of float32 additions (strides 16, 8, 4, 2, 1), plus the bias."""
    P = unpack(np.asarray(theta, np.float64), n_in, h1, h2)
    f32 = np.float32
    W1 = to_bf16(P["W1"]).astype(f32)
    W2 = to_bf16(P["W2"]).astype(f32)
    W3 = to_bf16(P["W3"]).astype(f32)
    b1 = np.asarray(P["b1"], f32)
    b2 = np.asarray(P["b2"], f32)
    b3 = f32(P["b3"])
    X = np.asarray(X, f32)
    xn = to_bf16((X - np.asarray(mu, f32)) * np.asarray(isd, f32)).astype(f32)
    n = X.shape[0]
    a = np.zeros((n, h1), f32)
    for i in range(n_in):
        a = _fma32(xn[:, i:i + 1], W1[i][None, :], a)
    hid1 = to_bf16(np.maximum(a + b1, f32(0))).astype(f32)
    a = np.zeros((n, h2), f32)
    for i in range(h1):
        a = _fma32(hid1[:, i:i + 1], W2[i][None, :], a)
    hid2 = to_bf16(np.maximum(a + b2, f32(0))).astype(f32)
    part = np.zeros((n, lanes), f32)
    for j in range(h2):
        part[:, j % lanes] = _fma32(hid2[:, j], W3[j], part[:, j % lanes])
    lane = np.arange(lanes)
    o = lanes // 2
    while o >= 1:
        part = (part + part[:, lane ^ o]).astype(f32)
        o //= 2
    return (part[:, 0] + b3).astype(f32)
