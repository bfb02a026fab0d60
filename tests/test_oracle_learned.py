"""Pins of the oracle side of the learned probe depth.

- octave encoding: its defining bounds on random 128-bit integers;
- features: recomputed by brute force (Python integers for the key gaps,
  numpy for the centre-window distances) from the oracle's lists;
- MLP backpropagation: central finite differences of the loss;
- Adam: the first step moves every parameter by lr * sign(gradient);
- bfloat16 rounding: torch's float32 -> bfloat16 conversion;
- depth labels: minimal (the top-k changes one step below) and sufficient.
"""
import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from paper_1209_0410_gb300 import datagen


def test_octave_definition():
    rng = np.random.default_rng(1)
    vals = [0, 1, 2, 3, 4, 5, 65535, 65536, 65537, 2**64 - 1, 2**64, 2**127, 2**128 - 1]
    vals += [int(rng.integers(1, 2**63)) << int(rng.integers(0, 64)) for _ in range(300)]
    for g in vals:
        o = O.octave(g)
        if g == 0:
            assert o == 0.0
            continue
        e = g.bit_length() - 1
        assert int(o) == 1 + e                     # 2^(o-1) <= g < 2^o
        frac = (o - 1 - e) * 65536
        assert frac == int(frac)
        # the 16 bits just below the top bit
        below = ((g << 16) >> e) & 0xFFFF
        assert int(frac) == below


def test_features_brute_force():
    db = datagen.make_db(6000, 128, seed=81)
    q = datagen.make_queries(db, 60, seed=82)
    index = O.build(db, curves=8, m=16)
    feat = O.features(index, db, q)
    _, _, pos = O.search(index, db, q, 1, 0, return_pos=True)
    qh, ql = O.query_keys(q, 8, 16)
    for i in range(len(q)):
        for c in range(8):
            sl = index.list_slice(c)
            keys = [O.key_int(h, l) for h, l in zip(index.keys_hi[sl], index.keys_lo[sl])]
            qk = O.key_int(qh[i, c], ql[i, c])
            p = int(pos[i, c])
            n = len(keys)
            exp0 = O.octave(qk - keys[p - 1]) if p > 0 else O.FEAT_NONE
            exp1 = O.octave(keys[p] - qk) if p < n else O.FEAT_NONE
            lo, hi = max(0, p - 4), min(n, p + 4)
            ids = index.ids[sl][lo:hi]
            d = ((db[ids].astype(np.int64) - q[i].astype(np.int64)) ** 2).sum(axis=1)
            assert feat[i, 4 * c + 0] == np.float32(exp0)
            assert feat[i, 4 * c + 1] == np.float32(exp1)
            assert feat[i, 4 * c + 2] == np.float32(O.octave(int(d.min())))
            assert feat[i, 4 * c + 3] == np.float32(O.octave(int(d.sum()) // len(d)))


@pytest.fixture(scope="module")
def small_mlp():
    rng = np.random.default_rng(3)
    n_in, h1, h2 = 12, 9, 7
    theta = M.init(5, n_in, h1, h2)
    X = rng.normal(0, 1, (40, n_in))
    T = rng.normal(0, 1, 40)
    mu = rng.normal(0, 0.2, n_in)
    isd = rng.uniform(0.5, 2.0, n_in)
    return theta, mu, isd, X, T, (n_in, h1, h2)


def test_backprop_matches_finite_differences(small_mlp):
    theta, mu, isd, X, T, dims = small_mlp
    g, _ = M.gradients(theta, mu, isd, X, T, *dims)
    h = 1e-6
    num = np.zeros_like(theta)
    for j in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        num[j] = (M.loss(tp, mu, isd, X, T, *dims) - M.loss(tm, mu, isd, X, T, *dims)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-7)


def test_backprop_catches_a_dropped_relu_mask(small_mlp):
    """Negative control: gradients without the ReLU mask disagree with the
    finite differences, so the check above can see such a mistake."""
    theta, mu, isd, X, T, (n_in, h1, h2) = small_mlp
    P = M.unpack(theta, n_in, h1, h2)
    y, (xn, z1, a1, z2, a2) = M.forward(theta, mu, isd, X, n_in, h1, h2)
    dy = 2.0 * (y - T) / X.shape[0]
    d2_wrong = np.outer(dy, P["W3"])               # mask dropped
    gW2_wrong = a1.T @ d2_wrong
    g, _ = M.gradients(theta, mu, isd, X, T, n_in, h1, h2)
    gW2 = M.unpack(g, n_in, h1, h2)["W2"]
    assert not np.allclose(gW2, gW2_wrong)


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    g[:5] = 0.0
    new, m, v = M.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01, eps=1e-12)
    step = theta - new
    assert np.allclose(step[5:], 0.01 * np.sign(g[5:]), rtol=1e-6)
    assert np.all(step[:5] == 0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(0, 3, 5000), rng.uniform(-1e-3, 1e-3, 500),
                        [0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.3e38]]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(M.to_bf16(x), ref)


def test_depth_labels_minimal_and_sufficient():
    db = datagen.make_db(5000, 128, seed=91)
    q = datagen.make_queries(db, 50, seed=92)
    index = O.build(db, curves=8, m=16)
    k, p_max = 10, 96
    lab = O.min_depth_labels(index, db, q, k, p_max)
    ref, _ = O.search(index, db, q, k, p_max)
    for i in range(len(q)):
        at, _ = O.search(index, db, q[i:i + 1], k, int(lab[i]))
        assert np.array_equal(at[0], ref[i])
        if lab[i] > 0:
            below, _ = O.search(index, db, q[i:i + 1], k, int(lab[i]) - 1)
            assert not np.array_equal(below[0], ref[i])


def test_gpu_order_forward_exact_on_representable_values():
    """With small-integer weights and inputs every partial sum is an integer
    below 2^24, exact in float32 and in float64 alike, so the GPU-order
    forward equals the float64-sum bfloat16 forward (same rounding points)
    bit for bit; and the first hidden layer (sums below 256, exact in
    bfloat16) matches the plain float64 forward's."""
    rng = np.random.default_rng(3)
    n_in, h1, h2 = 12, 40, 36
    theta = rng.integers(-3, 4, M.count(n_in, h1, h2)).astype(np.float64)
    X = rng.integers(0, 8, (50, n_in)).astype(np.float64)
    mu, isd = np.zeros(n_in), np.ones(n_in)
    yb = M.forward_bf16(theta, mu, isd, X, n_in, h1, h2)
    yg = M.forward_bf16_gpu_order(theta, mu, isd, X, n_in, h1, h2)
    assert np.array_equal(yg.astype(np.float64), yb)
    _, (_, _, a1, _, _) = M.forward(theta, mu, isd, X, n_in, h1, h2)
    assert np.abs(a1).max() < 256


def test_gpu_order_forward_close_to_float64_forward():
    """On random data the GPU-order forward stays within bfloat16 resolution
    of the float64 bfloat16 forward (which rounds the same values)."""
    rng = np.random.default_rng(4)
    n_in, h1, h2 = 32, 64, 64
    theta = M.init(5, n_in, h1, h2)
    X = rng.normal(0, 1, (400, n_in))
    mu, isd = np.zeros(n_in), np.ones(n_in)
    yg = M.forward_bf16_gpu_order(theta, mu, isd, X, n_in, h1, h2).astype(np.float64)
    yb = M.forward_bf16(theta, mu, isd, X, n_in, h1, h2)
    scale = 1 + np.abs(yb).max()
    assert np.median(np.abs(yg - yb)) <= 1e-4 * scale
    assert np.max(np.abs(yg - yb)) <= 3e-2 * scale


def test_gpu_order_output_butterfly():
    """The output sum: 64 units on 32 lanes, lane l holding units l and
    l + 32, combined by the butterfly; with one unit non-zero per lane the
    result is their float32 sum in the butterfly's order."""
    n_in, h1, h2 = 1, 1, 64
    theta = np.zeros(M.count(n_in, h1, h2))
    P = M.unpack(theta.copy(), n_in, h1, h2)
    P["W1"][:] = 1.0
    P["W2"][:] = 1.0
    P["W3"][:] = 2.0 ** -np.arange(64)          # exact in bfloat16
    theta = M.pack(P, n_in, h1, h2)
    y = M.forward_bf16_gpu_order(theta, np.zeros(1), np.ones(1), np.ones((1, 1)), n_in, h1, h2)
    lanes = np.zeros(32, np.float32)
    for j in range(64):
        lanes[j % 32] = np.float32(lanes[j % 32] + np.float32(2.0 ** -j))
    o = 16
    while o >= 1:
        lanes = (lanes + lanes[np.arange(32) ^ o]).astype(np.float32)
        o //= 2
    assert y[0] == lanes[0]
