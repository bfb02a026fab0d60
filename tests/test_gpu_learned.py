"""The learned probe depth on the GPU against the oracle.

- hc_features = oracle features, bit for bit (integer-derived values);
- hc_probe_labels = the oracle's minimal depths, exactly;
- FP32 gradients of the MSE = the oracle's float64 backpropagation (whose
  correctness is pinned by finite differences), to float32 rounding;
- one Adam step = the oracle's Adam step from the same gradients;
- FP32 inference = the oracle's float64 forward to float32 rounding;
  BF16-in/FP32-accumulate inference = the oracle's forward in the kernel's
  float32 order, within 4 ulps for 99.9% of samples;
- fused predicted depths = clamp(ceil(2^(y + margin))) of that y, equal for
  99.5% of queries and within one elsewhere;
- trained on GPU labels, the predictor reaches at least the agreement of a
  fixed depth with the same mean, and serving with p = 0 uses it.
"""
import numpy as np
import pytest

from helpers import dev
from oracle import mlp as OM
from oracle import oracle as O
from paper_1209_0410_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_0410_gb300 import hc as _hc
    _hc.lib()
    return _hc


@pytest.fixture(scope="module")
def case(hc):
    db = datagen.make_db(40000, 128, seed=101)
    q = datagen.make_queries(db, 700, seed=102)
    idx = hc.hc_build(dev(db), 8, 16)
    oidx = O.build(db, curves=8, m=16)
    return db, q, idx, oidx


def test_features_bit_exact(hc, case):
    import torch
    db, q, idx, oidx = case
    f = hc.hc_features(idx, dev(q))
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), O.features(oidx, db, q))


def test_labels_exact(hc, case):
    import torch
    db, q, idx, oidx = case
    lab = hc.hc_probe_labels(idx, dev(q[:300]), 10, 160)
    torch.cuda.synchronize()
    ref = O.min_depth_labels(oidx, db, q[:300], 10, 160)
    assert np.array_equal(lab.cpu().numpy().astype(np.int64), ref)


@pytest.fixture(scope="module")
def mlp_case(hc):
    rng = np.random.default_rng(7)
    n_in, h1, h2, n = 32, 64, 64, 1500
    X = rng.normal(3.0, 2.0, (n, n_in)).astype(np.float32)
    T = (rng.normal(0, 1, n) + 0.1 * X[:, 0]).astype(np.float32)
    theta = OM.init(11, n_in, h1, h2).astype(np.float32).astype(np.float64)
    mu = X.mean(axis=0).astype(np.float32)
    isd = (1.0 / X.std(axis=0)).astype(np.float32)
    mlp = hc.MLP(n_in, h1, h2, max_batch=2048)
    mlp.set_params(theta, mu, isd)
    return mlp, theta, mu.astype(np.float64), isd.astype(np.float64), X, T, (n_in, h1, h2)


def test_gradients_match_oracle(hc, mlp_case):
    mlp, theta, mu, isd, X, T, dims = mlp_case
    g, loss = mlp.gradients(dev(X), dev(T))
    ref, ref_loss = OM.gradients(theta, mu, isd, X.astype(np.float64), T.astype(np.float64), *dims)
    g = g.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert np.max(np.abs(g - ref)) <= 2e-4 * scale
    assert loss == pytest.approx(ref_loss, rel=1e-4)


def test_adam_step_matches_oracle(hc, mlp_case):
    mlp, theta, mu, isd, X, T, dims = mlp_case
    hc_theta = theta.astype(np.float32)
    mlp.set_params(hc_theta, mu.astype(np.float32), isd.astype(np.float32))
    g, _ = mlp.gradients(dev(X[:1024]), dev(T[:1024]))
    mlp.train_step(dev(X[:1024]), dev(T[:1024]), 1e-3)
    new, _, _ = mlp.get_params()
    ref, _, _ = OM.adam_step(hc_theta.astype(np.float64), g.cpu().numpy().astype(np.float64),
                             np.zeros(len(theta)), np.zeros(len(theta)), 1, 1e-3)
    assert np.max(np.abs(new - ref)) <= 1e-6
    mlp.set_params(theta.astype(np.float32), mu.astype(np.float32), isd.astype(np.float32))


def test_fit_on_device_matches_oracle_step(hc):
    """hc_mlp_fit over one epoch of one whole minibatch (the samples' order
    then changes nothing): the normalisation equals numpy's mean and unbiased
    standard deviation, and the parameters equal one Adam step (the oracle's
    float64 gradients of the MSE against log2(max(label, 1))) -- to float32
    rounding where a gradient is not negligibly small, and within the step's
    size where it is (its sign is then rounding noise)."""
    import torch
    rng = np.random.default_rng(17)
    n_in, h1, h2, n = 32, 64, 64, 1024
    X = rng.normal(20.0, 4.0, (n, n_in)).astype(np.float32)
    labels = rng.integers(0, 600, n).astype(np.int32)
    theta = OM.init(23, n_in, h1, h2).astype(np.float32)
    mlp = hc.MLP(n_in, h1, h2, max_batch=n)
    mlp.set_params(theta, np.zeros(n_in, np.float32), np.ones(n_in, np.float32))
    lr = 1e-3
    losses = mlp.fit(dev(X), torch.from_numpy(labels).cuda(), 1, n, lr, seed=5)
    got, mu, isd = mlp.get_params()
    Xd = X.astype(np.float64)
    ref_mu = Xd.mean(axis=0)
    ref_isd = 1.0 / np.maximum(Xd.std(axis=0, ddof=1), 1e-3)
    assert np.allclose(mu, ref_mu.astype(np.float32), rtol=1e-6, atol=0)
    assert np.allclose(isd, ref_isd.astype(np.float32), rtol=1e-6, atol=0)
    T = np.log2(np.maximum(labels, 1).astype(np.float32)).astype(np.float64)
    g, loss = OM.gradients(theta.astype(np.float64), mu.astype(np.float64),
                           isd.astype(np.float64), Xd, T, n_in, h1, h2)
    ref, _, _ = OM.adam_step(theta.astype(np.float64), g, np.zeros(len(g)), np.zeros(len(g)), 1, lr)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.max(np.abs(got[big] - ref[big])) <= 1e-6
    assert np.max(np.abs(got - ref)) <= 2 * lr + 1e-6
    assert losses[0] == pytest.approx(loss, rel=1e-4)


def test_fit_lowers_the_loss(hc):
    """Several epochs of shuffled minibatches on a learnable target."""
    rng = np.random.default_rng(19)
    n_in, n = 16, 20000
    X = rng.normal(0.0, 1.0, (n, n_in)).astype(np.float32)
    labels = np.exp2(np.clip(4 + 2 * X[:, 0] - X[:, 1], 0, 9)).astype(np.int32)
    import torch
    mlp = hc.MLP(n_in, 32, 32, max_batch=512)
    mlp.set_params(OM.init(3, n_in, 32, 32).astype(np.float32), np.zeros(n_in, np.float32),
                   np.ones(n_in, np.float32))
    losses = mlp.fit(dev(X), torch.from_numpy(labels).cuda(), 6, 512, 2e-3, seed=1)
    assert len(losses) == 6 and losses[-1] < 0.25 * losses[0]


def test_inference_fp32_and_bf16_match_oracle(hc, mlp_case):
    mlp, theta, mu, isd, X, T, dims = mlp_case
    y32 = mlp.forward(dev(X), bf16=False).cpu().numpy()
    ref32, _ = OM.forward(theta, mu, isd, X, *dims)
    assert np.max(np.abs(y32 - ref32)) <= 1e-4 * (1 + np.abs(ref32).max())
    ybf = mlp.forward(dev(X), bf16=True).cpu().numpy()
    # the oracle takes the kernel's float32 order (FMA chains in index order,
    # bfloat16 roundings at the same points, the warp's butterfly sum)
    refg = OM.forward_bf16_gpu_order(theta, mu, isd, X, *dims)
    ulp = np.spacing(np.abs(refg).astype(np.float32))
    assert (np.abs(ybf - refg) <= 4 * ulp).mean() >= 0.999
    # the rare rest: a fused multiply-add emulated in float64 rounded on the
    # other side of a hidden unit's bfloat16 rounding
    assert np.max(np.abs(ybf - refg)) <= 1e-2 * (1 + np.abs(refg).max())


def test_predicted_depths_follow_model(hc, case):
    import torch
    db, q, idx, oidx = case
    feats = O.features(oidx, db, q)
    rng = np.random.default_rng(5)
    theta = OM.init(21, 32, 64, 64)
    theta[-1] = 7.0                                       # bias near log2(128)
    mu = feats.mean(axis=0).astype(np.float32)
    isd = (1.0 / np.maximum(feats.std(axis=0), 1e-3)).astype(np.float32)
    mlp = hc.MLP(32, 64, 64, max_batch=1024)
    mlp.set_params(theta.astype(np.float32), mu, isd)
    p = mlp.predict_depths(idx, dev(q), margin=0.3, p_lo=4, p_hi=400).cpu().numpy()
    y = OM.forward_bf16_gpu_order(theta.astype(np.float32).astype(np.float64),
                                  mu.astype(np.float64), isd.astype(np.float64), feats, 32, 64, 64)
    e = np.clip((y + np.float32(0.3)).astype(np.float32), -1, 30)
    exp = np.clip(np.ceil(np.exp2(e.astype(np.float64))), 4, 400)
    # equal but where the model output or exp2 sits within a few ulps of an
    # integer depth's boundary
    assert (p == exp).mean() >= 0.995
    assert np.all(np.abs(p - exp) <= 1)
    # the depths are what hc_query_depths consumes: results equal fixed-depth
    # queries of the same p
    pt = torch.from_numpy(p.astype(np.int32)).cuda()
    ids, dist = hc.hc_query_depths(idx, dev(q), 10, pt)
    torch.cuda.synchronize()
    for i in range(0, len(q), 97):
        rid, _ = hc.hc_query(idx, dev(q[i:i + 1]), 10, int(p[i]))
        assert np.array_equal(ids[i].cpu().numpy(), rid[0].cpu().numpy())


def test_trained_predictor_gain_and_serving(hc):
    """Trained on GPU labels, the predictor is at least as good as the fixed
    depth of the same mean (agreement with the p_max top-10), and the serving
    loop answers p = 0 requests with it."""
    import torch
    from paper_1209_0410_gb300 import learned
    db = datagen.make_db(200_000, 128, seed=111)
    qt = datagen.make_queries(db, 40_000, seed=112)
    qv = datagen.make_queries(db, 4_000, seed=113)
    idx = hc.hc_build(dev(db), 8, 16)
    mlp, labels, losses = learned.fit(idx, dev(qt), k=10, p_max=256, epochs=8, batch=2048)
    assert losses[-1] < losses[0]
    tq = dev(qv)
    ref, _ = hc.hc_query(idx, tq, 10, 256)
    p = mlp.predict_depths(idx, tq, 0.25, 1, 256)
    ids, _ = hc.hc_query_depths(idx, tq, 10, p)
    mean_p = int(round(p.double().mean().item()))
    fixed, _ = hc.hc_query(idx, tq, 10, mean_p)
    learned_agree = learned.agreement(ids, ref)
    fixed_agree = learned.agreement(fixed, ref)
    assert learned_agree >= fixed_agree
    # serving: p = 0 requests take the learned depths
    srv = hc.hc_serve_create([idx], 64 << 20)
    srv.attach_predictor(0, mlp, 0.25, 1, 256)
    t = srv.submit(0, qv[:500], 10, 0)
    sids, _ = srv.poll(t, 30_000_000)
    srv.close()
    torch.cuda.synchronize()
    assert np.array_equal(sids, ids[:500].cpu().numpy())
