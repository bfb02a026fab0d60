"""Training and evaluation driver of the learned probe depth.

Every arithmetic step runs in libhc kernels: labels (hc_probe_labels, through
the query kernel), features (hc_features), training (hc_mlp_fit: targets,
normalisation statistics, the per-epoch order of the samples, minibatch
gathers and Adam steps, all on the device) and inference
(hc_mlp_predict_depths).  This module only orders the calls; the initial
weights are drawn on the host like any other seeded input.
"""
import numpy as np
import torch

from . import hc


def he_init(seed, n_in, h1, h2):
    """Seeded He-style initialisation in the hc_mlp parameter layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / n_in), n_in * h1), np.zeros(h1),
             rng.normal(0, np.sqrt(2.0 / h1), h1 * h2), np.zeros(h2),
             rng.normal(0, np.sqrt(1.0 / h2), h2), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def fit(index, q_train, k=10, p_max=512, epochs=12, batch=2048, lr=2e-3, seed=0,
        h1=64, h2=64, stream=None):
    """Labels, features and an Adam-trained MLP for one index.

    Returns (mlp, labels, losses) with losses the mean training loss per
    epoch."""
    labels = hc.hc_probe_labels(index, q_train, k, p_max, stream=stream)
    feats = hc.hc_features(index, q_train, stream=stream)
    n_in = feats.shape[1]
    mlp = hc.MLP(n_in, h1, h2, max_batch=batch)
    mlp.set_params(he_init(seed, n_in, h1, h2), np.zeros(n_in, np.float32),
                   np.ones(n_in, np.float32))
    losses = mlp.fit(feats, labels, epochs, batch, lr, seed=seed, stream=stream)
    return mlp, labels, losses


def agreement(ids, ref_ids):
    """Fraction of queries whose top-k ids equal the reference's."""
    return float((ids == ref_ids).all(dim=1).to(torch.float64).mean().item())


def recall_at_10(ids, dist, true_dist):
    kth = true_dist[:, 9:10].to(torch.float64)
    ok = (dist[:, :10].to(torch.float64) <= kth) & (ids[:, :10] >= 0)
    return float(ok.sum(dim=1).clamp(max=10).to(torch.float64).mean().item() / 10.0)


def choose_margin(mlp, index, q_val, ref_ids, k, target_agreement, p_lo=1, p_hi=512,
                  margins=None):
    """Smallest margin (log2 units) whose learned depths reach the target
    agreement with the reference top-k on validation queries."""
    if margins is None:
        margins = [m / 4.0 for m in range(-8, 17)]
    for m in margins:
        p = mlp.predict_depths(index, q_val, m, p_lo, p_hi)
        ids, _ = hc.hc_query_depths(index, q_val, k, p)
        if agreement(ids, ref_ids) >= target_agreement:
            return m
    return margins[-1]
