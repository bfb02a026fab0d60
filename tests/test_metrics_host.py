"""The quality metrics the benchmarks report, on hand-made CPU tensors:
recall@10 counts returned entries whose distance is within the true 10th
distance (ties count, padding does not), agreement is exact top-k equality."""
import os
import sys

import pytest
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1209_0410_gb300 import learned  # noqa: E402
import bench  # noqa: E402


def case():
    true_dist = torch.arange(1, 11, dtype=torch.int32).repeat(3, 1)   # 10th true distance = 10
    ids = torch.arange(10, dtype=torch.int32).repeat(3, 1)
    dist = torch.arange(1, 11, dtype=torch.int32).repeat(3, 1).clone()
    dist[1, 5:] = torch.tensor([10, 10, 11, 12, 13], dtype=torch.int32)  # ties at 10 count
    ids[2, 7:] = -1                                                       # padding
    dist[2, 7:] = 2**31 - 1
    return ids, dist, true_dist


@pytest.mark.parametrize("fn", [learned.recall_at_10, bench.recall_at_10])
def test_recall_at_10(fn):
    ids, dist, true_dist = case()
    # rows: 10/10, 7/10 (three beyond the 10th distance), 7/10 (three padded)
    assert fn(ids, dist, true_dist) == pytest.approx((10 + 7 + 7) / 30)


def test_agreement_is_exact_topk_equality():
    ref = torch.arange(20, dtype=torch.int32).reshape(2, 10)
    got = ref.clone()
    assert learned.agreement(got, ref) == 1.0
    got[1, 9] = 99
    assert learned.agreement(got, ref) == 0.5


def test_algorithmic_query_bytes_formula():
    """Window rows and ids, every binary-search probe (8 bytes each; a list
    of n entries takes ceil(log2(n + 1)) of them), the query row and the k
    results, from given positions."""
    import types
    import numpy as np
    # two lists of 10 and 5000 entries; two queries
    off = np.array([0, 10, 5010], dtype=np.uint64)
    pos = torch.tensor([[3, 4000], [10, 100]], dtype=torch.int64)
    fake = types.SimpleNamespace(hc_query_positions=lambda idx, q: pos,
                                 hc_index_describe=lambda idx: ({}, off))
    p, k, row = 4, 10, 128
    qbytes, windows = bench.algorithmic_query_bytes(fake, None, None, p, k, row)
    # windows: list 0 [0, 7) = 7 and [6, 10) = 4; list 1 [3996, 4004) and [96, 104) = 8 each
    assert windows == 7 + 4 + 8 + 8
    probes = 4 + 13   # ceil(log2(11)) + ceil(log2(5001))
    assert qbytes == windows * (row + 4) + 2 * (probes * 8 + row + k * 8)


def test_fixed_recall_point_picks_smallest_depth_reaching_reference():
    sweep = [{"p": 32, "recall_at_10": 0.50, "query_qps": 9e7},
             {"p": 64, "recall_at_10": 0.61, "query_qps": 5e7},
             {"p": 128, "recall_at_10": 0.61, "query_qps": 2.4e7},
             {"p": 256, "recall_at_10": 0.70, "query_qps": 1.2e7}]
    pt = bench.fixed_recall_point(sweep, 128)
    assert pt["p"] == 64 and pt["query_qps"] == 5e7
    assert pt["target_recall_at_10"] == 0.61
    # the reference depth itself when nothing smaller reaches it
    sweep[1]["recall_at_10"] = 0.60
    assert bench.fixed_recall_point(sweep, 128)["p"] == 128
    assert bench.fixed_recall_point(sweep, 100) is None


def test_build_bytes_counts_every_pass():
    """The algorithmic build bytes (rows once, 20-byte records written, every
    pass reading and writing every record) and the kernels' bytes, counted
    here pass by pass for a small case."""
    n, row, c = 1000, 128, 8
    alg, ker = bench.build_bytes(n, row, c, passes=3)
    r = c * n
    assert alg == n * row + 20 * r + 3 * 40 * r
    counts = 16 * 256 * r / 4096
    keys = n * row + 9 * r
    p1 = 1 * r + counts + 8 * r + 13 * r
    p2 = 1 * r + counts + 12 * r + 13 * r
    p3 = 1 * r + counts + 12 * r + 12 * r
    assert ker == pytest.approx(keys + p1 + p2 + p3 + 12 * r + 0.5 * r)
    # the headline workload (6 passes): about 16.0 GB moved per build
    _, k10 = bench.build_bytes(10_000_000, 128, 8)
    assert 15.5e9 < k10 < 16.5e9
