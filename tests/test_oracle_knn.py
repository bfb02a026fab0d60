"""Pins of the oracle's Algorithms 1 and 2 and of the exact kNN (Eq. 3).

- brute force over tiny inputs, computed here independently with numpy;
- a hand-worked fixture under tests/golden/;
- Algorithm 2 with a window covering every list returns the exact kNN;
- candidate sets are nested in p, so the i-th distance never grows with p;
- the sorted lists hold every id once, in (key, id) order, with the keys of
  the direct projection;
- lower_bound positions agree with numpy's searchsorted on the 128-bit keys.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1209_0410_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def numpy_exact_knn(db, q, k):
    """Exact kNN by numpy: squared distances in int64/float64, order by
    (distance, id), pad with (-1, inf)."""
    dbf = db.astype(np.float64) if db.dtype == np.float32 else db.astype(np.int64)
    qf = q.astype(np.float64) if q.dtype == np.float32 else q.astype(np.int64)
    ids = np.full((len(q), k), -1, np.int64)
    dist = np.full((len(q), k), np.inf)
    for i in range(len(q)):
        dd = ((dbf - qf[i]) ** 2).sum(axis=1).astype(np.float64)
        order = np.lexsort((np.arange(len(db)), dd))[:k]
        ids[i, :len(order)] = order
        dist[i, :len(order)] = dd[order]
    return ids, dist


def small_case(n=3000, nq=40, d=128, seed=21):
    db = datagen.make_db(n, d, seed=seed)
    q = datagen.make_queries(db, nq, seed=seed + 100)
    return db, q


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_bruteforce_matches_numpy(dtype):
    db, q = small_case(1500, 25)
    if dtype == "f32":
        db, q = datagen.to_f32(db), datagen.to_f32(q)
    ids, dist = O.bruteforce(db, q, 10)
    rids, rdist = numpy_exact_knn(db, q, 10)
    assert np.array_equal(ids, rids)
    if dtype == "u8":
        assert np.array_equal(dist, rdist)
    else:   # double sums in a different order: equal to rounding
        assert np.allclose(dist, rdist, rtol=1e-12, atol=0)


def test_bruteforce_pads_when_k_exceeds_n():
    db = np.array([[0, 0], [3, 4], [1, 1]], np.uint8)
    q = np.array([[0, 0]], np.uint8)
    ids, dist = O.bruteforce(db, q, 5)
    assert ids.tolist() == [[0, 2, 1, -1, -1]]
    assert dist[0, :3].tolist() == [0.0, 2.0, 25.0] and np.all(np.isinf(dist[0, 3:]))


def load_golden_knn():
    path = os.path.join(GOLDEN, "knn_hand_example.txt")
    sec, rows, queries, expect = None, [], [], []
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("["):
            sec = line
            continue
        vals = [int(v) for v in line.split()]
        {"[db]": rows, "[queries]": queries, "[expect]": expect}[sec].append(vals)
    return (np.array(rows, np.uint8), np.array(queries, np.uint8), expect)


def test_golden_hand_example():
    """Hand-computed squared distances and tie order (lower id first)."""
    db, q, expect = load_golden_knn()
    k = (len(expect[0]) - 1) // 2
    ids, dist = O.bruteforce(db, q, k)
    for e in expect:
        qi = e[0]
        assert ids[qi].tolist() == e[1:1 + k]
        assert dist[qi].tolist() == [float(v) for v in e[1 + k:]]
    # Algorithm 2 with a window over the whole list gives the same answer
    index = O.build(db, curves=2, m=2)
    sids, sdist = O.search(index, db, q, k, p=len(db))
    assert np.array_equal(sids, ids) and np.array_equal(sdist, dist)


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("m,curves", [(16, 8), (8, 16), (16, 4)])
def test_full_window_is_exact_knn(dtype, m, curves):
    db, q = small_case(2000, 30)
    if dtype == "f32":
        db, q = datagen.to_f32(db), datagen.to_f32(q)
    index = O.build(db, curves=curves, m=m)
    ids, dist = O.search(index, db, q, 10, p=len(db))
    bids, bdist = O.bruteforce(db, q, 10)
    assert np.array_equal(ids, bids) and np.array_equal(dist, bdist)


def test_lists_sorted_and_complete():
    db, _ = small_case(2500, 1)
    dim_map = np.random.default_rng(3).permutation(128).astype(np.uint32).reshape(8, 16)
    index = O.build(db, curves=8, m=16, dim_map=dim_map)
    for L in range(index.lists):
        sl = index.list_slice(L)
        ids = index.ids[sl]
        assert np.array_equal(np.sort(ids), np.arange(len(db)))
        hi, lo = index.keys_hi[sl], index.keys_lo[sl]
        # (key, id) strictly increasing
        order = np.lexsort((ids, lo, hi))
        assert np.array_equal(order, np.arange(len(ids)))
        # keys equal C^-1 of the projection of each row
        h2, l2 = O.hilbert_keys(16, 8, db[ids][:, dim_map[L]].astype(np.uint32))
        assert np.array_equal(h2, hi) and np.array_equal(l2, lo)


def test_positions_are_lower_bounds():
    db, q = small_case(3000, 50)
    index = O.build(db, curves=8, m=16)
    _, _, pos = O.search(index, db, q, 10, p=16, return_pos=True)
    qh, ql = O.query_keys(q, 8, 16)
    for L in range(8):
        sl = index.list_slice(L)
        keys = [O.key_int(h, l) for h, l in zip(index.keys_hi[sl], index.keys_lo[sl])]
        for i in range(len(q)):
            qk = O.key_int(qh[i, L], ql[i, L])
            exp = int(np.searchsorted(np.array(keys, dtype=object), qk, side="left"))
            assert pos[i, L] == exp


def window_ids(index, L, pos, p):
    sl = index.list_slice(L)
    n = sl.stop - sl.start
    lo, hi = max(0, pos - p), min(n, pos + p)
    return set(index.ids[sl][lo:hi].tolist())


def test_result_is_topk_of_window_union():
    """Algorithm 2: the answer is the k nearest of the union of the windows."""
    db, q = small_case(3000, 30)
    index = O.build(db, curves=8, m=16)
    p, k = 20, 10
    ids, dist, pos = O.search(index, db, q, k, p, return_pos=True)
    for i in range(len(q)):
        cand = set()
        for L in range(8):
            cand |= window_ids(index, L, int(pos[i, L]), p)
        cand = np.array(sorted(cand))
        dd = ((db[cand].astype(np.int64) - q[i].astype(np.int64)) ** 2).sum(axis=1)
        order = np.lexsort((cand, dd))[:k]
        assert ids[i].tolist() == cand[order].tolist()
        assert dist[i].tolist() == dd[order].astype(float).tolist()


def test_monotone_in_depth():
    """Windows are nested in p, so the i-th distance is non-increasing in p,
    and once the top-k equals the one at p_max it stays equal up to p_max."""
    db, q = small_case(3000, 40)
    index = O.build(db, curves=8, m=16)
    ps = [0, 1, 2, 4, 8, 16, 32, 64, 128, 3000]
    res = [O.search(index, db, q, 10, p) for p in ps]
    for (i1, d1), (i2, d2) in zip(res, res[1:]):
        assert np.all(d2 <= d1)
    final_ids = res[-1][0]
    for qi in range(len(q)):
        same = [np.array_equal(r[0][qi], final_ids[qi]) for r in res]
        first = same.index(True)
        assert all(same[first:])


def test_zero_depth_returns_padding():
    db, q = small_case(500, 5)
    index = O.build(db, curves=8, m=16)
    ids, dist = O.search(index, db, q, 7, 0)
    assert np.all(ids == -1) and np.all(np.isinf(dist))


def test_k_larger_than_candidates_pads():
    db, q = small_case(500, 5)
    index = O.build(db, curves=2, m=16)
    ids, dist = O.search(index, db, q, 100, 3)
    for i in range(len(q)):
        nvalid = int((ids[i] >= 0).sum())
        assert 3 <= nvalid <= 12
        assert np.all(ids[i, nvalid:] == -1) and np.all(np.isinf(dist[i, nvalid:]))
        assert np.all(np.diff(dist[i, :nvalid]) >= 0)


def test_duplicate_rows_tie_by_id():
    """Equal keys sort by ascending id; equal distances rank the lower id first."""
    rng = np.random.default_rng(7)
    base = rng.integers(0, 256, size=(50, 32), dtype=np.uint8)
    db = np.concatenate([base, base, base])       # every row three times
    q = base[:10]
    index = O.build(db, curves=2, m=16)
    for L in range(2):
        sl = index.list_slice(L)
        ids = index.ids[sl]
        keys = list(zip(index.keys_hi[sl], index.keys_lo[sl]))
        for a in range(len(ids) - 1):
            if keys[a] == keys[a + 1]:
                assert ids[a] < ids[a + 1]
    ids, dist = O.search(index, db, q, 3, 200)
    for i in range(10):
        assert ids[i].tolist() == [i, i + 50, i + 100]
        assert dist[i].tolist() == [0.0, 0.0, 0.0]


def test_generator_is_thread_independent():
    a = datagen.make_db(777, 64, seed=5, nthreads=1)
    b = datagen.make_db(777, 64, seed=5, nthreads=7)
    assert np.array_equal(a, b)
    qa = datagen.make_queries(a, 33, seed=6, nthreads=1)
    qb = datagen.make_queries(a, 33, seed=6, nthreads=5)
    assert np.array_equal(qa, qb)


def test_generator_published_splitmix64():
    """SplitMix64 from state 0: first output 0xE220A8397B1DCDAF."""
    out = datagen.splitmix64(0, 2)
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_generator_statistics():
    z = datagen.gaussians(9, 3, 0, 400_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    db = datagen.make_db(20_000, 128, seed=1)
    assert db.min() == 0 and db.max() == 255
    q, src = datagen.make_queries(db, 2000, seed=3, return_src=True)
    diff = q.astype(np.float64) - db[src.astype(np.int64)].astype(np.float64)
    inner = (db[src.astype(np.int64)] > 40) & (db[src.astype(np.int64)] < 215)
    assert abs(diff[inner].std() - 8.0) < 0.2
