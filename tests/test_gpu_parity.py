"""GPU path vs the CPU oracle, element by element, through the C ABI.

uint8: bit-exact (keys, sorted lists, positions, ids, int32 distances).
float32: distances within 1e-5 relative of the oracle's double sums; id sets
equal except inside the tie band at the k-th distance.
Sizes span several 4096-record sort tiles and 32-row gather chunks with
ragged tails; edge cases: p = 0, p beyond the list, k beyond the candidates,
duplicate rows, one query, queries not a multiple of the block's 8 warps.
"""
import numpy as np
import pytest

from helpers import compare_f32, dev, u64
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


def sync():
    import torch
    torch.cuda.synchronize()


def make_case(n, nq, d=128, seed=41, dtype="u8"):
    db = datagen.make_db(n, d, seed=seed)
    q = datagen.make_queries(db, nq, seed=seed + 7)
    if dtype == "f32":
        db, q = datagen.to_f32(db), datagen.to_f32(q)
    return db, q


# ------------------------------------------------------------------ K1
@pytest.mark.parametrize("m,curves,mapped", [(16, 8, False), (16, 8, True), (8, 16, False),
                                             (5, 3, True), (1, 4, False), (16, 1, False),
                                             (13, 2, True)])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_hilbert_keys_bit_exact(hc, m, curves, mapped, dtype):
    rng = np.random.default_rng(m * 100 + curves)
    d = 128
    x = rng.integers(0, 256, size=(5003, d), dtype=np.uint8)
    x[0] = 0
    x[1] = 255
    x[2, ::2] = 255
    if dtype == "f32":
        x = datagen.to_f32(x)
        x[3] = np.float32(-0.5)
        x[4] = np.float32(1.7)
        x[5, :7] = np.array([np.nan, np.inf, -np.inf, 0.5 / 255, 1.5 / 255, 254.5 / 255, 1.0],
                            np.float32)
        x[6:200] = rng.random((194, d), dtype=np.float32) * np.float32(1.2) - np.float32(0.1)
    dim_map = rng.permutation(d)[:curves * m].astype(np.uint32).reshape(curves, m) if mapped \
        else None
    hi, lo = hc.hc_hilbert_keys(dev(x), curves, m, dim_map)
    sync()
    ohi, olo = O.query_keys(x, curves, m, dim_map)
    assert np.array_equal(u64(hi), ohi)
    assert np.array_equal(u64(lo), olo)


# ------------------------------------------------------------------ K2
SORT_CASES = ["random", "duplicates", "narrow", "ragged", "reversed_ids", "runs32", "runs33",
              "hi_ties", "prefix_ties"]


@pytest.mark.parametrize("case", SORT_CASES)
def test_sort_keys_matches_stable_sort(hc, case):
    """Both sort paths: the high-word-first path with its run fix-up (runs of
    equal high words up to 32 long) and the every-digit path it falls back to."""
    import torch
    rng = np.random.default_rng(SORT_CASES.index(case) + 1)
    sizes = {"random": [30000], "duplicates": [20000, 5000], "narrow": [12289],
             "ragged": [0, 1, 4095, 4096, 4097, 9000, 33, 0, 2],
             "reversed_ids": [8192, 7000], "runs32": [32 * 700 + 5], "runs33": [33 * 300],
             "hi_ties": [40000], "prefix_ties": [50000, 7]}[case]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    total = int(off[-1])
    key_bits = 128
    hi = rng.integers(0, 2**63, size=total, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=total, dtype=np.uint64)
    lo = rng.integers(0, 2**63, size=total, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=total, dtype=np.uint64)
    if case == "duplicates":
        pool_hi = hi[:37].copy()
        pool_lo = lo[:37].copy()
        pick = rng.integers(0, 37, size=total)
        hi, lo = pool_hi[pick], pool_lo[pick]
    if case == "narrow":
        key_bits = 40
        hi[:] = 0
        lo &= np.uint64((1 << 40) - 1)
    if case in ("runs32", "runs33"):
        run = 32 if case == "runs32" else 33
        hi = np.repeat(hi[: total // run + 1], run)[:total].copy()
    if case == "hi_ties":          # short runs of equal high words, some equal keys
        hi = hi[rng.integers(0, total // 3, size=total)].copy()
        lo[rng.random(total) < 0.3] = np.uint64(5)
    if case == "prefix_ties":      # equal top 56 bits, differing low bytes of the high word
        top = hi[rng.integers(0, total // 4, size=total)] & np.uint64(0xFFFFFFFFFFFFFF00)
        hi = top | rng.integers(0, 4, size=total, dtype=np.uint64)
        lo[rng.random(total) < 0.5] = np.uint64(9)
    ids = np.arange(total, dtype=np.uint32)
    if case == "reversed_ids":
        ids = ids[::-1].copy()
        hi[:] = hi[:16].repeat(total // 16 + 1)[:total]
        lo[:] = 7
    th = torch.from_numpy(hi.view(np.int64)).cuda()
    tl = torch.from_numpy(lo.view(np.int64)).cuda()
    ti = torch.from_numpy(ids.view(np.int32)).cuda()
    hc.hc_sort_keys(th, tl, ti, off, key_bits)
    sync()
    gh, gl, gi = u64(th), u64(tl), ti.cpu().numpy().view(np.uint32)
    for s in range(len(sizes)):
        a, b = int(off[s]), int(off[s + 1])
        order = np.lexsort((np.arange(b - a), lo[a:b], hi[a:b]))  # stable by key
        assert np.array_equal(gh[a:b], hi[a:b][order])
        assert np.array_equal(gl[a:b], lo[a:b][order])
        assert np.array_equal(gi[a:b], ids[a:b][order])


# ------------------------------------------------------- Algorithm 1 lists
BUILD_CASES = [
    dict(n=10007, parts=1, dtype="u8", mapped=False, curves=8, m=16, d=128),
    dict(n=20000, parts=3, dtype="u8", mapped=False, curves=8, m=16, d=128),
    dict(n=9000, parts=1, dtype="u8", mapped=True, curves=8, m=16, d=128),
    dict(n=12000, parts=2, dtype="f32", mapped=False, curves=8, m=16, d=128),
    dict(n=7001, parts=1, dtype="u8", mapped=False, curves=4, m=16, d=64),
    dict(n=6000, parts=1, dtype="u8", mapped=False, curves=16, m=16, d=256),
    dict(n=5000, parts=1, dtype="u8", mapped=False, curves=10, m=6, d=64),
    dict(n=5, parts=1, dtype="u8", mapped=False, curves=8, m=16, d=128),
    dict(n=3, parts=4, dtype="u8", mapped=False, curves=2, m=16, d=32),
]


def build_both(hc, c):
    db, _ = make_case(c["n"], 1, d=c["d"], dtype=c["dtype"], seed=c["n"])
    rng = np.random.default_rng(c["n"])
    dim_map = rng.permutation(c["d"])[:c["curves"] * c["m"]].astype(np.uint32).reshape(
        c["curves"], c["m"]) if c["mapped"] else None
    idx = hc.hc_build(dev(db), curves=c["curves"], dims_per_curve=c["m"], dim_map=dim_map,
                      partitions=c["parts"])
    oidx = O.build(db, curves=c["curves"], m=c["m"], dim_map=dim_map, ell=c["parts"])
    return db, dim_map, idx, oidx


@pytest.mark.parametrize("c", BUILD_CASES, ids=lambda c: "n%d_l%d_%s_c%d_m%d_d%d%s" % (
    c["n"], c["parts"], c["dtype"], c["curves"], c["m"], c["d"], "_map" if c["mapped"] else ""))
def test_build_lists_bit_exact(hc, c):
    _, _, idx, oidx = build_both(hc, c)
    hi, lo, ids, off = hc.hc_index_copy_lists(idx)
    sync()
    assert np.array_equal(off, oidx.list_off)
    assert np.array_equal(u64(hi), oidx.keys_hi)
    assert np.array_equal(u64(lo), oidx.keys_lo)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), oidx.ids)
    idx.free()


@pytest.mark.parametrize("c", BUILD_CASES[:4])
def test_positions_bit_exact(hc, c):
    db, dim_map, idx, oidx = build_both(hc, c)
    _, q = make_case(c["n"], 203, d=c["d"], dtype=c["dtype"], seed=c["n"])
    pos = hc.hc_query_positions(idx, dev(q))
    sync()
    _, _, opos = O.search(oidx, db, q, 1, 0, return_pos=True)
    assert np.array_equal(pos.cpu().numpy(), opos)
    idx.free()


# ------------------------------------------------------- Algorithm 2 queries
@pytest.mark.parametrize("k,p", [(10, 64), (1, 5), (33, 17), (64, 50), (100, 40), (128, 200),
                                 (10, 0), (10, 1), (7, 1_000_000), (10, 3)])
def test_query_u8_bit_exact(hc, k, p):
    n, nq = 20011, 301
    db, q = make_case(n, nq, seed=5)
    idx = hc.hc_build(dev(db))
    ids, dist = hc.hc_query(idx, dev(q), k, p)
    sync()
    oidx = O.build(db, curves=8, m=16)
    rids, rdist = O.search(oidx, db, q, k, p)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("d,curves,m,k,p", [(64, 4, 16, 10, 40), (256, 16, 16, 10, 30),
                                            (32, 2, 16, 5, 20), (48, 3, 16, 10, 25),
                                            (128, 12, 10, 10, 33)])
def test_query_u8_other_shapes(hc, d, curves, m, k, p):
    n, nq = 9001, 77
    db, q = make_case(n, nq, d=d, seed=d)
    idx = hc.hc_build(dev(db), curves=curves, dims_per_curve=m)
    ids, dist = hc.hc_query(idx, dev(q), k, p)
    sync()
    oidx = O.build(db, curves=curves, m=m)
    rids, rdist = O.search(oidx, db, q, k, p)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("parts,scheme_p", [(2, 64), (3, 20), (8, 10), (5, 100000), (32, 13),
                                             (32, 4)])
def test_query_partitioned_bit_exact(hc, parts, scheme_p):
    n, nq, k = 24000, 150, 10
    db, q = make_case(n, nq, seed=parts)
    idx = hc.hc_build(dev(db), partitions=parts)
    ids, dist = hc.hc_query(idx, dev(q), k, scheme_p)
    sync()
    oidx = O.build(db, curves=8, m=16, ell=parts)
    rids, rdist = O.search(oidx, db, q, k, scheme_p)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("d,k,p,parts", [(128, 10, 64, 1), (64, 10, 50, 1), (256, 10, 30, 1),
                                         (128, 100, 40, 1), (128, 10, 64, 3), (16, 3, 9, 1)])
def test_query_f32_within_tolerance(hc, d, k, p, parts):
    n, nq = 15013, 211
    curves = max(1, d // 16)
    db, q = make_case(n, nq, d=d, seed=d + 1, dtype="f32")
    idx = hc.hc_build(dev(db), curves=curves, dims_per_curve=16, partitions=parts)
    ids, dist = hc.hc_query(idx, dev(q), k, p)
    sync()
    oidx = O.build(db, curves=curves, m=16, ell=parts)
    rids, rdist = O.search(oidx, db, q, k, p)
    probs = compare_f32(ids.cpu().numpy(), dist.cpu().numpy(), rids, rdist)
    assert not probs, probs[:5]
    idx.free()


def test_f32_index_has_u8_windows(hc):
    """x = u8/255 in float32 quantises back to the bytes: same keys and lists."""
    n = 8000
    db, _ = make_case(n, 1, seed=77)
    a = hc.hc_build(dev(db))
    b = hc.hc_build(dev(datagen.to_f32(db)))
    ha, la, ia, _ = hc.hc_index_copy_lists(a)
    hb, lb, ib, _ = hc.hc_index_copy_lists(b)
    sync()
    assert np.array_equal(u64(ha), u64(hb)) and np.array_equal(u64(la), u64(lb))
    assert np.array_equal(ia.cpu().numpy(), ib.cpu().numpy())


def test_duplicate_rows_rank_lower_id_first(hc):
    rng = np.random.default_rng(3)
    base = rng.integers(0, 256, size=(1500, 128), dtype=np.uint8)
    db = np.concatenate([base, base, base, base])
    q = base[:100].copy()
    idx = hc.hc_build(dev(db))
    ids, dist = hc.hc_query(idx, dev(q), 4, 64)
    sync()
    oidx = O.build(db, curves=8, m=16)
    rids, rdist = O.search(oidx, db, q, 4, 64)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    g = ids.cpu().numpy()
    for i in range(100):
        assert g[i].tolist() == [i, i + 1500, i + 3000, i + 4500]


@pytest.mark.parametrize("parts,copies", [(1, 40), (3, 40), (1, 32), (1, 33), (2, 31)])
def test_build_long_runs_of_equal_keys(hc, parts, copies):
    """Rows repeated `copies` times: runs of equal keys (equal high words,
    so the low words are read from the rows) of up to 32 entries are ordered
    by one warp each, longer ones by one block each.  The lists (low words
    recomputed from the rows) and queries (which tie on the high word) match
    the oracle."""
    rng = np.random.default_rng(17)
    base = rng.integers(0, 256, size=(60, 128), dtype=np.uint8)
    db = np.concatenate([np.repeat(base, copies, axis=0),
                         rng.integers(0, 256, size=(3001, 128), dtype=np.uint8)])
    db = db[rng.permutation(len(db))]
    idx = hc.hc_build(dev(db), partitions=parts)
    hi, lo, ids, off = hc.hc_index_copy_lists(idx)
    sync()
    oidx = O.build(db, curves=8, m=16, ell=parts)
    assert np.array_equal(u64(hi), oidx.keys_hi)
    assert np.array_equal(u64(lo), oidx.keys_lo)
    assert np.array_equal(ids.cpu().numpy().astype(np.int64), oidx.ids.astype(np.int64))
    q = np.concatenate([base[:20], db[:30]])
    rids, rdist = O.search(oidx, db, q, 10, 24)
    gids, gdist = hc.hc_query(idx, dev(q), 10, 24)
    sync()
    assert np.array_equal(gids.cpu().numpy(), rids)
    assert np.array_equal(gdist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("n", [1, 2, 31, 33, 70])
def test_query_tiny_databases(hc, n):
    """Lists shorter than one 32-entry step (and than the 16 entries of one
    fence point, which some lists then lack): the packed walk fills steps
    from several windows and pads the top-k when fewer than k rows exist;
    the ordered path's batch search agrees."""
    db, q = make_case(n, 40, seed=n + 11)
    idx = hc.hc_build(dev(db))
    oidx = O.build(db, curves=8, m=16)
    for k, p in [(10, 2), (10, 100), (1, 1), (128, 40)]:
        rids, rdist = O.search(oidx, db, q, k, p)
        for query in (hc.hc_query, hc.hc_query_ordered):
            ids, dist = query(idx, dev(q), k, p)
            sync()
            assert np.array_equal(ids.cpu().numpy(), rids)
            assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


def test_query_depths_per_query_matches_fixed(hc):
    """hc_query_depths with a different depth per query (0 included) equals
    one fixed-depth query per distinct depth."""
    import torch
    n, nq = 15013, 257
    db, q = make_case(n, nq, seed=41)
    idx = hc.hc_build(dev(db))
    rng = np.random.default_rng(3)
    depths = rng.choice([0, 1, 5, 16, 31, 32, 33, 100, 700], size=nq).astype(np.int32)
    ids, dist = hc.hc_query_depths(idx, dev(q), 10, torch.from_numpy(depths).cuda())
    sync()
    oidx = O.build(db, curves=8, m=16)
    for p in np.unique(depths):
        sel = np.flatnonzero(depths == p)
        rids, rdist = O.search(oidx, db, q[sel], 10, int(p))
        assert np.array_equal(ids.cpu().numpy()[sel], rids)
        assert np.array_equal(dist.cpu().numpy()[sel], O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("dtype,nq,k,p,parts", [("u8", 1000, 10, 64, 1), ("u8", 1, 10, 50, 1),
                                                 ("u8", 7, 33, 20, 1), ("u8", 2049, 100, 30, 3),
                                                 ("f32", 300, 10, 40, 1)])
def test_query_ordered_equals_query(hc, dtype, nq, k, p, parts):
    """Answering the queries in curve-0 key order changes no result."""
    import torch
    db, q = make_case(20011, nq, seed=nq + 5, dtype=dtype)
    idx = hc.hc_build(dev(db), partitions=parts)
    ids_a, dist_a = hc.hc_query(idx, dev(q), k, p)
    ids_b, dist_b = hc.hc_query_ordered(idx, dev(q), k, p)
    sync()
    assert torch.equal(ids_a, ids_b)
    assert torch.equal(dist_a.view(torch.int32), dist_b.view(torch.int32))
    if dtype == "u8":
        oidx = O.build(db, curves=8, m=16, ell=parts)
        rids, _ = O.search(oidx, db, q, k, p)
        assert np.array_equal(ids_b.cpu().numpy(), rids)
    idx.free()


def test_free_async_on_streams(hc):
    """Indexes built, queried and released in stream order on two streams
    give the same answers as on the default stream."""
    import torch
    db, q = make_case(12000, 64, seed=8)
    tdb, tq = dev(db), dev(q)
    ref = hc.hc_query(hc.hc_build(tdb), tq, 10, 30)[0].clone()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(6):
        s = streams[i % 2]
        idx = hc.hc_build(tdb, stream=s)
        ids, _ = hc.hc_query(idx, tq, 10, 30, stream=s)
        idx.free(stream=s)
        outs.append(ids)
    sync()
    for ids in outs:
        assert torch.equal(ids, ref)


@pytest.mark.parametrize("d,curves,m,parts", [(64, 10, 6, 1), (128, 12, 10, 1), (256, 16, 16, 1),
                                               (64, 10, 6, 2), (128, 12, 10, 3), (64, 4, 16, 5)])
def test_query_ordered_other_key_widths(hc, d, curves, m, parts):
    """Order keys from 48-, 80- and 128-bit extended-keys (indexes that keep
    low words; their fence is written after the sort), on one to five
    partitions: the ordered path gives hc_query's results, and the oracle's
    on the partitioned cases."""
    import torch
    db, q = make_case(9001, 333, d=d, seed=d + m + parts)
    idx = hc.hc_build(dev(db), curves=curves, dims_per_curve=m, partitions=parts)
    ids_a, dist_a = hc.hc_query(idx, dev(q), 10, 25)
    ids_b, dist_b = hc.hc_query_ordered(idx, dev(q), 10, 25)
    sync()
    assert torch.equal(ids_a, ids_b) and torch.equal(dist_a, dist_b)
    if parts > 1:
        oidx = O.build(db, curves=curves, m=m, ell=parts)
        rids, rdist = O.search(oidx, db, q, 10, 25)
        assert np.array_equal(ids_b.cpu().numpy(), rids)
        assert np.array_equal(dist_b.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("parts,curves,m,nq", [(8, 8, 16, 1000), (32, 8, 16, 333),
                                                (16, 16, 8, 65), (256, 1, 16, 40),
                                                (3, 32, 4, 97), (2, 8, 16, 501),
                                                (1, 8, 16, 1000), (1, 3, 16, 130)])
def test_query_ordered_batch_search_many_lists(hc, parts, curves, m, nq):
    """The ordered path's batch search (a warp per 32 neighbouring keys of one
    curve, over that curve's list in every partition; with one or two
    partitions a lane takes four or two queries) gives the positions of
    Algorithm 2: the walk over 3 to 256 lists equals the oracle's search,
    with batches that end in a partial warp."""
    db, q = make_case(20011, nq, seed=parts * 7 + curves)
    idx = hc.hc_build(dev(db), curves=curves, dims_per_curve=m, partitions=parts)
    ids, dist = hc.hc_query_ordered(idx, dev(q), 10, 6)
    sync()
    oidx = O.build(db, curves=curves, m=m, ell=parts)
    rids, rdist = O.search(oidx, db, q, 10, 6)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


def nibble_variants(rng, row, count):
    """Rows equal to `row` in the top 4 bits of every coordinate: their keys
    share the high word (the top 4 bits of each of a curve's 16 coordinates)
    and differ in the low word."""
    low = rng.integers(0, 16, size=(count, row.shape[0]), dtype=np.uint8)
    return (row & np.uint8(0xF0))[None, :] | low


@pytest.mark.parametrize("parts", [1, 3])
def test_searches_with_high_words_tied_across_fence_blocks(hc, parts):
    """Entries whose high words tie over runs of 16 to 700 entries (many
    16-entry fence blocks, fence words equal to the query's high word) and
    queries that tie them: the lower_bound falls back to the low words, and
    the positions of both search paths (per-query warps, the ordered batch
    pass) and the answers equal the oracle's."""
    rng = np.random.default_rng(29)
    base = rng.integers(0, 256, size=(3, 128), dtype=np.uint8)
    db = np.concatenate([rng.integers(0, 256, size=(3000, 128), dtype=np.uint8),
                         nibble_variants(rng, base[0], 700), nibble_variants(rng, base[1], 40),
                         nibble_variants(rng, base[2], 16)])
    db = db[rng.permutation(len(db))]
    q = np.concatenate([nibble_variants(rng, base[0], 30), nibble_variants(rng, base[1], 10),
                        nibble_variants(rng, base[2], 5), db[:25]])
    idx = hc.hc_build(dev(db), partitions=parts)
    oidx = O.build(db, curves=8, m=16, ell=parts)
    rids, rdist, opos = O.search(oidx, db, q, 10, 24, return_pos=True)
    pos = hc.hc_query_positions(idx, dev(q))
    ids_a, dist_a = hc.hc_query(idx, dev(q), 10, 24)
    ids_b, dist_b = hc.hc_query_ordered(idx, dev(q), 10, 24)
    sync()
    assert np.array_equal(pos.cpu().numpy(), opos)
    for ids, dist in ((ids_a, dist_a), (ids_b, dist_b)):
        assert np.array_equal(ids.cpu().numpy(), rids)
        assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


def test_query_ordered_rejects_a_small_workspace(hc):
    import torch
    db, q = make_case(5000, 100, seed=2)
    idx = hc.hc_build(dev(db))
    ws = torch.empty(hc.hc_query_ordered_workspace(idx, 100) - 256, dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(hc.HCError):
        hc.hc_query_ordered(idx, dev(q), 10, 20, workspace=ws)
    idx.free()


@pytest.mark.parametrize("nq", [0, 1, 7, 9, 1000])
def test_query_batch_sizes(hc, nq):
    n = 6000
    db, q = make_case(n, max(nq, 1), seed=nq + 3)
    q = q[:nq]
    idx = hc.hc_build(dev(db))
    ids, dist = hc.hc_query(idx, dev(q), 10, 32)
    sync()
    assert ids.shape == (nq, 10)
    if nq:
        oidx = O.build(db, curves=8, m=16)
        rids, rdist = O.search(oidx, db, q, 10, 32)
        assert np.array_equal(ids.cpu().numpy(), rids)
        assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))


def test_query_host_matches_device(hc):
    n, nq = 8000, 123
    db, q = make_case(n, nq, seed=9)
    idx = hc.hc_build_host(db)
    ids_h, dist_h = hc.hc_query_host(idx, q, 10, 50)
    oidx = O.build(db, curves=8, m=16)
    rids, rdist = O.search(oidx, db, q, 10, 50)
    assert np.array_equal(ids_h.numpy(), rids)
    assert np.array_equal(dist_h.numpy(), O.int32_dist(rdist))
    # twice more, with a smaller and a larger batch (staging reuse / growth)
    for m in (17, nq):
        ids_h, dist_h = hc.hc_query_host(idx, q[:m], 10, 50)
        assert np.array_equal(ids_h.numpy(), rids[:m])


@pytest.mark.parametrize("parts", [1, 3])
def test_build_host_from_pinned_rows(hc, parts):
    """hc_build_host from pinned host rows: the lists equal those of a build
    from device memory, and a full-depth query (every row of the library's
    device copy) is the exact kNN."""
    import torch
    n, nq = 20011, 97
    db, q = make_case(n, nq, seed=29)
    pinned = torch.from_numpy(db).pin_memory()
    idx_h = hc.hc_build_host(pinned, partitions=parts)
    idx_d = hc.hc_build(dev(db), partitions=parts)
    a = hc.hc_index_copy_lists(idx_h)
    b = hc.hc_index_copy_lists(idx_d)
    sync()
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    ids_h, dist_h = hc.hc_query_host(idx_h, q, 10, 40)
    oidx = O.build(db, curves=8, m=16, ell=parts)
    rids, rdist = O.search(oidx, db, q, 10, 40)
    assert np.array_equal(ids_h.numpy(), rids)
    assert np.array_equal(dist_h.numpy(), O.int32_dist(rdist))
    ids_f, dist_f = hc.hc_query_host(idx_h, q[:20], 10, n)
    fids, fdist = O.bruteforce(db, q[:20], 10)
    assert np.array_equal(ids_f.numpy(), fids)
    assert np.array_equal(dist_f.numpy(), O.int32_dist(fdist))


# ------------------------------------------------------------- exact kNN
@pytest.mark.parametrize("dtype,k,d", [("u8", 10, 128), ("u8", 100, 128), ("u8", 1, 64),
                                       ("f32", 10, 128), ("f32", 33, 256), ("u8", 128, 32)])
def test_bruteforce_matches_oracle(hc, dtype, k, d):
    n, nq = 7013, 61
    db, q = make_case(n, nq, d=d, seed=k, dtype=dtype)
    ids, dist = hc.hc_bruteforce(dev(db), dev(q), k)
    sync()
    rids, rdist = O.bruteforce(db, q, k)
    if dtype == "u8":
        assert np.array_equal(ids.cpu().numpy(), rids)
        assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    else:
        probs = compare_f32(ids.cpu().numpy(), dist.cpu().numpy(), rids, rdist)
        assert not probs, probs[:5]


def test_full_depth_query_equals_bruteforce(hc):
    n, nq = 4000, 64
    db, q = make_case(n, nq, seed=12)
    idx = hc.hc_build(dev(db))
    ids, dist = hc.hc_query(idx, dev(q), 10, n)
    bids, bdist = hc.hc_bruteforce(dev(db), dev(q), 10)
    sync()
    assert np.array_equal(ids.cpu().numpy(), bids.cpu().numpy())
    assert np.array_equal(dist.cpu().numpy(), bdist.cpu().numpy())


# ------------------------------------------------------------- error paths
def test_invalid_arguments_are_rejected(hc):
    import torch
    db, q = make_case(2000, 4, seed=1)
    idx = hc.hc_build(dev(db))
    tq = dev(q)
    for k, p in ((0, 10), (129, 10), (10, (1 << 30) + 1)):
        with pytest.raises(hc.HCError) as e:
            hc.hc_query(idx, tq, k, p, out_ids=torch.empty((4, max(k, 1)), dtype=torch.int32,
                                                           device="cuda"),
                        out_dist=torch.empty((4, max(k, 1)), dtype=torch.int32, device="cuda"))
        assert e.value.status == hc.HC_ERR_ARG
    # a host buffer where a device buffer is required
    rc = hc.lib().hc_query(idx.handle, q.ctypes.data, 4, 10, 10,
                           torch.empty((4, 10), dtype=torch.int32, device="cuda").data_ptr(),
                           torch.empty((4, 10), dtype=torch.int32, device="cuda").data_ptr(), None)
    assert rc == hc.HC_ERR_ARG
    # build parameter checks
    with pytest.raises(hc.HCError):
        hc.hc_build(dev(db), curves=9)                 # 9*16 > d
    with pytest.raises(hc.HCError):
        hc.hc_build(dev(db), dims_per_curve=17)
    with pytest.raises(hc.HCError):
        hc.hc_build(dev(db[:, :120].copy()))           # rows not a multiple of 16 bytes
    with pytest.raises(hc.HCError):
        hc.hc_build(dev(db), curves=8, partitions=33)  # 264 lists


def test_injected_allocation_failure_reports_oom(hc):
    db, q = make_case(3000, 5, seed=2)
    tdb = dev(db)
    for after in range(0, 6):
        hc.hc_debug_fail_alloc(after)
        try:
            idx = hc.hc_build(tdb)
        except hc.HCError as e:
            assert e.status == hc.HC_ERR_OOM
        else:
            idx.free()
        finally:
            hc.hc_debug_fail_alloc(-1)
    # the library is usable afterwards
    idx = hc.hc_build(tdb)
    ids, _ = hc.hc_query(idx, dev(q), 5, 16)
    sync()
    oidx = O.build(db, curves=8, m=16)
    rids, _ = O.search(oidx, db, q, 5, 16)
    assert np.array_equal(ids.cpu().numpy(), rids)


def test_query_at_precomputed_positions(hc):
    """hc_query_positions + hc_query_at = hc_query, bit for bit."""
    import torch
    n, nq = 20011, 333
    db, q = make_case(n, nq, seed=17)
    idx = hc.hc_build(dev(db))
    tq = dev(q)
    pos = hc.hc_query_positions(idx, tq)
    ids, dist = hc.hc_query_at(idx, tq, 10, 64, pos)
    rids, rdist = hc.hc_query(idx, tq, 10, 64)
    torch.cuda.synchronize()
    assert torch.equal(ids, rids) and torch.equal(dist, rdist)
