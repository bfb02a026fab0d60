"""Algorithm 1's sorted lists from hc_build, against the oracle.

hc_build radix-sorts the top 48 bits of every 16-coordinate key; runs of
entries with equal 48-bit prefixes are then ordered by (key, low word, id)
on the device: runs of up to 8 entries inside one 32-entry chunk, without two
equal high words, by the streaming pass that finds the runs; other runs of
up to 32 entries by one warp each; up to 256 by one warp through shared
memory; longer runs by one block each through global memory.  The cases below reach each of those paths
at sizes the oracle builds in seconds, and the lists must equal the oracle's
bit for bit (keys, low words recomputed from the rows, ids).  The last case
checks that hc_build returns without waiting for its stream.
"""
import time

import numpy as np
import pytest

from helpers import dev, u64
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


def assert_lists_equal(hc, idx, oidx):
    hi, lo, ids, off = hc.hc_index_copy_lists(idx)
    sync()
    assert np.array_equal(off, oidx.list_off)
    gh, gl = u64(hi), u64(lo)
    gi = ids.cpu().numpy().view(np.uint32)
    for L in range(len(off) - 1):
        a, b = int(off[L]), int(off[L + 1])
        assert np.array_equal(gh[a:b], oidx.keys_hi[a:b]), "high words of list %d" % L
        assert np.array_equal(gl[a:b], oidx.keys_lo[a:b]), "low words of list %d" % L
        assert np.array_equal(gi[a:b], oidx.ids[a:b]), "ids of list %d" % L


@pytest.mark.parametrize("n,parts", [(600_000, 1), (900_000, 3), (3_000_000, 1)])
def test_long_lists_bit_exact(hc, n, parts):
    """Lists of 300k to 3M entries: many sort tiles per list, ragged last
    tiles, and the short runs of equal 48-bit prefixes such lists hold."""
    db = datagen.make_db(n, 128, seed=n + parts)
    idx = hc.hc_build(dev(db), partitions=parts)
    oidx = O.build(db, curves=8, m=16, ell=parts)
    assert_lists_equal(hc, idx, oidx)
    idx.free()


def test_long_runs_sorted_on_the_device(hc):
    """30,000 copies of one row make a run of equal keys far longer than a
    warp sorts, and groups of 40 copies make runs just beyond it: both are
    ordered by one block each, by (key, low word, id)."""
    rng = np.random.default_rng(5)
    base = datagen.make_db(170_000, 128, seed=77)
    dup = np.repeat(base[:1], 30_000, axis=0)
    groups = np.repeat(base[1:101], 40, axis=0)
    db = np.concatenate([base, dup, groups])[rng.permutation(170_000 + 30_000 + 4_000)]
    db = np.ascontiguousarray(db)
    idx = hc.hc_build(dev(db))
    oidx = O.build(db, curves=8, m=16)
    assert_lists_equal(hc, idx, oidx)
    q = np.ascontiguousarray(np.concatenate([base[:5], db[:20]]))
    rids, rdist = O.search(oidx, db, q, 10, 50)
    gids, gdist = hc.hc_query(idx, dev(q), 10, 50)
    sync()
    assert np.array_equal(gids.cpu().numpy(), rids)
    assert np.array_equal(gdist.cpu().numpy(), O.int32_dist(rdist))
    idx.free()


@pytest.mark.parametrize("seed", [1, 2])
def test_runs_of_every_length_with_and_without_tied_high_words(hc, seed):
    """Groups of 2 to 300 variants of one row.  Low nibbles redrawn: equal
    high words (bit planes 7..4), different low words, so the run needs the
    low words.  Bit 4 redrawn: equal 48-bit prefixes (planes 7..5) but
    different high words.  Every run class of the fix-up is reached (inside a
    chunk or across its edge, up to 8, 32, 256 records and beyond), and the
    lists must equal the oracle's bit for bit."""
    rng = np.random.default_rng(seed)
    base = datagen.make_db(40_000, 128, seed=100 + seed)
    parts = [base]
    for size in (2, 3, 5, 8, 9, 20, 33, 100, 300):
        for g in range(20):
            row = base[rng.integers(0, len(base))]
            v = np.repeat(row[None, :], size, axis=0)
            if g % 2 == 0:
                v = (v & 0xF0) | rng.integers(0, 16, size=v.shape, dtype=np.uint8)
            else:
                v = (v & 0xEF) | (rng.integers(0, 2, size=v.shape, dtype=np.uint8) << 4)
            parts.append(v.astype(np.uint8))
    db = np.concatenate(parts)
    db = np.ascontiguousarray(db[rng.permutation(len(db))])
    idx = hc.hc_build(dev(db))
    oidx = O.build(db, curves=8, m=16)
    assert_lists_equal(hc, idx, oidx)
    idx.free()


def test_run_of_a_million_equal_keys(hc):
    """Half of 2M rows equal: every list holds one run of a million equal
    keys, ordered by id."""
    rng = np.random.default_rng(9)
    base = datagen.make_db(1_000_000, 128, seed=91)
    db = np.concatenate([base, np.repeat(base[:1], 1_000_000, axis=0)])
    db = np.ascontiguousarray(db[rng.permutation(len(db))])
    idx = hc.hc_build(dev(db))
    oidx = O.build(db, curves=8, m=16)
    assert_lists_equal(hc, idx, oidx)
    idx.free()


def test_identical_rows_only(hc):
    """Every row equal: every key of a list is equal and the lists are the
    ids in order."""
    db = np.repeat(datagen.make_db(1, 128, seed=3), 50_000, axis=0)
    idx = hc.hc_build(dev(db), partitions=2)
    oidx = O.build(db, curves=8, m=16, ell=2)
    assert_lists_equal(hc, idx, oidx)
    idx.free()


def test_build_returns_without_waiting(hc):
    """hc_build queues its work and returns: behind a kernel that keeps the
    stream busy for about a second, the call comes back long before the
    stream is idle, and the lists are then right."""
    import torch
    db = datagen.make_db(300_000, 128, seed=12)
    tdb = dev(db)
    hc.hc_build(tdb).free()          # load the kernels first
    sync()
    stream = torch.cuda.current_stream()
    torch.cuda._sleep(2_000_000_000)   # ~1 s of clock cycles on the stream
    t0 = time.perf_counter()
    idx = hc.hc_build(tdb, stream=stream)
    t_call = time.perf_counter() - t0
    busy = not stream.query()
    sync()
    assert busy, "the stream went idle before the call returned"
    assert t_call < 0.25, "hc_build took %.3f s on the host" % t_call
    assert_lists_equal(hc, idx, O.build(db, curves=8, m=16))
    idx.free()
