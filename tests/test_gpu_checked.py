"""The bounds-checked build (libhc_check.so, -DHC_CHECK): the paths run
through it give the oracle's results bit for bit and refuse no access; a
byte written into a buffer's guard and a row id past the database are
reported (both planted inside memory the test owns, so nothing outside an
allocation is touched whatever the build)."""
import numpy as np
import pytest

from helpers import dev
from oracle import oracle as O
from paper_1209_0410_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_0410_gb300 import _build
    from paper_1209_0410_gb300 import hc as _hc
    _build.build_hc_check()
    checked = _hc.load_library(_hc.CHECK_LIB_PATH)
    with _hc.use_library(checked):
        _hc.hc_check_status(reset=True)
        yield _hc
        _hc.hc_check_status(reset=True)


def sync():
    import torch
    torch.cuda.synchronize()


def clean(hc):
    r = hc.hc_check_status()
    assert r["enabled"] == 1
    assert r["violations"] == 0, r


class DeviceWords:
    """A CUDA tensor over library-owned device memory (no copy)."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


def raw(ptr, count, typestr):
    import torch
    return torch.as_tensor(DeviceWords(ptr, count, typestr), device="cuda")


@pytest.mark.parametrize("n,curves,m,parts,k,p", [
    (6000, 8, 16, 1, 10, 40), (5003, 4, 16, 5, 7, 0), (4000, 4, 16, 1, 33, 5000),
    (3001, 4, 8, 2, 10, 64),
])
def test_paths_match_the_oracle_and_refuse_nothing(hc, n, curves, m, parts, k, p):
    db = datagen.make_db(n, 128 if m == 16 else 64, seed=n)
    q = datagen.make_queries(db, 100, seed=n + 1)
    idx = hc.hc_build(dev(db), curves=curves, dims_per_curve=m, partitions=parts)
    ids, dist = hc.hc_query(idx, dev(q), k, p)
    ids2, dist2 = hc.hc_query_ordered(idx, dev(q), k, p)
    sync()
    oidx = O.build(db, curves=curves, m=m, ell=parts)
    rids, rdist = O.search(oidx, db, q, k, p)
    for a, b in ((ids, dist), (ids2, dist2)):
        assert np.array_equal(a.cpu().numpy(), rids)
        assert np.array_equal(b.cpu().numpy(), O.int32_dist(rdist))
    idx.free()
    clean(hc)


def test_runs_of_equal_keys_refuse_nothing(hc):
    """Identical rows: every list is one run (the long-run fix-up)."""
    base = datagen.make_db(40, 128, seed=3)
    db = np.concatenate([np.repeat(base[:1], 3000, 0), base, np.repeat(base[5:6], 50, 0)])
    idx = hc.hc_build(dev(db))
    q = datagen.make_queries(db, 20, seed=4)
    ids, dist = hc.hc_query(idx, dev(q), 10, 64)
    sync()
    oidx = O.build(db, curves=8, m=16)
    rids, rdist = O.search(oidx, db, q, 10, 64)
    assert np.array_equal(ids.cpu().numpy(), rids)
    idx.free()
    clean(hc)


def test_multi_and_file_paths_refuse_nothing(hc, tmp_path):
    import torch
    jobs_db = [datagen.make_db(n, 128, seed=n) for n in (3000, 7000)]
    idxs = [hc.hc_build(dev(d)) for d in jobs_db]
    qs = [dev(datagen.make_queries(d, 50, seed=1)) for d in jobs_db]
    for wpq in (1, 2, 4):
        jobs = [hc.MultiJob(i, q, 10, 40, warps_per_query=wpq) for i, q in zip(idxs, qs)]
        hc.hc_query_multi(jobs)
        sync()
        for j in jobs:
            rids, rdist = hc.hc_query(j.index, j.q, 10, 40)
            sync()
            assert torch.equal(j.ids, rids) and torch.equal(j.dist, rdist)
    path = tmp_path / "i.hcx"
    hc.hc_save(idxs[0], path)
    back = hc.hc_load(path, idxs[0].db)
    back.free()
    for i in idxs:
        i.free()
    clean(hc)


def test_guard_overwrite_is_reported(hc):
    db = datagen.make_db(2000, 128, seed=8)
    idx = hc.hc_build(dev(db), curves=4, dims_per_curve=16)
    info, _ = hc.hc_index_describe(idx)
    sync()
    total = 2000 * 4
    guard = raw(info["keys_hi_dev"] + 8 * total, 256, "|u1")   # inside the checked allocation
    saved = guard.clone()
    guard[17] = 0
    sync()
    r = hc.hc_check_status(reset=True)
    assert r["violations"] == 1 and r["site"] == 13 and r["index"] == 17, r
    guard.copy_(saved)
    sync()
    idx.free()
    clean(hc)


def test_row_id_past_the_database_is_refused(hc):
    """An id equal to n in a list: the checked walk records it (site 9) and
    reads row 0 instead.  The rows sit in a larger tensor, so row n exists in
    memory either way."""
    import torch
    n = 2000
    big = dev(datagen.make_db(n + 16, 128, seed=9))
    db = big[:n]
    idx = hc.hc_build(db, curves=2, dims_per_curve=16)
    info, _ = hc.hc_index_describe(idx)
    sync()
    ids = raw(info["ids_dev"], 2 * n, "<i4")
    keep = ids[100].clone()
    ids[100] = n
    sync()
    q = db[:8].clone()
    hc.hc_query(idx, q, 10, 4 * n)   # full windows: every entry is visited
    sync()
    r = hc.hc_check_status(reset=True)
    assert r["violations"] >= 1 and r["site"] == 9, r
    assert r["index"] == n and r["bound"] == n
    ids[100] = keep
    sync()
    idx.free()
    clean(hc)
