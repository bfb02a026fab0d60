"""hc_save / hc_load: an index written to a file and read back over the same
rows has the same lists and answers every query as the index that was saved
(and as the oracle); files damaged or crafted one field at a time, or loaded
over other rows, are refused with HC_ERR_FORMAT and leave nothing behind."""
import ctypes
import os
import struct

import numpy as np
import pytest

import index_file as F
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


def lists_of(hc, idx):
    hi, lo, ids, off = hc.hc_index_copy_lists(idx)
    sync()
    return u64(hi), u64(lo), ids.cpu().numpy().view(np.uint32), off


CASES = {
    # name: (n, d, dtype, curves, m, partitions, dim_map seed)
    "u8_m16": (20_000, 128, "u8", 8, 16, 1, None),
    "u8_m16_parts": (12_345, 128, "u8", 4, 16, 3, None),
    "u8_m8_dimmap": (9_001, 64, "u8", 4, 8, 2, 11),
    "f32_m16": (7_000, 32, "f32", 2, 16, 1, None),
}


def make_case(hc, name):
    n, d, dtype, curves, m, parts, dm_seed = CASES[name]
    db = datagen.make_db(n, d, seed=n)
    if dtype == "f32":
        db = datagen.to_f32(db)
    dim_map = None
    if dm_seed is not None:
        dim_map = np.random.default_rng(dm_seed).integers(0, d, (curves, m)).astype(np.uint32)
    t = dev(db)
    idx = hc.hc_build(t, curves=curves, dims_per_curve=m, dim_map=dim_map, partitions=parts)
    return db, t, idx, dim_map


@pytest.mark.parametrize("name", sorted(CASES))
def test_round_trip(hc, tmp_path, name):
    import torch
    db, t, idx, dim_map = make_case(hc, name)
    n, d, dtype, curves, m, parts, _ = CASES[name]
    path = tmp_path / "idx.hcx"
    hc.hc_save(idx, path)
    assert not os.path.exists(str(path) + ".tmp")
    total = n * curves
    lo_words = 8 * total if m < 16 else 0
    dm_bytes = 0 if dim_map is None else 4 * curves * m + (4 * curves * m) % 8
    want = 80 + 8 * (curves * parts + 1) + dm_bytes + 8 * total + lo_words + \
        4 * total + (4 * total) % 8 + 8
    assert os.path.getsize(path) == want
    back = hc.hc_load(path, t)
    assert (back.n, back.d, back.curves, back.m, back.partitions) == (n, d, curves, m, parts)
    for a, b in zip(lists_of(hc, idx), lists_of(hc, back)):
        assert np.array_equal(a, b)
    q = datagen.make_queries(datagen.make_db(n, d, seed=n), 300, seed=5)
    if dtype == "f32":
        q = datagen.to_f32(q)
    qt = dev(q)
    for k, p in ((10, 16), (33, 100)):
        i1, d1 = hc.hc_query(idx, qt, k, p)
        i2, d2 = hc.hc_query(back, qt, k, p)
        i3, d3 = hc.hc_query_ordered(back, qt, k, p)
        sync()
        assert torch.equal(i1, i2) and torch.equal(d1, d2)
        assert torch.equal(i1, i3) and torch.equal(d1, d3)
    idx.free()
    back.free()


def test_loaded_index_matches_the_oracle(hc, tmp_path):
    db, t, idx, _ = make_case(hc, "u8_m16_parts")
    path = tmp_path / "idx.hcx"
    hc.hc_save(idx, path)
    idx.free()
    back = hc.hc_load(path, t)
    q = datagen.make_queries(db, 200, seed=9)
    ids, dist = hc.hc_query(back, dev(q), 10, 40)
    sync()
    oidx = O.build(db, curves=4, m=16, ell=3)
    rids, rdist = O.search(oidx, db, q, 10, 40)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(dist.cpu().numpy(), O.int32_dist(rdist))
    back.free()


def try_load(hc, path, t):
    """(status, index handle or None) of one raw hc_load call."""
    h = ctypes.c_void_p()
    rc = hc.lib().hc_load(os.fsencode(str(path)), ctypes.c_void_p(t.data_ptr()), None,
                          ctypes.byref(h))
    assert (rc == hc.HC_OK) == bool(h.value)
    return rc, h


def load_status(hc, path, t):
    rc, h = try_load(hc, path, t)
    if h.value:
        hc.lib().hc_free(h)
    return rc


@pytest.fixture(scope="module")
def saved(hc, tmp_path_factory):
    """A saved 8-curve index of 20,000 rows and the section offsets of its file."""
    db, t, idx, _ = make_case(hc, "u8_m16")
    path = tmp_path_factory.mktemp("saved") / "idx.hcx"
    hc.hc_save(idx, path)
    idx.free()
    secs = F.sections(path, 20_000, 8)
    return db, t, path, secs


def edited(tmp_path, src, offset, fmt, value, reseal):
    data = bytearray(open(src, "rb").read())
    struct.pack_into(fmt, data, offset, value)
    p = tmp_path / "edited.hcx"
    p.write_bytes(bytes(data))
    if reseal:
        F.reseal(p)
    return p


def test_damaged_files_are_refused(hc, tmp_path, saved):
    db, t, path, (hi, _, ids, end) = saved
    orig = open(path, "rb").read()
    for off in (hi + 8 * 5_000, ids + 4 * 77, end):   # a key, an id, the checksum
        word = struct.unpack_from("<Q", orig, off - off % 8)[0]
        p = edited(tmp_path, path, off - off % 8, "<Q", word ^ (1 << 40), reseal=False)
        assert load_status(hc, p, t) == hc.HC_ERR_FORMAT


def test_crafted_files_are_refused(hc, tmp_path, saved):
    """Each with a valid checksum: only the content check can refuse it."""
    db, t, path, (hi, _, ids, end) = saved
    orig = open(path, "rb").read()
    id0 = struct.unpack_from("<I", orig, ids)[0]
    id1 = struct.unpack_from("<I", orig, ids + 4)[0]
    h0 = struct.unpack_from("<Q", orig, hi)[0]
    h1 = struct.unpack_from("<Q", orig, hi + 8)[0]
    cases = [
        (ids + 4, "<I", id0),            # a row twice, another missing
        (ids + 4, "<I", 20_000),         # a row past the end
        (ids + 4, "<I", 0xFFFFFFFF),
        (hi, "<Q", h1 + 1),              # keys out of order
    ]
    assert h1 >= h0 and id1 != id0
    for off, fmt, val in cases:
        p = edited(tmp_path, path, off, fmt, val, reseal=True)
        assert load_status(hc, p, t) == hc.HC_ERR_FORMAT, (off, val)
    # two ids swapped: still a permutation, sorted keys, valid checksum, but
    # the keys no longer belong to those rows
    data = bytearray(orig)
    struct.pack_into("<II", data, ids, id1, id0)
    p = tmp_path / "swapped.hcx"
    p.write_bytes(bytes(data))
    F.reseal(p)
    assert load_status(hc, p, t) == hc.HC_ERR_FORMAT


def test_other_rows_are_refused(hc, saved):
    db, t, path, _ = saved
    other = dev(datagen.make_db(20_000, 128, seed=4242))
    assert load_status(hc, path, other) == hc.HC_ERR_FORMAT
    assert load_status(hc, path, t) == hc.HC_OK


def test_allocation_failure_leaves_nothing(hc, saved):
    """Each device allocation of hc_load failing in turn: HC_ERR_OOM, no index."""
    db, t, path, _ = saved
    ooms = 0
    for after in range(8):
        hc.hc_debug_fail_alloc(after)
        try:
            rc = load_status(hc, path, t)
        finally:
            hc.hc_debug_fail_alloc(-1)
        if rc == hc.HC_OK:
            break
        assert rc == hc.HC_ERR_OOM
        ooms += 1
    assert ooms >= 3   # list offsets, keys, ids
    assert load_status(hc, path, t) == hc.HC_OK
