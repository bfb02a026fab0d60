"""hc_load's checks that run on the host before any device work (no GPU):
the header, the list layout and the file size of the format documented in
include/hc.h.  A file that passes them reaches the database check, which
refuses a null database with HC_ERR_ARG."""
import ctypes
import os

import numpy as np
import pytest

from paper_1209_0410_gb300 import hc
import index_file as F


def status(path, db=None):
    h = ctypes.c_void_p()
    rc = hc.lib().hc_load(os.fsencode(str(path)), db, None, ctypes.byref(h))
    assert not h.value, "no index may come back from a failed load"
    return rc


def small_file(tmp_path, name="idx.bin", n=100, d=16, curves=1, m=16, partitions=1, **hkw):
    """A well-formed file of n rows: sorted keys, each list a permutation."""
    rng = np.random.default_rng(7)
    lists = curves * partitions
    starts = [(j * n) // partitions for j in range(partitions + 1)]
    list_off = [0]
    hi, ids = [], []
    for L in range(lists):
        j = L // curves
        ln = starts[j + 1] - starts[j]
        list_off.append(list_off[-1] + ln)
        hi.append(np.sort(rng.integers(0, 2**63, ln, dtype=np.uint64)))
        ids.append(rng.permutation(np.arange(starts[j], starts[j + 1], dtype=np.uint32)))
    head = F.header(n, d, curves, m, partitions=partitions, **hkw)
    data = F.assemble(head, list_off, np.concatenate(hi), np.concatenate(ids))
    path = tmp_path / name
    path.write_bytes(data)
    return path, data


def test_statuses_are_named():
    assert hc.hc_strerror(hc.HC_ERR_IO) == "file input/output failed"
    assert hc.hc_strerror(hc.HC_ERR_FORMAT) == "not a valid index file for this database"


def test_null_arguments():
    h = ctypes.c_void_p()
    assert hc.lib().hc_load(None, None, None, ctypes.byref(h)) == hc.HC_ERR_ARG
    assert hc.lib().hc_load(b"x", None, None, None) == hc.HC_ERR_ARG
    assert hc.lib().hc_save(None, b"x", None) == hc.HC_ERR_ARG


def test_missing_file_is_io(tmp_path):
    assert status(tmp_path / "nope.bin") == hc.HC_ERR_IO


def test_well_formed_file_reaches_the_database_check(tmp_path):
    path, _ = small_file(tmp_path)
    assert status(path) == hc.HC_ERR_ARG
    path, _ = small_file(tmp_path, "p3.bin", n=1001, d=64, curves=4, partitions=3)
    assert status(path) == hc.HC_ERR_ARG


@pytest.mark.parametrize("cut", [0, 7, 80, 88, 200])
def test_short_files(tmp_path, cut):
    _, data = small_file(tmp_path)
    p = tmp_path / "short.bin"
    p.write_bytes(data[:cut])
    assert status(p) == hc.HC_ERR_FORMAT


def test_size_must_match(tmp_path):
    _, data = small_file(tmp_path)
    for extra in (data[:-8], data + b"\0" * 8):
        p = tmp_path / "size.bin"
        p.write_bytes(extra)
        assert status(p) == hc.HC_ERR_FORMAT


@pytest.mark.parametrize("field", [
    dict(magic=b"HCURVIDY"), dict(version=2), dict(bom=0x04030201), dict(flags=4),
    dict(reserved=1), dict(bits=7), dict(dtype=2), dict(row_bytes=32), dict(lists=2),
    dict(flags=1),            # low words stored for 16-coordinate keys: not this layout
])
def test_header_fields(tmp_path, field):
    path, _ = small_file(tmp_path, **field)
    assert status(path) == hc.HC_ERR_FORMAT


def test_invalid_parameters(tmp_path):
    # d = 15 gives 15-byte rows (not a multiple of 16); curves * m > d
    for kw in (dict(d=15), dict(d=16, m=16, curves=2)):
        n = 50
        curves = kw.get("curves", 1)
        head = F.header(n, kw["d"], curves, kw.get("m", 16))
        list_off = [c * n for c in range(curves + 1)]
        hi = np.arange(n * curves, dtype=np.uint64)
        ids = np.tile(np.arange(n, dtype=np.uint32), curves)
        p = tmp_path / "bad.bin"
        p.write_bytes(F.assemble(head, list_off, hi, ids))
        assert status(p) == hc.HC_ERR_FORMAT


def test_list_offsets_must_match_the_partition_layout(tmp_path):
    n, curves, parts = 1001, 2, 3
    starts = [(j * n) // parts for j in range(parts + 1)]
    good = [0]
    for L in range(curves * parts):
        j = L // curves
        good.append(good[-1] + starts[j + 1] - starts[j])
    bad = list(good)
    bad[1] += 1   # one entry moved from list 1 to list 0
    hi = np.arange(n * curves, dtype=np.uint64)
    ids = np.zeros(n * curves, np.uint32)
    p = tmp_path / "off.bin"
    p.write_bytes(F.assemble(F.header(n, 16, curves, 8, partitions=parts), bad, hi, ids))
    assert status(p) == hc.HC_ERR_FORMAT
    # m = 8 needs the low words too: the same offsets but no low section is short
    p.write_bytes(F.assemble(F.header(n, 16, curves, 8, partitions=parts), good, hi, ids))
    assert status(p) == hc.HC_ERR_FORMAT
