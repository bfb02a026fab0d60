"""hc_sort_keys_noalloc against hc_sort_keys, through the C ABI.

hc_sort_keys_noalloc serves callers that cannot let the library allocate
device memory (a memory manager that already reserved the whole GPU, or code
that cannot take the device synchronisation of cudaMalloc/cudaFree); its
scratch is a fixed array inside libhc.so.  The sort is integer work, so the
two entry points must agree bit for bit.  Two calls in a row with different
data show that what the first call leaves in the shared scratch does not leak
into the second.  This file is collected last on purpose, so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from helpers import u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_0410_gb300 import hc as _hc
    _hc.lib()
    return _hc


def random_records(seed, sizes, dup_pool=None):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    total = int(off[-1])
    hi = rng.integers(0, 2**63, size=total, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=total, dtype=np.uint64)
    lo = rng.integers(0, 2**63, size=total, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=total, dtype=np.uint64)
    if dup_pool:
        pick = rng.integers(0, dup_pool, size=total)
        hi, lo = hi[:dup_pool][pick], lo[:dup_pool][pick]
    ids = rng.permutation(total).astype(np.uint32)
    return off, hi, lo, ids


def to_dev(hi, lo, ids):
    import torch
    return (torch.from_numpy(hi.view(np.int64)).cuda(), torch.from_numpy(lo.view(np.int64)).cuda(),
            torch.from_numpy(ids.view(np.int32)).cuda())


def test_noalloc_matches_allocating_sort_twice(hc):
    import torch
    cases = [dict(seed=1, sizes=[100_000, 4097, 0, 33, 60_000]),
             dict(seed=2, sizes=[262_144 - 5000, 5000], dup_pool=101)]
    for c in cases:                                   # two calls in a row
        off, hi, lo, ids = random_records(c["seed"], c["sizes"], c.get("dup_pool"))
        a = to_dev(hi, lo, ids)
        b = to_dev(hi, lo, ids)
        hc.hc_sort_keys(*a, off, 128)
        hc.hc_sort_keys_noalloc(*b, off, 128)
        torch.cuda.synchronize()
        assert np.array_equal(u64(a[0]), u64(b[0]))
        assert np.array_equal(u64(a[1]), u64(b[1]))
        assert np.array_equal(a[2].cpu().numpy(), b[2].cpu().numpy())
        # and both are the stable order by key
        for s in range(len(c["sizes"])):
            x, y = int(off[s]), int(off[s + 1])
            order = np.lexsort((np.arange(y - x), lo[x:y], hi[x:y]))
            assert np.array_equal(u64(b[0])[x:y], hi[x:y][order])
            assert np.array_equal(b[2].cpu().numpy().view(np.uint32)[x:y], ids[x:y][order])


def test_noalloc_at_its_limits_allocates_nothing(hc):
    """The largest problem within both limits -- 255 one-record segments and
    one segment of the rest, 262,144 records in all -- needs nearly the whole
    scratch array; it sorts like hc_sort_keys.  After a first call (which
    loads the array on the device), a further call leaves the device's free
    memory unchanged: the library allocated nothing."""
    import torch
    sizes = [1] * 255 + [262_144 - 255]
    off, hi, lo, ids = random_records(4, sizes)
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    hc.hc_sort_keys_noalloc(empty, empty, empty.to(torch.int32), np.zeros(2, np.uint64), 128)
    a = to_dev(hi, lo, ids)
    b = to_dev(hi, lo, ids)
    c = to_dev(hi, lo, ids)
    hc.hc_sort_keys(*a, off, 128)
    hc.hc_sort_keys_noalloc(*b, off, 128)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    hc.hc_sort_keys_noalloc(*c, off, 128)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for t in (b, c):
        assert np.array_equal(u64(a[0]), u64(t[0]))
        assert np.array_equal(u64(a[1]), u64(t[1]))
        assert np.array_equal(a[2].cpu().numpy(), t[2].cpu().numpy())


def test_noalloc_rejects_problems_above_its_limit(hc):
    off, hi, lo, ids = random_records(3, [262_145])
    t = to_dev(hi, lo, ids)
    with pytest.raises(hc.HCError) as e:
        hc.hc_sort_keys_noalloc(*t, off, 128)
    assert e.value.status == hc.HC_ERR_ARG
    off = np.arange(258, dtype=np.uint64)             # 257 segments of one record
    with pytest.raises(hc.HCError) as e:
        hc.hc_sort_keys_noalloc(*t, off, 128)
    assert e.value.status == hc.HC_ERR_ARG
