"""Python face of the CPU oracle (oracle/hc_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use this module; the library's product path never imports it.
It shares no code with the CUDA path: arrays go in as numpy buffers and come
back as numpy buffers.

Each function follows a passage of arXiv:1209.0410:
  hilbert_keys / hilbert_axes  -- extended-key C^-1 and its inverse (Sec. 2.2.1)
  build                        -- Algorithm 1 (per partition for Hypercurves)
  search                       -- Algorithm 2; with ell > 1 the local answers
                                  are reduced as the Aggregator does (Sec. 4.1)
  bruteforce                   -- exact kNN, Eq. 3
  binom_tail / equiv_bound     -- the equivalence bound of Sec. 4.2 (Eq. 6)
"""
import ctypes
import os

import numpy as np

from . import build as _build  # noqa: F401  (package-relative when imported as oracle.oracle)

_LIB = None
U8, F32 = 0, 1

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build_oracle()
        lib = ctypes.CDLL(path)
        lib.orc_hilbert_keys_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                               _u32p, _u64p, _u64p]
        lib.orc_hilbert_axes_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                               _u64p, _u64p, _u32p]
        lib.orc_quantize_batch.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_uint64, _u32p]
        lib.orc_build.argtypes = [ctypes.c_int, _vp, ctypes.c_uint64, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32, _u32p,
                                  _u64p, _u64p, _u64p, _u32p, ctypes.c_int]
        lib.orc_search.argtypes = [ctypes.c_int, _vp, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                   _u64p, _u64p, _u64p, _u32p, _vp, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_uint32, _i32p, _f64p, _i64p,
                                   ctypes.c_int]
        lib.orc_query_keys.argtypes = [ctypes.c_int, _vp, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, _u32p, _u64p, _u64p]
        lib.orc_bruteforce.argtypes = [ctypes.c_int, _vp, ctypes.c_uint64, ctypes.c_uint32, _vp,
                                       ctypes.c_uint64, ctypes.c_uint32, _i32p, _f64p, ctypes.c_int]
        lib.orc_binom_tail.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_binom_tail.restype = ctypes.c_double
        lib.orc_equiv_bound.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_double]
        lib.orc_equiv_bound.restype = ctypes.c_double
        lib.orc_slack_depth.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double]
        lib.orc_slack_depth.restype = ctypes.c_uint32
        lib.orc_features.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, _u32p, _u64p, _u64p, _u64p, _u32p, _vp,
                                     ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]
        lib.orc_octave.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_octave.restype = ctypes.c_double
        _LIB = lib
    return _LIB


def _ptr(a, typ):
    return a.ctypes.data_as(typ)


def _dtype_code(a):
    if a.dtype == np.uint8:
        return U8
    if a.dtype == np.float32:
        return F32
    raise TypeError("oracle handles uint8 and float32 vectors, got %s" % a.dtype)


def _dim_map_arg(dim_map):
    if dim_map is None:
        return None, None
    dm = np.ascontiguousarray(dim_map, dtype=np.uint32).ravel()
    return dm, _ptr(dm, _u32p)


def default_threads():
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- Hilbert map
def hilbert_keys(n, b, axes):
    """Extended-keys of points: axes is (count, n) with coordinates < 2**b.
    Returns (hi, lo) uint64 arrays holding the n*b-bit key right-aligned."""
    ax = np.ascontiguousarray(axes, dtype=np.uint32).reshape(-1, n)
    cnt = ax.shape[0]
    hi = np.zeros(cnt, np.uint64)
    lo = np.zeros(cnt, np.uint64)
    rc = _lib().orc_hilbert_keys_batch(n, b, cnt, _ptr(ax, _u32p), _ptr(hi, _u64p), _ptr(lo, _u64p))
    if rc != 0:
        raise ValueError("unsupported Hilbert shape n=%d b=%d" % (n, b))
    return hi, lo


def hilbert_axes(n, b, hi, lo):
    """Inverse of hilbert_keys."""
    hi = np.ascontiguousarray(hi, dtype=np.uint64).ravel()
    lo = np.ascontiguousarray(lo, dtype=np.uint64).ravel()
    ax = np.zeros((hi.shape[0], n), np.uint32)
    rc = _lib().orc_hilbert_axes_batch(n, b, hi.shape[0], _ptr(hi, _u64p), _ptr(lo, _u64p),
                                       _ptr(ax, _u32p))
    if rc != 0:
        raise ValueError("unsupported Hilbert shape n=%d b=%d" % (n, b))
    return ax


def key_int(hi, lo):
    """Python int of one 128-bit key."""
    return (int(hi) << 64) | int(lo)


def quantize(x):
    """Float32 coordinates -> 8-bit key coordinates (decided in float32)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape, np.uint32)
    _lib().orc_quantize_batch(_ptr(x.ravel(), ctypes.POINTER(ctypes.c_float)), x.size,
                              _ptr(out.ravel(), _u32p))
    return out


# ------------------------------------------------------- Algorithms 1 and 2
class Index:
    """ell*curves sorted lists of (key, id); list L = part*curves + curve."""

    def __init__(self, dtype, n, d, curves, m, dim_map, ell, list_off, keys_hi, keys_lo, ids):
        self.dtype, self.n, self.d = dtype, n, d
        self.curves, self.m, self.ell = curves, m, ell
        self.dim_map = dim_map
        self.list_off, self.keys_hi, self.keys_lo, self.ids = list_off, keys_hi, keys_lo, ids

    @property
    def lists(self):
        return self.ell * self.curves

    def list_slice(self, L):
        return slice(int(self.list_off[L]), int(self.list_off[L + 1]))


def build(db, curves, m, dim_map=None, ell=1, part_of=None, nthreads=None):
    """Algorithm 1 (run per partition when ell > 1)."""
    db = np.ascontiguousarray(db)
    n, d = db.shape
    code = _dtype_code(db)
    dm, dm_p = _dim_map_arg(dim_map)
    po = None
    po_p = None
    if part_of is not None:
        po = np.ascontiguousarray(part_of, dtype=np.uint32)
        po_p = _ptr(po, _u32p)
    lists = ell * curves
    list_off = np.zeros(lists + 1, np.uint64)
    keys_hi = np.zeros(n * curves, np.uint64)
    keys_lo = np.zeros(n * curves, np.uint64)
    ids = np.zeros(n * curves, np.uint32)
    rc = _lib().orc_build(code, db.ctypes.data, n, d, curves, m, dm_p, ell, po_p,
                          _ptr(list_off, _u64p), _ptr(keys_hi, _u64p), _ptr(keys_lo, _u64p),
                          _ptr(ids, _u32p), nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_build failed (%d)" % rc)
    return Index(code, n, d, curves, m, dm, ell, list_off, keys_hi, keys_lo, ids)


def search(index, db, queries, k, p, nthreads=None, return_pos=False):
    """Algorithm 2 at depth p per side in every list (Hypercurves reduction
    across partitions).  Returns (ids int32 (nq,k), dist float64 (nq,k)) and,
    with return_pos, the (nq, lists) lower_bound positions."""
    db = np.ascontiguousarray(db)
    queries = np.ascontiguousarray(queries, dtype=db.dtype)
    nq = queries.shape[0]
    out_ids = np.zeros((nq, k), np.int32)
    out_dist = np.zeros((nq, k), np.float64)
    pos = np.zeros((nq, index.lists), np.int64) if return_pos else None
    dm_p = _ptr(index.dim_map, _u32p) if index.dim_map is not None else None
    rc = _lib().orc_search(index.dtype, db.ctypes.data, index.n, index.d, index.curves, index.m,
                           dm_p, index.ell, _ptr(index.list_off, _u64p),
                           _ptr(index.keys_hi, _u64p), _ptr(index.keys_lo, _u64p),
                           _ptr(index.ids, _u32p), queries.ctypes.data, nq, k, p,
                           _ptr(out_ids, _i32p), _ptr(out_dist, _f64p),
                           _ptr(pos, _i64p) if pos is not None else None,
                           nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_search failed (%d)" % rc)
    if return_pos:
        return out_ids, out_dist, pos
    return out_ids, out_dist


def query_keys(queries, curves, m, dim_map=None):
    """Extended-keys of every (query, curve): two (nq, curves) uint64 arrays."""
    queries = np.ascontiguousarray(queries)
    nq, d = queries.shape
    hi = np.zeros((nq, curves), np.uint64)
    lo = np.zeros((nq, curves), np.uint64)
    dm, dm_p = _dim_map_arg(dim_map)
    rc = _lib().orc_query_keys(_dtype_code(queries), queries.ctypes.data, nq, d, curves, m, dm_p,
                               _ptr(hi, _u64p), _ptr(lo, _u64p))
    if rc != 0:
        raise ValueError("orc_query_keys failed")
    return hi, lo


def bruteforce(db, queries, k, nthreads=None):
    """Exact kNN (Eq. 3), ties by lower id, padded with (-1, +inf)."""
    db = np.ascontiguousarray(db)
    queries = np.ascontiguousarray(queries, dtype=db.dtype)
    n, d = db.shape
    nq = queries.shape[0]
    out_ids = np.zeros((nq, k), np.int32)
    out_dist = np.zeros((nq, k), np.float64)
    rc = _lib().orc_bruteforce(_dtype_code(db), db.ctypes.data, n, d, queries.ctypes.data, nq, k,
                               _ptr(out_ids, _i32p), _ptr(out_dist, _f64p),
                               nthreads or default_threads())
    if rc != 0:
        raise ValueError("orc_bruteforce failed (%d)" % rc)
    return out_ids, out_dist


# ------------------------------------------------- equivalence (Sec. 4.2)
def binom_tail(Phi, ell, phi):
    """P(Bin(Phi, 1/ell) > phi)."""
    return _lib().orc_binom_tail(Phi, ell, phi)


def equiv_bound(Phi, ell, phi, mult=None):
    """Upper bound of Eq. 6 on missing a window entry; mult defaults to Phi
    (the multiplier as printed)."""
    return _lib().orc_equiv_bound(Phi, ell, phi, float(Phi if mult is None else mult))


def slack_depth(Phi, ell, slack):
    """phi = ceil((1 + slack) * ceil(Phi / ell))."""
    return _lib().orc_slack_depth(Phi, ell, float(slack))


# --------------------------------------------------------------- utilities
def int32_dist(dist):
    """uint8 distances as int32 with +inf padding mapped to INT32_MAX."""
    out = np.where(np.isinf(dist), np.iinfo(np.int32).max, dist)
    return out.astype(np.int64).astype(np.int32)


def recall_at(ids, dist, true_dist, k=10):
    """Tie-aware recall@k: fraction of returned entries whose distance is at
    most the true k-th nearest distance (capped at k per query)."""
    kth = true_dist[:, k - 1:k]
    ok = (dist[:, :k] <= kth) & (ids[:, :k] >= 0)
    hits = np.minimum(ok.sum(axis=1), k)
    return float(hits.mean() / k)


# -------------------------------------------- learned probe depth features
FEAT_NONE = 130.0


def octave(g):
    """Octave encoding of a non-negative integer below 2**128 (see hc_oracle.c)."""
    g = int(g)
    return _lib().orc_octave((g >> 64) & (2**64 - 1), g & (2**64 - 1))


def features(index, db, queries):
    """(nq, 4*curves) float32 features of uint8 queries (partition 0 lists)."""
    db = np.ascontiguousarray(db)
    queries = np.ascontiguousarray(queries, dtype=np.uint8)
    if index.dtype != U8 or index.ell != 1:
        raise ValueError("features are defined for uint8, single-partition indexes")
    nq = queries.shape[0]
    feat = np.zeros((nq, 4 * index.curves), np.float32)
    dm_p = _ptr(index.dim_map, _u32p) if index.dim_map is not None else None
    rc = _lib().orc_features(db.ctypes.data, index.n, index.d, index.curves, index.m, dm_p,
                             _ptr(index.list_off, _u64p), _ptr(index.keys_hi, _u64p),
                             _ptr(index.keys_lo, _u64p), _ptr(index.ids, _u32p),
                             queries.ctypes.data, nq,
                             feat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise ValueError("orc_features failed")
    return feat


def min_depth_labels(index, db, queries, k, p_max, nthreads=None):
    """Minimal p in [0, p_max] whose top-k equals the top-k at p_max, by
    direct search over p (valid because results are monotone in p)."""
    ref_ids, _ = search(index, db, queries, k, p_max, nthreads)
    nq = queries.shape[0]
    lo = np.zeros(nq, np.int64)            # top-k(lo) may differ
    hi = np.full(nq, p_max, np.int64)      # top-k(hi) equals the reference
    while True:
        active = lo < hi
        if not active.any():
            break
        mid = (lo + hi) // 2
        for p in np.unique(mid[active]):
            sel = np.nonzero(active & (mid == p))[0]
            ids, _ = search(index, db, queries[sel], k, int(p), nthreads)
            same = (ids == ref_ids[sel]).all(axis=1)
            hi[sel[same]] = p
            lo[sel[~same]] = p + 1
    return hi
