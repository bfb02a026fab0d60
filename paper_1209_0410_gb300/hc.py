"""Python binding of libhc.so (include/hc.h): the same entry points, with
torch tensors in place of raw pointers.

Only argument marshalling happens here: every step of the path runs in the
library's CUDA kernels.  torch provides device memory and streams.  There is
no fallback: if libhc.so is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhc.so")

HC_OK, HC_PENDING = 0, 1
HC_ERR_ARG, HC_ERR_OOM, HC_ERR_CUDA, HC_ERR_BUDGET = -1, -2, -3, -4
HC_ERR_TIMEOUT, HC_ERR_DEVICE_STATUS, HC_ERR_STATE = -5, -6, -7
HC_ERR_IO, HC_ERR_FORMAT = -8, -9
HC_U8, HC_F32 = 0, 1


class HCError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (%d)" % (what, hc_strerror(status), status))


class _BuildParams(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d", ctypes.c_uint32), ("curves", ctypes.c_uint32),
                ("dims_per_curve", ctypes.c_uint32), ("bits", ctypes.c_uint32),
                ("dtype", ctypes.c_int), ("dim_map", ctypes.POINTER(ctypes.c_uint32)),
                ("partitions", ctypes.c_uint32)]


class _IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d", ctypes.c_uint32), ("curves", ctypes.c_uint32),
                ("dims_per_curve", ctypes.c_uint32), ("partitions", ctypes.c_uint32),
                ("lists", ctypes.c_uint32), ("dtype", ctypes.c_int),
                ("keys_hi_dev", ctypes.c_void_p), ("keys_lo_dev", ctypes.c_void_p),
                ("ids_dev", ctypes.c_void_p), ("db_dev", ctypes.c_void_p)]


class _ServeParams(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_uint32), ("max_batch_queries", ctypes.c_uint32),
                ("default_p", ctypes.c_uint32), ("max_wait_us", ctypes.c_uint32)]


class _ServeStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batches_done", ctypes.c_uint64), ("queries_done", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint32), ("arena_used", ctypes.c_uint64),
                ("queued_queries", ctypes.c_uint64)]


class _MultiJob(ctypes.Structure):
    _fields_ = [("index", ctypes.c_void_p), ("q_dev", ctypes.c_void_p), ("nq", ctypes.c_uint32),
                ("k", ctypes.c_uint32), ("p", ctypes.c_uint32), ("out_ids_dev", ctypes.c_void_p),
                ("out_dist_dev", ctypes.c_void_p), ("warps_per_query", ctypes.c_uint32)]


class _MultiConfig(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("tile", ctypes.c_uint32), ("use_graph", ctypes.c_uint32)]


_LIB = None
_vp = ctypes.c_void_p
_u32, _u64, _i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32


class _CheckReport(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_uint32), ("site", ctypes.c_uint32),
                ("violations", ctypes.c_uint64), ("index", ctypes.c_uint64),
                ("bound", ctypes.c_uint64)]


def lib():
    """The loaded libhc.so; raises if it is not built."""
    global _LIB
    if _LIB is None:
        _LIB = load_library(LIB_PATH)
    return _LIB


def load_library(path):
    """A libhc build (libhc.so or the bounds-checked libhc_check.so) loaded
    from path with the argument types of every entry point."""
    if not os.path.exists(path):
        raise RuntimeError("%s is not built (%s); run __graft_entry__.build()"
                           % (os.path.basename(path), path))
    L = ctypes.CDLL(path)
    L.hc_strerror.restype = ctypes.c_char_p
    L.hc_strerror.argtypes = [ctypes.c_int]
    L.hc_build.argtypes = [_vp, ctypes.POINTER(_BuildParams), _vp, ctypes.POINTER(_vp)]
    L.hc_build_host.argtypes = [_vp, ctypes.POINTER(_BuildParams), _vp, ctypes.POINTER(_vp)]
    L.hc_build_host_async.argtypes = [_vp, ctypes.POINTER(_BuildParams), _vp, _vp,
                                      ctypes.POINTER(_vp)]
    L.hc_query.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp]
    L.hc_query_host.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp]
    L.hc_query_host_async.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp, _vp]
    L.hc_free.argtypes = [_vp]
    L.hc_free.restype = None
    L.hc_free_async.argtypes = [_vp, _vp]
    L.hc_free_async.restype = None
    L.hc_index_describe.argtypes = [_vp, ctypes.POINTER(_IndexInfo), _vp]
    L.hc_index_copy_lists.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.hc_hilbert_keys.argtypes = [_vp, ctypes.c_int, _u64, _u32, _u32, _u32, _vp, _vp, _vp,
                                  _vp]
    L.hc_sort_keys.argtypes = [_vp, _vp, _vp, _vp, _u32, _u32, _vp]
    L.hc_sort_keys_noalloc.argtypes = [_vp, _vp, _vp, _vp, _u32, _u32, _vp]
    L.hc_query_positions.argtypes = [_vp, _vp, _u32, _vp, _vp]
    L.hc_bruteforce.argtypes = [_vp, ctypes.c_int, _u64, _u32, _vp, _u32, _u32, _vp, _vp, _vp]
    L.hc_query_depths.argtypes = [_vp, _vp, _u32, _u32, _vp, _vp, _vp, _vp]
    L.hc_query_at.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp, _vp]
    L.hc_query_ordered_workspace.restype = ctypes.c_size_t
    L.hc_query_ordered_workspace.argtypes = [_vp, _u32]
    L.hc_query_ordered.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp,
                                   ctypes.c_size_t, _vp]
    L.hc_serve_create_ex.argtypes = [ctypes.POINTER(_vp), _u32, _u64,
                                     ctypes.POINTER(_ServeParams), ctypes.POINTER(_vp)]
    L.hc_serve_create.argtypes = [ctypes.POINTER(_vp), _u32, _u64, ctypes.POINTER(_vp)]
    L.hc_serve_submit.argtypes = [_vp, _u32, _vp, _u32, _u32, _u32,
                                  ctypes.POINTER(ctypes.c_uint64)]
    L.hc_serve_poll.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _u32]
    L.hc_serve_stats_get.argtypes = [_vp, ctypes.POINTER(_ServeStats)]
    L.hc_serve_poll_ex.argtypes = [_vp, ctypes.c_uint64, _vp, _vp, _u32,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.hc_serve_destroy.argtypes = [_vp]
    L.hc_serve_destroy.restype = None
    L.hc_features.argtypes = [_vp, _vp, _u32, _vp, _vp]
    L.hc_probe_labels.argtypes = [_vp, _vp, _u32, _u32, _u32, _vp, _vp]
    L.hc_mlp_create.argtypes = [_u32, _u32, _u32, _u32, ctypes.POINTER(_vp)]
    L.hc_mlp_param_count.argtypes = [_vp]
    L.hc_mlp_param_count.restype = ctypes.c_uint32
    L.hc_mlp_set_params.argtypes = [_vp, _vp, _vp, _vp]
    L.hc_mlp_get_params.argtypes = [_vp, _vp, _vp, _vp]
    L.hc_mlp_gradients.argtypes = [_vp, _vp, _vp, _u32, _vp, _vp, _vp]
    L.hc_mlp_train_step.argtypes = [_vp, _vp, _vp, _u32, ctypes.c_float, _vp, _vp]
    L.hc_mlp_forward.argtypes = [_vp, _vp, _u32, ctypes.c_int, _vp, _vp]
    L.hc_mlp_predict_depths.argtypes = [_vp, _vp, _vp, _u32, ctypes.c_float, _u32, _u32, _vp,
                                        _vp]
    L.hc_mlp_free.argtypes = [_vp]
    L.hc_mlp_free.restype = None
    L.hc_serve_attach_predictor.argtypes = [_vp, _u32, _vp, ctypes.c_float, _u32, _u32]
    L.hc_multi_plan_create.argtypes = [ctypes.POINTER(_MultiJob), _u32,
                                       ctypes.POINTER(_MultiConfig), _vp, ctypes.POINTER(_vp)]
    L.hc_multi_run.argtypes = [_vp, _vp]
    L.hc_multi_plan_free.argtypes = [_vp]
    L.hc_multi_plan_free.restype = None
    L.hc_query_multi.argtypes = [ctypes.POINTER(_MultiJob), _u32, ctypes.POINTER(_MultiConfig),
                                 _vp]
    L.hc_launch_count.argtypes = []
    L.hc_launch_count.restype = ctypes.c_uint64
    L.hc_mlp_fit.argtypes = [_vp, _vp, _vp, _u32, _u32, _u32, ctypes.c_float, _u64, _vp, _vp]
    L.hc_save.argtypes = [_vp, ctypes.c_char_p, _vp]
    L.hc_load.argtypes = [ctypes.c_char_p, _vp, _vp, ctypes.POINTER(_vp)]
    L.hc_debug_fail_alloc.argtypes = [ctypes.c_long]
    L.hc_debug_fail_alloc.restype = None
    L.hc_check_status.argtypes = [ctypes.POINTER(_CheckReport), ctypes.c_int]
    return L


CHECK_LIB_PATH = os.path.join(_HERE, "libhc_check.so")


class use_library:
    """Routes this module's calls to another loaded build for a with-block,
    e.g. ``with hc.use_library(hc.load_library(hc.CHECK_LIB_PATH)):``."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _LIB
        self.saved = _LIB
        _LIB = self.L
        return self.L

    def __exit__(self, *exc):
        global _LIB
        _LIB = self.saved
        return False


def hc_check_status(reset=False):
    """The checked build's report (enabled, site, violations, index, bound)."""
    r = _CheckReport()
    _check(lib().hc_check_status(ctypes.byref(r), 1 if reset else 0), "hc_check_status")
    return dict(enabled=r.enabled, site=r.site, violations=r.violations, index=r.index,
                bound=r.bound)


def hc_strerror(status):
    return lib().hc_strerror(int(status)).decode()


def _check(rc, what):
    if rc != HC_OK:
        raise HCError(rc, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    if t.dtype == torch.uint8:
        return HC_U8
    if t.dtype == torch.float32:
        return HC_F32
    raise TypeError("vectors must be uint8 or float32, got %s" % t.dtype)


def _dev(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _dim_map_arr(dim_map, curves, m):
    if dim_map is None:
        return None, None
    dm = np.ascontiguousarray(np.asarray(dim_map, dtype=np.uint32).reshape(curves * m))
    return dm, dm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class Index:
    """An hc_index handle; keeps the database tensor alive while it exists."""

    def __init__(self, handle, db, params):
        self.handle = handle
        self._lib = lib()   # the build that made it frees it
        self.db = db
        self.dtype = params.dtype
        self.d = params.d
        self.n = params.n
        self.curves = params.curves
        self.m = params.dims_per_curve
        self.partitions = max(1, params.partitions)
        self.lists = self.curves * self.partitions

    def free(self, stream=None):
        """Release the index; with a stream, in stream order on it (hc_free_async)."""
        if self.handle:
            if stream is None:
                self._lib.hc_free(self.handle)
            else:
                self._lib.hc_free_async(self.handle, _stream(stream))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _params(n, d, dtype, curves, m, dim_map, partitions):
    p = _BuildParams()
    p.n, p.d, p.curves, p.dims_per_curve, p.bits = n, d, curves, m, 8
    p.dtype = dtype
    dm, dm_p = _dim_map_arr(dim_map, curves, m)
    p.dim_map = dm_p
    p.partitions = partitions
    return p, dm


def hc_build(db, curves=8, dims_per_curve=16, dim_map=None, partitions=1, stream=None):
    """Algorithm 1 on the GPU over a (n, d) CUDA tensor (not copied)."""
    n, d = db.shape
    p, keep = _params(n, d, _dtype_code(db), curves, dims_per_curve, dim_map, partitions)
    h = ctypes.c_void_p()
    _check(lib().hc_build(_dev(db, "db"), ctypes.byref(p), _stream(stream), ctypes.byref(h)),
           "hc_build")
    del keep
    return Index(h, db, p)


def hc_build_host(db_host, curves=8, dims_per_curve=16, dim_map=None, partitions=1, stream=None):
    """hc_build from a host array (numpy or CPU tensor); the library copies it."""
    arr = db_host.numpy() if isinstance(db_host, torch.Tensor) else np.asarray(db_host)
    arr = np.ascontiguousarray(arr)
    dtype = HC_U8 if arr.dtype == np.uint8 else (HC_F32 if arr.dtype == np.float32 else None)
    if dtype is None:
        raise TypeError("vectors must be uint8 or float32")
    n, d = arr.shape
    p, keep = _params(n, d, dtype, curves, dims_per_curve, dim_map, partitions)
    h = ctypes.c_void_p()
    _check(lib().hc_build_host(arr.ctypes.data_as(_vp), ctypes.byref(p), _stream(stream),
                               ctypes.byref(h)), "hc_build_host")
    del keep
    return Index(h, None, p)


def hc_build_host_async(db_host, curves=8, dims_per_curve=16, dim_map=None, partitions=1,
                        stream=None, copy_stream=None):
    """hc_build_host without waiting: db_host is a pinned CPU tensor, uploaded on
    copy_stream (None: the build stream) while the build waits behind it on
    stream.  The index keeps db_host alive until it is freed."""
    if not isinstance(db_host, torch.Tensor) or db_host.is_cuda or not db_host.is_pinned():
        raise ValueError("db_host must be a pinned CPU tensor")
    if not db_host.is_contiguous():
        raise ValueError("db_host must be contiguous")
    dtype = _dtype_code(db_host)
    n, d = db_host.shape
    p, keep = _params(n, d, dtype, curves, dims_per_curve, dim_map, partitions)
    h = ctypes.c_void_p()
    cs = _stream(copy_stream) if copy_stream is not None else None
    _check(lib().hc_build_host_async(ctypes.c_void_p(db_host.data_ptr()), ctypes.byref(p), cs,
                                     _stream(stream), ctypes.byref(h)), "hc_build_host_async")
    del keep
    idx = Index(h, None, p)
    idx.host_rows = db_host
    return idx


def _dist_dtype(index_dtype):
    return torch.float32 if index_dtype == HC_F32 else torch.int32


def hc_query(index, q, k, p, out_ids=None, out_dist=None, stream=None):
    """Algorithm 2 for a (nq, d) CUDA tensor of queries; returns (ids, dist)."""
    nq = q.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype), device=q.device)
    if nq:
        _check(lib().hc_query(index.handle, _dev(q, "q"), nq, k, p, _dev(out_ids, "out_ids"),
                              _dev(out_dist, "out_dist"), _stream(stream)), "hc_query")
    return out_ids, out_dist


def hc_query_at(index, q, k, p, positions, out_ids=None, out_dist=None, stream=None):
    """hc_query with positions from hc_query_positions ((nq, lists) int64)."""
    nq = q.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype), device=q.device)
    if nq:
        _check(lib().hc_query_at(index.handle, _dev(q, "q"), nq, k, p, _dev(positions, "pos"),
                                 _dev(out_ids, "out_ids"), _dev(out_dist, "out_dist"),
                                 _stream(stream)), "hc_query_at")
    return out_ids, out_dist


def hc_query_ordered_workspace(index, nq):
    """Bytes of device workspace hc_query_ordered needs for nq queries on
    this index (on any index of the same curves and lists)."""
    return int(lib().hc_query_ordered_workspace(index.handle, nq))


def hc_query_ordered(index, q, k, p, out_ids=None, out_dist=None, workspace=None, stream=None):
    """hc_query answering the queries in curve-0 key order, their lower_bound
    positions found first by one batch pass (results identical); workspace: a
    CUDA uint8 tensor of at least hc_query_ordered_workspace(index, nq) bytes
    (allocated here when None)."""
    nq = q.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype), device=q.device)
    if nq:
        need = hc_query_ordered_workspace(index, nq)
        if workspace is None:
            workspace = torch.empty(need, dtype=torch.uint8, device=q.device)
        _check(lib().hc_query_ordered(index.handle, _dev(q, "q"), nq, k, p,
                                      _dev(out_ids, "out_ids"), _dev(out_dist, "out_dist"),
                                      _dev(workspace, "workspace"), workspace.numel(),
                                      _stream(stream)), "hc_query_ordered")
    return out_ids, out_dist


def hc_query_depths(index, q, k, p_per_query, out_ids=None, out_dist=None, stream=None):
    """hc_query with one depth per query (a (nq,) int32/uint32 CUDA tensor)."""
    nq = q.shape[0]
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype), device=q.device)
    if nq:
        _check(lib().hc_query_depths(index.handle, _dev(q, "q"), nq, k, _dev(p_per_query, "p"),
                                     _dev(out_ids, "out_ids"), _dev(out_dist, "out_dist"),
                                     _stream(stream)), "hc_query_depths")
    return out_ids, out_dist


def hc_query_host(index, q_host, k, p, out_ids=None, out_dist=None, stream=None):
    """hc_query from host buffers (numpy or CPU tensors, pinned or not)."""
    if isinstance(q_host, torch.Tensor):
        qa = q_host
        nq = qa.shape[0]
        qptr = qa.data_ptr()
    else:
        qa = np.ascontiguousarray(q_host)
        nq = qa.shape[0]
        qptr = qa.ctypes.data
    if out_ids is None:
        out_ids = torch.empty((nq, k), dtype=torch.int32)
    if out_dist is None:
        out_dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype))
    if nq:
        _check(lib().hc_query_host(index.handle, ctypes.c_void_p(qptr), nq, k, p,
                                   ctypes.c_void_p(out_ids.data_ptr()),
                                   ctypes.c_void_p(out_dist.data_ptr()), _stream(stream)),
               "hc_query_host")
    return out_ids, out_dist


def hc_query_host_async(index, q_host, k, p, out_ids, out_dist, stream=None,
                        copy_stream=None):
    """hc_query_host without waiting: pinned CPU tensors in and out; the results
    are valid once `stream` reaches this point."""
    for t, name in ((q_host, "q_host"), (out_ids, "out_ids"), (out_dist, "out_dist")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_pinned() or \
                not t.is_contiguous():
            raise ValueError("%s must be a contiguous pinned CPU tensor" % name)
    nq = q_host.shape[0]
    if nq:
        cs = _stream(copy_stream) if copy_stream is not None else None
        _check(lib().hc_query_host_async(index.handle, ctypes.c_void_p(q_host.data_ptr()), nq,
                                         k, p, ctypes.c_void_p(out_ids.data_ptr()),
                                         ctypes.c_void_p(out_dist.data_ptr()), cs,
                                         _stream(stream)), "hc_query_host_async")
    return out_ids, out_dist


def hc_free(index):
    index.free()


def hc_index_describe(index):
    """(info dict, list_off numpy array); the device arrays stay owned by the index."""
    info = _IndexInfo()
    off = np.zeros(index.lists + 1, np.uint64)
    _check(lib().hc_index_describe(index.handle, ctypes.byref(info), off.ctypes.data_as(_vp)),
           "hc_index_describe")
    d = {f: getattr(info, f) for f, _ in _IndexInfo._fields_}
    return d, off


def hc_index_copy_lists(index, stream=None):
    """Copies of the sorted lists: (keys_hi, keys_lo, ids) as CUDA tensors
    (int64, int64, int32; the key words are uint64 bit patterns) and the list
    offsets (numpy uint64)."""
    info, off = hc_index_describe(index)
    total = int(off[-1])
    hi = torch.empty(total, dtype=torch.int64, device="cuda")
    lo = torch.empty(total, dtype=torch.int64, device="cuda")
    ids = torch.empty(total, dtype=torch.int32, device="cuda")
    if total:
        _check(lib().hc_index_copy_lists(index.handle, _dev(hi, "hi"), _dev(lo, "lo"),
                                         _dev(ids, "ids"), _stream(stream)),
               "hc_index_copy_lists")
    return hi, lo, ids, off


def hc_save(index, path, stream=None):
    """Writes the index's sorted lists to a file (the rows are not written)."""
    _check(lib().hc_save(index.handle, os.fsencode(path), _stream(stream)), "hc_save")


def hc_load(path, db, stream=None):
    """An index from a file hc_save wrote, over the (n, d) CUDA tensor it indexes."""
    h = ctypes.c_void_p()
    _check(lib().hc_load(os.fsencode(path), _dev(db, "db"), _stream(stream), ctypes.byref(h)),
           "hc_load")
    info = _IndexInfo()
    _check(lib().hc_index_describe(h, ctypes.byref(info), None), "hc_index_describe")
    p = _BuildParams()
    p.n, p.d, p.curves, p.dims_per_curve, p.bits = info.n, info.d, info.curves, \
        info.dims_per_curve, 8
    p.dtype, p.partitions = info.dtype, info.partitions
    return Index(h, db, p)


def hc_hilbert_keys(x, curves, dims_per_curve, dim_map=None, stream=None):
    """Extended-keys of every (vector, curve): two (count, curves) int64
    tensors holding the uint64 words (hi, lo)."""
    count, d = x.shape
    hi = torch.empty((count, curves), dtype=torch.int64, device=x.device)
    lo = torch.empty((count, curves), dtype=torch.int64, device=x.device)
    dm, dm_p = _dim_map_arr(dim_map, curves, dims_per_curve)
    if count:
        _check(lib().hc_hilbert_keys(_dev(x, "x"), _dtype_code(x), count, d, curves,
                                     dims_per_curve, dm_p, _dev(hi, "hi"), _dev(lo, "lo"),
                                     _stream(stream)), "hc_hilbert_keys")
    del dm
    return hi, lo


def hc_sort_keys(hi, lo, ids, seg_off, key_bits=128, stream=None):
    """Stable in-place radix sort by 128-bit key within segments."""
    off = np.ascontiguousarray(np.asarray(seg_off, dtype=np.uint64))
    _check(lib().hc_sort_keys(_dev(hi, "hi"), _dev(lo, "lo"), _dev(ids, "ids"),
                              off.ctypes.data_as(_vp), len(off) - 1, key_bits, _stream(stream)),
           "hc_sort_keys")


def hc_sort_keys_noalloc(hi, lo, ids, seg_off, key_bits=128, stream=None):
    """hc_sort_keys without any device allocation by the library (scratch is a
    fixed array inside libhc.so; at most 262,144 records and 256 segments).
    Asynchronous on the stream, unlike hc_sort_keys."""
    off = np.ascontiguousarray(np.asarray(seg_off, dtype=np.uint64))
    _check(lib().hc_sort_keys_noalloc(_dev(hi, "hi"), _dev(lo, "lo"), _dev(ids, "ids"),
                                      off.ctypes.data_as(_vp), len(off) - 1, key_bits,
                                      _stream(stream)), "hc_sort_keys_noalloc")


def hc_query_positions(index, q, stream=None):
    """lower_bound position of each query in each list: (nq, lists) int64."""
    nq = q.shape[0]
    pos = torch.empty((nq, index.lists), dtype=torch.int64, device=q.device)
    if nq:
        _check(lib().hc_query_positions(index.handle, _dev(q, "q"), nq, _dev(pos, "pos"),
                                        _stream(stream)), "hc_query_positions")
    return pos


def hc_bruteforce(db, q, k, stream=None):
    """Exact kNN (Eq. 3) on the GPU: (ids, dist)."""
    n, d = db.shape
    nq = q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
    dist = torch.empty((nq, k), dtype=_dist_dtype(_dtype_code(db)), device=q.device)
    if nq:
        _check(lib().hc_bruteforce(_dev(db, "db"), _dtype_code(db), n, d, _dev(q, "q"), nq, k,
                                   _dev(ids, "ids"), _dev(dist, "dist"), _stream(stream)),
               "hc_bruteforce")
    return ids, dist


def hc_launch_count():
    """Kernel launches issued by the library since it was loaded."""
    return int(lib().hc_launch_count())


def hc_debug_fail_alloc(after):
    lib().hc_debug_fail_alloc(int(after))


# ------------------------------------------------------------------ serving
class Server:
    """An hc_server: continuous batching over resident indexes (see hc.h)."""

    def __init__(self, indexes, hbm_budget, streams=4, max_batch_queries=16384, default_p=128,
                 max_wait_us=200):
        self.indexes = list(indexes)      # keep them alive while serving
        arr = (_vp * len(self.indexes))(*[ix.handle for ix in self.indexes])
        prm = _ServeParams(streams, max_batch_queries, default_p, max_wait_us)
        h = ctypes.c_void_p()
        _check(lib().hc_serve_create_ex(arr, len(self.indexes), hbm_budget, ctypes.byref(prm),
                                        ctypes.byref(h)), "hc_serve_create")
        self.handle = h
        self._meta = {}

    def submit(self, index_id, q, k, p):
        """Queues a (nq, d) host array of queries; returns the ticket."""
        q = np.ascontiguousarray(q)
        t = ctypes.c_uint64()
        _check(lib().hc_serve_submit(self.handle, index_id, q.ctypes.data_as(_vp), q.shape[0], k,
                                     p, ctypes.byref(t)), "hc_serve_submit")
        dt = np.float32 if self.indexes[index_id].dtype == HC_F32 else np.int32
        self._meta[t.value] = (q.shape[0], k, dt)
        return t.value

    def poll(self, ticket, timeout_us=0, with_latency=False):
        """(ids, dist) numpy arrays when done (plus the latency in seconds
        with with_latency), None while pending."""
        nq, k, dt = self._meta[ticket]
        ids = np.empty((nq, k), np.int32)
        dist = np.empty((nq, k), dt)
        lat = ctypes.c_uint64()
        rc = lib().hc_serve_poll_ex(self.handle, ticket, ids.ctypes.data_as(_vp),
                                    dist.ctypes.data_as(_vp), timeout_us, ctypes.byref(lat))
        if rc == HC_PENDING:
            return None
        del self._meta[ticket]
        _check(rc, "hc_serve_poll")
        if with_latency:
            return ids, dist, lat.value * 1e-9
        return ids, dist

    def attach_predictor(self, index_id, mlp, margin=0.0, p_lo=1, p_hi=512):
        """Requests submitted with p = 0 get learned per-query depths."""
        self._pred = getattr(self, "_pred", {})
        self._pred[index_id] = mlp
        _check(lib().hc_serve_attach_predictor(self.handle, index_id,
                                               mlp.handle if mlp is not None else None, margin,
                                               p_lo, p_hi), "hc_serve_attach_predictor")

    def stats(self):
        st = _ServeStats()
        _check(lib().hc_serve_stats_get(self.handle, ctypes.byref(st)), "hc_serve_stats_get")
        return {f: getattr(st, f) for f, _ in _ServeStats._fields_}

    def close(self):
        if self.handle:
            lib().hc_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hc_serve_create(indexes, hbm_budget, **params):
    return Server(indexes, hbm_budget, **params)


def hc_serve_submit(server, index_id, q_host, k, p):
    return server.submit(index_id, q_host, k, p)


def hc_serve_poll(server, ticket, timeout_us=0):
    return server.poll(ticket, timeout_us)


def hc_serve_destroy(server):
    server.close()


# ------------------------------------------------------ learned probe depth
def hc_features(index, q, stream=None):
    """(nq, 4*curves) float32 CUDA tensor of depth-predictor features."""
    nq = q.shape[0]
    feat = torch.empty((nq, 4 * index.curves), dtype=torch.float32, device=q.device)
    if nq:
        _check(lib().hc_features(index.handle, _dev(q, "q"), nq, _dev(feat, "feat"),
                                 _stream(stream)), "hc_features")
    return feat


def hc_probe_labels(index, q, k, p_max, stream=None):
    """(nq,) int32 CUDA tensor: minimal depth reproducing the top-k at p_max."""
    nq = q.shape[0]
    out = torch.empty(nq, dtype=torch.int32, device=q.device)
    if nq:
        _check(lib().hc_probe_labels(index.handle, _dev(q, "q"), nq, k, p_max, _dev(out, "out"),
                                     _stream(stream)), "hc_probe_labels")
    return out


class MLP:
    """hc_mlp: in -> h1 -> h2 -> 1 regressor with device-side Adam training."""

    def __init__(self, n_in, h1=64, h2=64, max_batch=4096):
        h = ctypes.c_void_p()
        _check(lib().hc_mlp_create(n_in, h1, h2, max_batch, ctypes.byref(h)), "hc_mlp_create")
        self.handle = h
        self.n_in, self.h1, self.h2, self.max_batch = n_in, h1, h2, max_batch
        self.nparam = int(lib().hc_mlp_param_count(h))

    def set_params(self, theta, mu, isd):
        t = np.ascontiguousarray(theta, np.float32)
        m = np.ascontiguousarray(mu, np.float32)
        i = np.ascontiguousarray(isd, np.float32)
        assert t.size == self.nparam and m.size == self.n_in and i.size == self.n_in
        _check(lib().hc_mlp_set_params(self.handle, t.ctypes.data_as(_vp), m.ctypes.data_as(_vp),
                                       i.ctypes.data_as(_vp)), "hc_mlp_set_params")

    def get_params(self):
        t = np.empty(self.nparam, np.float32)
        m = np.empty(self.n_in, np.float32)
        i = np.empty(self.n_in, np.float32)
        _check(lib().hc_mlp_get_params(self.handle, t.ctypes.data_as(_vp), m.ctypes.data_as(_vp),
                                       i.ctypes.data_as(_vp)), "hc_mlp_get_params")
        return t, m, i

    def gradients(self, x, t, stream=None):
        g = torch.empty(self.nparam, dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        _check(lib().hc_mlp_gradients(self.handle, _dev(x, "x"), _dev(t, "t"), x.shape[0],
                                      _dev(g, "g"), ctypes.byref(loss), _stream(stream)),
               "hc_mlp_gradients")
        return g, loss.value

    def train_step(self, x, t, lr, want_loss=False, stream=None):
        loss = ctypes.c_float()
        _check(lib().hc_mlp_train_step(self.handle, _dev(x, "x"), _dev(t, "t"), x.shape[0], lr,
                                       ctypes.byref(loss) if want_loss else None,
                                       _stream(stream)), "hc_mlp_train_step")
        return loss.value if want_loss else None

    def fit(self, feats, labels, epochs, batch, lr, seed=0, stream=None):
        """hc_mlp_fit: trains on (n, in) features and n depth labels on the
        device; returns the mean loss per epoch."""
        n = feats.shape[0]
        losses = np.zeros(epochs, np.float32)
        _check(lib().hc_mlp_fit(self.handle, _dev(feats, "feats"),
                                _dev(labels.contiguous(), "labels"), n,
                                epochs, batch, lr, seed, losses.ctypes.data_as(_vp),
                                _stream(stream)), "hc_mlp_fit")
        return [float(x) for x in losses]

    def forward(self, x, bf16=False, stream=None):
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        if x.shape[0]:
            _check(lib().hc_mlp_forward(self.handle, _dev(x, "x"), x.shape[0], 1 if bf16 else 0,
                                        _dev(y, "y"), _stream(stream)), "hc_mlp_forward")
        return y

    def predict_depths(self, index, q, margin=0.0, p_lo=1, p_hi=512, stream=None):
        nq = q.shape[0]
        p = torch.empty(nq, dtype=torch.int32, device=q.device)
        if nq:
            _check(lib().hc_mlp_predict_depths(self.handle, index.handle, _dev(q, "q"), nq,
                                               margin, p_lo, p_hi, _dev(p, "p"), _stream(stream)),
                   "hc_mlp_predict_depths")
        return p

    def free(self):
        if self.handle:
            lib().hc_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hc_mlp_create(n_in, h1=64, h2=64, max_batch=4096):
    return MLP(n_in, h1, h2, max_batch)


# ---------------------------------------------- many indexes, one launch
class MultiJob:
    """One hc_query inside a persistent multi-index launch; owns its outputs."""

    def __init__(self, index, q, k, p, warps_per_query=1):
        self.index, self.q, self.k, self.p = index, q, k, p
        self.warps_per_query = warps_per_query
        nq = q.shape[0]
        self.ids = torch.empty((nq, k), dtype=torch.int32, device=q.device)
        self.dist = torch.empty((nq, k), dtype=_dist_dtype(index.dtype), device=q.device)

    def _c(self):
        nq = self.q.shape[0]
        return _MultiJob(self.index.handle.value, self.q.data_ptr() if nq else 0, nq, self.k,
                         self.p, self.ids.data_ptr() if nq else 0,
                         self.dist.data_ptr() if nq else 0, self.warps_per_query)


def _multi_arrays(jobs, config):
    arr = (_MultiJob * len(jobs))(*[j._c() for j in jobs])
    cfg = None
    if config is not None:
        cfg = _MultiConfig(config.get("warps_per_block", 8), config.get("blocks_per_sm", 4),
                           config.get("tile", 2), 1 if config.get("use_graph", True) else 0)
    return arr, cfg


class MultiPlan:
    """hc_multi_plan: a persistent launch over many jobs, optionally a CUDA graph."""

    def __init__(self, jobs, config=None, stream=None):
        self.jobs = list(jobs)
        arr, cfg = _multi_arrays(self.jobs, config)
        h = ctypes.c_void_p()
        _check(lib().hc_multi_plan_create(arr, len(self.jobs),
                                          ctypes.byref(cfg) if cfg is not None else None,
                                          _stream(stream), ctypes.byref(h)),
               "hc_multi_plan_create")
        self.handle = h

    def run(self, stream=None):
        _check(lib().hc_multi_run(self.handle, _stream(stream)), "hc_multi_run")

    def free(self):
        if self.handle:
            lib().hc_multi_plan_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hc_query_multi(jobs, config=None, stream=None):
    """Answers every job in one persistent launch (no graph); returns when done."""
    arr, cfg = _multi_arrays(jobs, config)
    _check(lib().hc_query_multi(arr, len(jobs), ctypes.byref(cfg) if cfg is not None else None,
                                _stream(stream)), "hc_query_multi")
    return jobs
