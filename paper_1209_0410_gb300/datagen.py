"""Seeded synthetic inputs (a module of its own: no arithmetic of the method).

The database and query vectors stand in for the 128-d SIFT descriptors the
paper measures on (Sec. 7): a mixture of isotropic Gaussian clusters, rounded
half-to-even and clipped to [0, 255]; queries are database rows plus Gaussian
noise.  Both the CPU oracle and the CUDA path consume these bytes.  The draws
come from a counter-based SplitMix64 generator, so every byte depends only on
(seed, stream, index) and not on the thread count.
"""
import ctypes
import os

import numpy as np

from . import _build

_LIB = None

# seeds of the standard workloads
SEED_DB = 1
SEED_QUERIES = 3
SEED_TRAIN_QUERIES = 4
SEED_HELDOUT_QUERIES = 5

N_CLUSTERS = 64
SIGMA_DB = 20.0
SIGMA_QUERY = 8.0


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build_datagen()
        lib = ctypes.CDLL(path)
        lib.hcgen_db_u8.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
        lib.hcgen_queries_u8.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.hcgen_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_void_p]
        lib.hcgen_gauss.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_void_p]
        lib.hcgen_splitmix64_seq.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
        _LIB = lib
    return _LIB


def _threads(nthreads):
    return nthreads or max(1, os.cpu_count() or 1)


def make_db(n, d=128, seed=SEED_DB, n_clusters=N_CLUSTERS, sigma=SIGMA_DB, nthreads=None,
            out=None):
    """(n, d) uint8 database drawn from the clustered Gaussian mixture."""
    if out is None:
        out = np.empty((n, d), np.uint8)
    assert out.shape == (n, d) and out.dtype == np.uint8 and out.flags.c_contiguous
    rc = _lib().hcgen_db_u8(seed, n, d, n_clusters, sigma, out.ctypes.data, _threads(nthreads))
    if rc != 0:
        raise RuntimeError("hcgen_db_u8 failed (%d)" % rc)
    return out


def make_queries(db, nq, seed=SEED_QUERIES, sigma=SIGMA_QUERY, nthreads=None,
                 return_src=False):
    """(nq, d) uint8 queries: a uniformly drawn database row plus noise."""
    db = np.ascontiguousarray(db, dtype=np.uint8)
    n, d = db.shape
    out = np.empty((nq, d), np.uint8)
    src = np.empty(nq, np.uint64) if return_src else None
    rc = _lib().hcgen_queries_u8(seed, db.ctypes.data, n, d, nq, sigma, out.ctypes.data,
                                 src.ctypes.data if src is not None else None, _threads(nthreads))
    if rc != 0:
        raise RuntimeError("hcgen_queries_u8 failed (%d)" % rc)
    return (out, src) if return_src else out


def to_f32(x):
    """The float32 variant of a uint8 array: x / 255 rounded to float32."""
    return (np.asarray(x, dtype=np.float32) / np.float32(255.0)).astype(np.float32)


def draws(seed, stream, idx0, count):
    out = np.empty(count, np.uint64)
    _lib().hcgen_draws(seed, stream, idx0, count, out.ctypes.data)
    return out


def splitmix64(state, count):
    """The first count outputs of the SplitMix64 sequence started at state."""
    out = np.empty(count, np.uint64)
    _lib().hcgen_splitmix64_seq(state, count, out.ctypes.data)
    return out


def gaussians(seed, stream, e0, count):
    out = np.empty(count, np.float64)
    _lib().hcgen_gauss(seed, stream, e0, count, out.ctypes.data)
    return out


def uneven_workload(seed=11, n_indexes=64, n_min=10_000, n_max=2_000_000, b_min=1, b_max=4096):
    """Shapes of the batched-uneven workload: per index (n, d, dtype, nq, k),
    n and the batch size log-uniform, d in {64, 128, 256}, dtype mixed."""
    u = draws(seed, 7, 0, n_indexes * 5).reshape(n_indexes, 5)
    f = (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    out = []
    for i in range(n_indexes):
        n = int(round(np.exp(np.log(n_min) + f[i, 0] * (np.log(n_max) - np.log(n_min)))))
        d = (64, 128, 256)[int(f[i, 1] * 3)]
        dtype = "u8" if f[i, 2] < 0.5 else "f32"
        nq = int(round(np.exp(np.log(b_min) + f[i, 3] * (np.log(b_max) - np.log(b_min)))))
        k = (1, 10, 100)[int(f[i, 4] * 3)]
        out.append(dict(n=n, d=d, dtype=dtype, nq=max(1, nq), k=k, seed=1000 + i))
    return out
