"""Index files (include/hc.h, hc_save) written and patched from Python by the
documented layout, so tests can hand hc_load files that are damaged or
crafted in one field at a time."""
import struct

import numpy as np

MAGIC = b"HCURVIDX"
MASK = (1 << 64) - 1


def file_hash(words):
    """The checksum of hc_save: h = (h xor w) * 0x9e3779b97f4a7c15, h ^= h >> 29."""
    x = 0x6a09e667f3bcc908
    for w in words:
        x = ((x ^ int(w)) * 0x9e3779b97f4a7c15) & MASK
        x ^= x >> 29
    return x


def header(n, d, curves, m, bits=8, dtype=0, partitions=1, lists=None, row_bytes=None,
           flags=0, total=None, version=1, bom=0x01020304, magic=MAGIC, reserved=0):
    lists = curves * partitions if lists is None else lists
    row_bytes = (d if dtype == 0 else 4 * d) if row_bytes is None else row_bytes
    total = n * curves if total is None else total
    h = magic + struct.pack("<IIQIIIIIIIIIIQ", version, bom, n, d, curves, m, bits, dtype,
                            partitions, lists, row_bytes, flags, reserved, total)
    return h + b"\0" * (80 - len(h))


def pad8(b):
    return b + b"\0" * (-len(b) % 8)


def assemble(head, list_off, hi, ids, lo=None, dim_map=None):
    """The file's bytes, checksum included."""
    body = head + np.asarray(list_off, "<u8").tobytes()
    if dim_map is not None:
        body += pad8(np.asarray(dim_map, "<u4").tobytes())
    body += np.asarray(hi, "<u8").tobytes()
    if lo is not None:
        body += np.asarray(lo, "<u8").tobytes()
    body += pad8(np.asarray(ids, "<u4").tobytes())
    return body + struct.pack("<Q", file_hash(np.frombuffer(body, "<u8")))


def reseal(path):
    """Rewrites the checksum of a file whose other words were edited."""
    data = bytearray(open(path, "rb").read())
    words = np.frombuffer(bytes(data[:-8]), "<u8")
    data[-8:] = struct.pack("<Q", file_hash(words))
    open(path, "wb").write(bytes(data))


def sections(path, n, curves, partitions=1, lo=False, dim_map_words=0):
    """Byte offsets of (keys_hi, keys_lo or None, ids, checksum) in a file."""
    lists = curves * partitions
    total = n * curves
    o = 80 + 8 * (lists + 1) + 8 * dim_map_words
    hi = o
    o += 8 * total
    lo_off = None
    if lo:
        lo_off = o
        o += 8 * total
    ids = o
    o += 4 * total + (4 * total) % 8
    return hi, lo_off, ids, o
