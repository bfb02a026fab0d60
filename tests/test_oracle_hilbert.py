"""Pins of the oracle's Hilbert extended-key C^-1 (Sec. 2.2.1).

The paper fixes: the map is bijective at finite order and keeps the bit count
(d coordinates of m bits -> one key of d*m bits), and it is a Hilbert curve.
These tests check exactly those properties by brute force on tiny grids, the
2-D case against the textbook curve built from its recursive definition, and
round trips / unit steps on full-size 16 x 8-bit keys.  A Z-order curve is
run through the same adjacency check as a negative control.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O

TINY_GRIDS = [(2, b) for b in range(1, 7)] + [(3, b) for b in range(1, 5)] + \
             [(4, b) for b in range(1, 4)] + [(8, 2), (16, 1)]


def all_points(n, b):
    side = 1 << b
    g = np.indices((side,) * n).reshape(n, -1).T
    return np.ascontiguousarray(g, dtype=np.uint32)


def keys_as_int(hi, lo):
    return np.array([O.key_int(h, l) for h, l in zip(hi, lo)], dtype=object)


def curve_order(n, b):
    """Points of the grid listed in key order (uses bijectivity)."""
    pts = all_points(n, b)
    hi, lo = O.hilbert_keys(n, b, pts)
    k = keys_as_int(hi, lo)
    order = sorted(range(len(k)), key=lambda i: k[i])
    return pts[order], [k[i] for i in order]


@pytest.mark.parametrize("n,b", TINY_GRIDS)
def test_bijective_and_bit_preserving(n, b):
    pts = all_points(n, b)
    hi, lo = O.hilbert_keys(n, b, pts)
    k = sorted(keys_as_int(hi, lo))
    assert k == list(range(1 << (n * b)))


@pytest.mark.parametrize("n,b", TINY_GRIDS)
def test_unit_step_adjacency(n, b):
    seq, _ = curve_order(n, b)
    diff = np.abs(seq[1:].astype(np.int64) - seq[:-1].astype(np.int64))
    assert np.all(diff.sum(axis=1) == 1)
    assert np.all((diff > 0).sum(axis=1) == 1)


@pytest.mark.parametrize("n,b", TINY_GRIDS)
def test_dyadic_nesting(n, b):
    """Keys sharing their top n*j bits cover one aligned sub-cube of side
    2^(b-j): the curve visits sub-cubes whole (recursive refinement)."""
    seq, keys = curve_order(n, b)
    for j in range(1, b):
        shift = n * (b - j)
        prefix = np.array([kk >> shift for kk in keys], dtype=object)
        cell = seq >> (b - j)
        for pref in set(prefix.tolist()):
            sel = prefix == pref
            cells = {tuple(c) for c in cell[sel]}
            assert len(cells) == 1
            assert sel.sum() == 1 << shift


@pytest.mark.parametrize("n,b", TINY_GRIDS)
def test_origin_first(n, b):
    hi, lo = O.hilbert_keys(n, b, np.zeros((1, n), np.uint32))
    assert int(hi[0]) == 0 and int(lo[0]) == 0


def textbook_hilbert_2d(order):
    """The 2-D Hilbert curve from its recursive definition: the order-r curve
    is four copies of the order-(r-1) curve in the quadrants visited in a U;
    the first copy is reflected in the main diagonal and the last one in the
    anti-diagonal so that consecutive copies join with unit steps."""
    if order == 0:
        return [(0, 0)]
    prev = textbook_hilbert_2d(order - 1)
    h = 1 << (order - 1)
    out = [(y, x) for (x, y) in prev]                      # lower-left, transposed
    out += [(x, y + h) for (x, y) in prev]                 # upper-left
    out += [(x + h, y + h) for (x, y) in prev]             # upper-right
    out += [(2 * h - 1 - y, h - 1 - x) for (x, y) in prev]  # lower-right, anti-transposed
    return out


def dihedral(pt, side, g):
    x, y = pt
    m = side - 1
    return [(x, y), (y, x), (m - x, y), (x, m - y), (m - x, m - y), (m - y, x), (y, m - x),
            (m - y, m - x)][g]


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_2d_equals_textbook_up_to_symmetry(order):
    ref = textbook_hilbert_2d(order)
    side = 1 << order
    # the textbook construction is itself a unit-step curve over the grid
    assert len(set(ref)) == side * side
    assert all(abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1 for a, b in zip(ref, ref[1:]))
    seq, _ = curve_order(2, order)
    got = [tuple(int(v) for v in p) for p in seq]
    assert any([dihedral(p, side, g) for p in ref] == got for g in range(8))


def zorder_key(pt, n, b):
    k = 0
    for q in range(b - 1, -1, -1):
        for i in range(n):
            k = (k << 1) | ((int(pt[i]) >> q) & 1)
    return k


def test_adjacency_check_rejects_zorder():
    """Negative control: the unit-step check fails for the Z-order curve, so it
    distinguishes a Hilbert curve from a plain bit interleave."""
    n, b = 2, 3
    pts = all_points(n, b)
    order = sorted(range(len(pts)), key=lambda i: zorder_key(pts[i], n, b))
    seq = pts[order].astype(np.int64)
    steps = np.abs(seq[1:] - seq[:-1]).sum(axis=1)
    assert not np.all(steps == 1)


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(12345)


def test_full_size_round_trip_points(rng):
    pts = rng.integers(0, 256, size=(300_000, 16), dtype=np.uint32)
    hi, lo = O.hilbert_keys(16, 8, pts)
    back = O.hilbert_axes(16, 8, hi, lo)
    assert np.array_equal(back, pts)


def test_full_size_round_trip_keys(rng):
    hi = rng.integers(0, 2**63, size=300_000, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=300_000, dtype=np.uint64)
    lo = rng.integers(0, 2**63, size=300_000, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=300_000, dtype=np.uint64)
    pts = O.hilbert_axes(16, 8, hi, lo)
    assert pts.max() < 256
    hi2, lo2 = O.hilbert_keys(16, 8, pts)
    assert np.array_equal(hi, hi2) and np.array_equal(lo, lo2)


def test_full_size_unit_steps(rng):
    """K and K+1 decode to points one unit step apart, for random 128-bit K
    (including carries from lo into hi)."""
    cnt = 200_000
    hi = rng.integers(0, 2**63, size=cnt, dtype=np.uint64)
    lo = rng.integers(0, 2**63, size=cnt, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    lo[:1000] = np.uint64(2**64 - 1)   # force carries
    lo1 = lo + np.uint64(1)
    hi1 = hi + (lo1 == 0).astype(np.uint64)
    a = O.hilbert_axes(16, 8, hi, lo).astype(np.int64)
    b = O.hilbert_axes(16, 8, hi1, lo1).astype(np.int64)
    d = np.abs(a - b)
    assert np.all(d.sum(axis=1) == 1)


def test_quantize_reading():
    """Float32 key coordinates: rint(x*255) in float32, clamped; the x = u/255
    float32 values of the workload map back to u exactly."""
    u = np.arange(256, dtype=np.uint8)
    x = (u.astype(np.float32) / np.float32(255.0)).astype(np.float32)
    assert np.array_equal(O.quantize(x), u.astype(np.uint32))
    special = np.array([-1.0, -0.0, 0.0, np.nan, 2.0, np.inf, 0.5 / 255, 1.5 / 255,
                        254.5 / 255], np.float32)
    got = O.quantize(special)
    s = special * np.float32(255.0)
    exp = []
    for v in s:
        if not (v > 0):
            exp.append(0)
        elif v >= 255:
            exp.append(255)
        else:
            exp.append(int(np.rint(v)))
    assert got.tolist() == exp


def test_curve_keys_match_direct_projection(rng):
    """Algorithm 1's projection: query_keys(v, curve c) = C^-1(v[a[c, :]])."""
    q = rng.integers(0, 256, size=(50, 128), dtype=np.uint8)
    dim_map = rng.permutation(128).astype(np.uint32).reshape(8, 16)
    hi, lo = O.query_keys(q, 8, 16, dim_map)
    for c in range(8):
        h2, l2 = O.hilbert_keys(16, 8, q[:, dim_map[c]].astype(np.uint32))
        assert np.array_equal(hi[:, c], h2) and np.array_equal(lo[:, c], l2)


def test_small_m_key_width():
    """m dims of 8 bits give keys below 2^(8m)."""
    pts = np.array(list(itertools.product(range(0, 256, 51), repeat=3)), np.uint32)
    hi, lo = O.hilbert_keys(3, 8, pts)
    assert np.all(hi == 0) and np.all(lo < (1 << 24))
