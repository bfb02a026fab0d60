"""Pins of the partitioned (Hypercurves) search and of the equivalence bound
(Sec. 4.1 and Sec. 4.2).

- The reduction is conservative: with the sequential depth used in every
  partition, the sequential candidates are a subset of the partitioned ones
  and every result distance is at most the sequential one.
- Depth covering every partition gives the exact kNN.
- Local top-k then reduce = top-k of the union of all partitions' windows.
- The binomial tail equals scipy's survival function; the printed bound
  holds against a Monte-Carlo of the half-list model at 2*Phi = 256 and
  falls towards zero as the slack grows.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1209_0410_gb300 import datagen


def case(n=4000, nq=40, seed=31):
    db = datagen.make_db(n, 128, seed=seed)
    q = datagen.make_queries(db, nq, seed=seed + 1)
    return db, q


def random_parts(n, ell, seed):
    return np.random.default_rng(seed).integers(0, ell, size=n).astype(np.uint32)


def windows(index, pos, L, p):
    sl = index.list_slice(L)
    n = sl.stop - sl.start
    return set(index.ids[sl][max(0, pos - p):min(n, pos + p)].tolist())


@pytest.mark.parametrize("ell", [2, 3, 4, 8])
@pytest.mark.parametrize("scheme", ["contiguous", "random"])
def test_partitioned_superset_of_sequential(ell, scheme):
    db, q = case()
    p, k = 24, 10
    part_of = None if scheme == "contiguous" else random_parts(len(db), ell, ell)
    seq = O.build(db, curves=8, m=16)
    par = O.build(db, curves=8, m=16, ell=ell, part_of=part_of)
    sids, sdist, spos = O.search(seq, db, q, k, p, return_pos=True)
    pids, pdist, ppos = O.search(par, db, q, k, p, return_pos=True)
    for i in range(len(q)):
        cs, cp = set(), set()
        for c in range(8):
            cs |= windows(seq, int(spos[i, c]), c, p)
        for L in range(par.lists):
            cp |= windows(par, int(ppos[i, L]), L, p)
        assert cs <= cp
    assert np.all(pdist <= sdist)


@pytest.mark.parametrize("ell", [2, 5])
@pytest.mark.parametrize("scheme", ["contiguous", "random"])
def test_partitioned_full_depth_is_exact(ell, scheme):
    db, q = case(2500, 30)
    part_of = None if scheme == "contiguous" else random_parts(len(db), ell, 99)
    par = O.build(db, curves=8, m=16, ell=ell, part_of=part_of)
    ids, dist = O.search(par, db, q, 10, len(db))
    bids, bdist = O.bruteforce(db, q, 10)
    assert np.array_equal(ids, bids) and np.array_equal(dist, bdist)


def test_reduce_equals_topk_of_union():
    """Local kNN per partition then the Aggregator's reduction = the k nearest
    of the union of every partition's candidates (the order on (dist, id) is
    total, so every global winner is a local winner)."""
    db, q = case(4000, 30)
    ell, p, k = 4, 10, 10
    par = O.build(db, curves=8, m=16, ell=ell, part_of=random_parts(len(db), ell, 5))
    ids, dist, pos = O.search(par, db, q, k, p, return_pos=True)
    for i in range(len(q)):
        cand = set()
        for L in range(par.lists):
            cand |= windows(par, int(pos[i, L]), L, p)
        cand = np.array(sorted(cand))
        dd = ((db[cand].astype(np.int64) - q[i].astype(np.int64)) ** 2).sum(axis=1)
        order = np.lexsort((cand, dd))[:k]
        assert ids[i].tolist() == cand[order].tolist()


def test_contiguous_partition_boundaries():
    db, _ = case(1003, 1)
    ell = 4
    par = O.build(db, curves=2, m=16, ell=ell)
    for j in range(ell):
        lo, hi = (j * len(db)) // ell, ((j + 1) * len(db)) // ell
        for c in range(2):
            ids = par.ids[par.list_slice(j * 2 + c)]
            assert np.array_equal(np.sort(ids), np.arange(lo, hi))


# ----------------------------------------------------------- Sec. 4.2 bound
@pytest.mark.parametrize("Phi,ell,phi", [(128, 2, 64), (128, 4, 32), (128, 8, 20), (128, 16, 8),
                                         (10, 3, 0), (10, 3, 10), (1, 1, 0), (300, 7, 60)])
def test_binom_tail_matches_scipy(Phi, ell, phi):
    from scipy import stats
    ref = stats.binom.sf(phi, Phi, 1.0 / ell)
    got = O.binom_tail(Phi, ell, phi)
    assert got == pytest.approx(ref, rel=1e-9, abs=1e-300)


def test_slack_depth():
    assert O.slack_depth(128, 4, 0.0) == 32
    assert O.slack_depth(128, 4, 0.5) == 48
    assert O.slack_depth(128, 3, 0.0) == 43
    assert O.slack_depth(128, 8, 0.1) == 18      # 1.1 * 16 = 17.6 -> 18
    assert O.slack_depth(100, 10, 0.1) == 11     # exact product, no round-up


def monte_carlo_miss(Phi, ell, phi, trials, rng):
    """Half-list model: each of the Phi entries below and the Phi entries at or
    above the query goes to one of ell lists uniformly; a miss happens when any
    list holds more than phi entries of either half."""
    lo = rng.integers(0, ell, size=(trials, Phi))
    hi = rng.integers(0, ell, size=(trials, Phi))
    cl = np.stack([(lo == j).sum(axis=1) for j in range(ell)], axis=1)
    ch = np.stack([(hi == j).sum(axis=1) for j in range(ell)], axis=1)
    miss = (cl.max(axis=1) > phi) | (ch.max(axis=1) > phi)
    return miss.mean()


@pytest.mark.parametrize("ell", [2, 4, 8, 16])
def test_bound_dominates_monte_carlo(ell):
    rng = np.random.default_rng(ell)
    Phi, trials = 128, 20_000
    prev = 1.0
    for slack in np.round(np.arange(0.0, 1.01, 0.1), 2):
        phi = O.slack_depth(Phi, ell, slack)
        emp = monte_carlo_miss(Phi, ell, phi, trials, rng)
        printed = O.equiv_bound(Phi, ell, phi)            # multiplier Phi, as printed
        by_lists = O.equiv_bound(Phi, ell, phi, mult=ell)  # multiplier ell
        # 3-sigma Monte-Carlo slack
        tol = 3 * np.sqrt(max(emp, 1.0 / trials) * (1 - emp) / trials)
        assert emp <= printed + tol
        assert emp <= by_lists + tol
        assert by_lists <= printed + 1e-15
        assert printed <= prev + 1e-15
        prev = printed
    # a "Pessimist" slack (bound below 2%) exists well below phi = Phi
    pess = [s for s in np.arange(0.0, 4.01, 0.05)
            if O.equiv_bound(Phi, ell, O.slack_depth(Phi, ell, s)) < 0.02]
    assert pess and O.slack_depth(Phi, ell, pess[0]) < Phi


def test_bound_degenerate_cases():
    assert O.equiv_bound(128, 1, 128) == 0.0      # one list: nothing spills
    assert O.equiv_bound(128, 4, 128) == 0.0      # phi = Phi: nothing spills
    assert O.equiv_bound(128, 16, 0) == 1.0       # phi = 0 with entries present
