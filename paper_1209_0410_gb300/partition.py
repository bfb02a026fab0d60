"""Per-partition probe depth of partitioned Hypercurves (Sec. 4.2).

A database split into ell disjoint partitions is searched with a local depth
phi in every partition.  The sequential window of Phi entries below and Phi
at or above the query key spreads over the partitions like a multinomial
draw; phi = ceil((1 + slack) * ceil(Phi / ell)) leaves room for the uneven
spread, and Eq. 6 bounds the probability that some partition's half-window
overflows phi (then the partitioned answer may differ from the sequential
one).  "Optimist" takes slack 0, "Pessimist" the smallest slack whose bound
falls below 2% (Sec. 7).

Host-side arithmetic only (exact rationals, no floating-point tail sums):
the depths it returns are what hc_query takes as p on a partitioned index.
"""
import math
from fractions import Fraction


def _frac(x):
    return x if isinstance(x, Fraction) else Fraction(str(x))


def slack_depth(Phi, ell, slack):
    """phi = ceil((1 + slack) * ceil(Phi / ell)), computed exactly."""
    if Phi < 0 or ell < 1:
        raise ValueError("Phi >= 0 and ell >= 1 required")
    base = -(-Phi // ell)
    return math.ceil((1 + _frac(slack)) * base)


def binom_tail(Phi, ell, phi):
    """P(Bin(Phi, 1/ell) > phi), as an exact fraction."""
    pr = Fraction(1, ell)
    qr = 1 - pr
    return sum((math.comb(Phi, j) * pr ** j * qr ** (Phi - j)
                for j in range(phi + 1, Phi + 1)), Fraction(0))


def equiv_bound(Phi, ell, phi, mult=None):
    """Eq. 6: 1 - max(0, 1 - mult * P(Bin(Phi, 1/ell) > phi))^2.

    mult is the union-bound multiplier; the paper prints Phi (the default).
    Returned as a float."""
    m = Fraction(Phi if mult is None else mult)
    inner = max(Fraction(0), 1 - m * binom_tail(Phi, ell, phi))
    return float(1 - inner * inner)


def pessimist_slack(Phi, ell, target=0.02, step="0.05", max_slack=8):
    """Smallest slack on the grid {0, step, 2 step, ...} whose bound (printed
    multiplier) is below target; ell = 1 needs none."""
    if ell == 1:
        return Fraction(0)
    st = _frac(step)
    s = Fraction(0)
    while s <= max_slack:
        if equiv_bound(Phi, ell, slack_depth(Phi, ell, s)) < target:
            return s
        s += st
    raise ValueError("no slack up to %s reaches the target" % max_slack)
