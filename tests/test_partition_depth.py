"""The host-side partition depth (Sec. 4.2) of the product package against
the oracle's independent long-double version, plus the exact-rational cases
where float arithmetic would round the wrong way."""
from fractions import Fraction

import pytest

from oracle import oracle as O
from paper_1209_0410_gb300 import partition as P


@pytest.mark.parametrize("Phi", [1, 7, 64, 128, 256])
@pytest.mark.parametrize("ell", [1, 2, 3, 4, 8, 16, 32])
def test_slack_depth_and_bound_match_oracle(Phi, ell):
    for s in ["0", "0.1", "0.25", "0.5", "1"]:
        phi = P.slack_depth(Phi, ell, s)
        assert phi == O.slack_depth(Phi, ell, float(s))
        for mult in (None, ell):
            ours = P.equiv_bound(Phi, ell, phi, mult)
            ref = O.equiv_bound(Phi, ell, phi, mult)
            assert ours == pytest.approx(ref, rel=1e-9, abs=1e-15)


def test_slack_depth_is_exact():
    # (1 + 0.1) * 50 = 55 exactly; in binary floating point it lands above 55
    assert (1 + 0.1) * 50 > 55
    assert P.slack_depth(500, 10, "0.1") == 55
    assert P.slack_depth(128, 8, Fraction(1, 4)) == 20
    assert P.slack_depth(0, 4, "0.5") == 0


def test_pessimist_slack_is_smallest_on_grid():
    for ell in (2, 4, 8, 16, 32):
        s = P.pessimist_slack(128, ell)
        assert P.equiv_bound(128, ell, P.slack_depth(128, ell, s)) < 0.02
        if s > 0:
            below = s - Fraction(1, 20)
            assert P.equiv_bound(128, ell, P.slack_depth(128, ell, below)) >= 0.02
    assert P.pessimist_slack(128, 1) == 0


def test_argument_errors():
    with pytest.raises(ValueError):
        P.slack_depth(10, 0, 0)
