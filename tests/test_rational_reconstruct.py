"""Host logic of the Smith-form driver, no GPU: rational reconstruction
(extended Euclid with Lehmer's single-precision quotient runs, over the
library's own big integers) against fractions
planted with Python's exact integers.  A fraction a / b with |a| < 2^nb,
0 < b < 2^db and gcd(a, b) = 1 is the unique one with a = b u (mod P) when
P > 2^(nb + db + 1), so the planted fraction is the only correct answer."""
import math
import random

import pytest

from paper_2605_19254_gb300 import smf


def _plant(rng, nb, db, P):
    while True:
        b = rng.randrange(1, 1 << db)
        a = rng.randrange(-(1 << nb) + 1, 1 << nb)
        if math.gcd(a, b) == 1 and math.gcd(b, P) == 1:
            return a, b


@pytest.mark.parametrize("p,nb,db", [(16777213, 20, 20), (16777213, 900, 700), (65521, 4000, 3000),
                                     (3, 64, 1), (16777213, 1, 31), (16777213, 20000, 19000),
                                     (16777213, 30000, 96)])
def test_planted_fractions(p, nb, db):
    rng = random.Random(p + nb + db)
    k = (nb + db + 1) // (p.bit_length() - 1) + 2
    P = p ** k
    assert P > 1 << (nb + db + 1)
    for _ in range(6):
        a, b = _plant(rng, nb, db, P)
        u = a * pow(b, -1, P) % P
        assert smf.rational_reconstruct(u, P, nb, db) == (a, b)


def test_integers_zero_and_signs():
    p = 16777213
    P = p ** 4
    assert smf.rational_reconstruct(0, P, 40, 40) == (0, 1)
    assert smf.rational_reconstruct(12345, P, 40, 40) == (12345, 1)
    assert smf.rational_reconstruct(P - 12345, P, 40, 40) == (-12345, 1)
    assert smf.rational_reconstruct(pow(7, -1, P), P, 40, 40) == (1, 7)
    assert smf.rational_reconstruct((-5) * pow(9, -1, P) % P, P, 40, 40) == (-5, 9)
    # u given above P is reduced first
    assert smf.rational_reconstruct(P + 12345, P, 40, 40) == (12345, 1)


def test_no_fraction_within_the_bounds():
    # with a tight denominator bound a generic residue has no small fraction
    P = 16777213 ** 6
    u = pow(3, -1, P) * 1000003 % P
    with pytest.raises(smf.SmfError):
        smf.rational_reconstruct(u, P, 10, 10)


def test_row_with_a_common_factor_has_no_fraction():
    # u = 6 mod 2^8 with |a| < 2: Euclid's stopping row is (0, -128), whose
    # remainder and cofactor share 128, so no fraction a / b with a = 6 b (mod 256)
    # is within the bounds (0 / 1 would not satisfy it)
    with pytest.raises(smf.SmfError):
        smf.rational_reconstruct(6, 256, 1, 8)
    # while 2 / 43 (43 * 6 = 258 = 2 mod 256) is found with a larger numerator bound
    a, b = smf.rational_reconstruct(6, 256, 2, 8)
    assert (a - b * 6) % 256 == 0 and abs(a) < 4 and 0 < b < 256
