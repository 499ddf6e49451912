"""Pins for the oracle's conversion between RNS bases (Section 3.1): the
output must be x mod q for the integer x the input residues represent.  The
expected values come from Python integers alone.  CPU only."""
import random

import numpy as np


def _bases(orc):
    P = [int(p) for p in orc.basis(1 << 24, 500)]           # 23 primes below 2^24
    Q = [int(p) for p in orc.primes_below(min(P), 23)]     # the next 23, disjoint
    return P, Q


def _prod(ps):
    m = 1
    for p in ps:
        m *= p
    return m


def test_base_convert_random_and_endpoints(orc):
    P, Q = _bases(orc)
    M = _prod(P)
    H = (M - 1) // 2
    rng = random.Random(5)
    xs = [0, 1, -1, 2, -2, H, -H, H - 1, -H + 1, P[0], -P[0], M // P[-1], -(M // P[-1])]
    xs += [rng.randint(-H, H) for _ in range(400)]
    xs += [rng.randint(-(1 << 64), 1 << 64) for _ in range(50)]   # small magnitudes
    r_in = np.array([[x % p for x in xs] for p in P], dtype=np.int32)
    got = orc.base_convert(r_in, P, Q)
    want = np.array([[x % q for x in xs] for q in Q], dtype=np.int32)
    assert got.shape == (len(Q), len(xs))
    assert np.array_equal(got, want)


def test_base_convert_exhaustive_tiny_basis(orc):
    # every representable x for a 3-prime basis, into a basis of larger primes
    P, Q = [5, 7, 11], [13, 17, 19, 23]
    M = _prod(P)
    xs = list(range(-(M - 1) // 2, (M - 1) // 2 + 1))
    r_in = np.array([[x % p for x in xs] for p in P], dtype=np.int32)
    got = orc.base_convert(r_in, P, Q)
    want = np.array([[x % q for x in xs] for q in Q], dtype=np.int32)
    assert np.array_equal(got, want)


def test_base_convert_keeps_matrix_shape_and_overlapping_primes(orc):
    # a [L, rows, cols] residue matrix; a target prime shared with the source
    # basis gives back that prime's residues unchanged
    P, Q = _bases(orc)
    M = _prod(P)
    rng = random.Random(9)
    xs = [[rng.randint(-(M - 1) // 2, (M - 1) // 2) for _ in range(7)] for _ in range(5)]
    r_in = np.array([[[x % p for x in row] for row in xs] for p in P], dtype=np.int32)
    Q2 = [P[3]] + Q[:4]
    got = orc.base_convert(r_in, P, Q2)
    assert got.shape == (5, 5, 7)
    assert np.array_equal(got[0], r_in[3])
    want = np.array([[[x % q for x in row] for row in xs] for q in Q2], dtype=np.int32)
    assert np.array_equal(got, want)
