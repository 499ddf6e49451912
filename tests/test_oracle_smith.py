"""Pins for the Smith-form oracle: each check ties it to something other than
itself (brute force over minors, sympy, the known construction U diag(s) V,
the invariants of the Smith form).  CPU only."""
import itertools
import random
from math import gcd, prod

import pytest
import sympy
from sympy.matrices.normalforms import smith_normal_form

from oracle import smith
from paper_2605_19254_gb300 import inputs


def _rand_nonsingular(rng, n, lo=-9, hi=9):
    while True:
        A = [[rng.randint(lo, hi) for _ in range(n)] for _ in range(n)]
        if sympy.Matrix(A).det() != 0:
            return A


def test_det_bareiss_matches_sympy():
    rng = random.Random(1)
    for n in [1, 2, 3, 5, 8, 12]:
        for _ in range(5):
            A = [[rng.randint(-50, 50) for _ in range(n)] for _ in range(n)]
            assert smith.det_bareiss(A) == sympy.Matrix(A).det()
    big = [[rng.randint(-(1 << 70), 1 << 70) for _ in range(6)] for _ in range(6)]
    assert smith.det_bareiss(big) == sympy.Matrix(big).det()
    assert smith.det_bareiss([[0, 1], [1, 0]]) == -1
    assert smith.det_bareiss([[1, 2], [2, 4]]) == 0


def test_det_mod_matches_exact():
    rng = random.Random(2)
    qs = [(1 << 61) - 1, 4611686018427387847, 2305843009213693921]
    qs = [q for q in qs if sympy.isprime(q)]
    assert qs
    for n in [3, 7, 16]:
        A = [[rng.randint(-1000, 1000) for _ in range(n)] for _ in range(n)]
        d = smith.det_bareiss(A)
        for q in qs:
            assert smith.det_mod(A, q) == d % q


def _brute_force_snf(A):
    # s_k = d_k / d_(k-1), d_k = gcd of all k x k minors (determinants by sympy)
    n = len(A)
    M = sympy.Matrix(A)
    dk = [1]
    for k in range(1, n + 1):
        g = 0
        for rows in itertools.combinations(range(n), k):
            for cols in itertools.combinations(range(n), k):
                g = gcd(g, int(M.extract(list(rows), list(cols)).det()))
        dk.append(g)
    return [dk[k] // dk[k - 1] for k in range(1, n + 1)]


def test_smith_form_matches_minors_brute_force():
    rng = random.Random(3)
    for n in [1, 2, 3, 4]:
        for _ in range(6):
            A = _rand_nonsingular(rng, n)
            assert smith.smith_form(A) == _brute_force_snf(A)
    # structured: large common factors
    A = [[6, 12, 18], [4, 10, 2], [8, 0, 14]]
    assert smith.smith_form(A) == _brute_force_snf(A)


def test_smith_form_matches_sympy():
    rng = random.Random(4)
    for n in [5, 8, 11]:
        for _ in range(3):
            A = _rand_nonsingular(rng, n, -20, 20)
            D = smith_normal_form(sympy.Matrix(A), domain=sympy.ZZ)
            want = sorted(abs(int(D[i, i])) for i in range(n))
            got = smith.smith_form(A)
            assert sorted(got) == want
            assert got == want  # non-decreasing as returned


def test_known_construction_config1():
    # U diag(s) V with U, V products of 4n elementary operations, multipliers in [-3, 3]
    s = [1] * 58 + [2, 6, 12, 60, 120, 840]
    A = inputs.smith_known_matrix(0, s)
    assert prod(s) == 870912000
    assert abs(smith.det_bareiss(A)) == 870912000
    assert smith.smith_form(A) == s


def test_invariants_on_random_and_known():
    rng = random.Random(5)
    for n in [6, 10, 20]:
        A = _rand_nonsingular(rng, n, -30, 30)
        S = smith.smith_form(A)
        assert all(x > 0 for x in S)
        assert all(S[i + 1] % S[i] == 0 for i in range(n - 1))
        assert prod(S) == abs(smith.det_bareiss(A))
    s = [1, 1, 3, 3, 6, 30, 30, 210]
    A = inputs.smith_known_matrix(7, s)
    assert smith.smith_form(A) == s


def test_singular_and_unimodular():
    with pytest.raises(smith.SingularMatrix):
        smith.smith_form([[1, 2], [2, 4]])
    U = inputs.smith_known_matrix(9, [1] * 12)
    assert smith.smith_form(U) == [1] * 12


def test_smith_form_of_the_papers_test_matrices_matches_sympy():
    # A_ij = i^j mod n (Section 4): many non-trivial invariant factors, and
    # pivots equal to the entries they clear (an elimination that swapped the
    # pivot column back and forth on those never ended)
    for n in [3, 5, 7, 11, 13, 17]:
        A = inputs.vandermonde_mod(n).tolist()
        assert A == [[pow(i, j, n) for j in range(n)] for i in range(n)]
        S = smith_normal_form(sympy.Matrix(A), domain=sympy.ZZ)
        assert smith.smith_form(A) == sorted(abs(int(S[i, i])) for i in range(n))
    s = smith.smith_form(inputs.vandermonde_mod(53).tolist())
    assert all(b % a == 0 for a, b in zip(s, s[1:]))
    assert prod(s) == abs(smith.det_bareiss(inputs.vandermonde_mod(53).tolist()))


def test_c_det_mod_matches_exact_determinant(orc):
    # oracle.det_mod (plain C over GF(q)) against the exact Bareiss determinant
    # (itself pinned to sympy) reduced mod q, and against the Python elimination
    import numpy as np
    rng = random.Random(7)
    qs = [int(sympy.prevprime(1 << 62)), int(sympy.prevprime(1 << 31)), 1000003, 3]
    for n in [1, 2, 3, 6, 11, 24]:
        for trial in range(3):
            A = [[rng.randint(-(1 << 40), 1 << 40) for _ in range(n)] for _ in range(n)]
            d = smith.det_bareiss(A)
            for q in qs:
                got = orc.det_mod(np.array(A, dtype=np.int64), q)
                assert got == d % q, (n, trial, q)
                assert got == smith.det_mod(A, q)
    # extremes of int64, pivots that need row swaps, singular matrices
    A = np.array([[0, -(1 << 63)], [(1 << 63) - 1, 5]], dtype=np.int64)
    assert orc.det_mod(A, qs[0]) == (0 * 5 - (-(1 << 63)) * ((1 << 63) - 1)) % qs[0]
    P = np.zeros((9, 9), dtype=np.int64)
    for i in range(9):
        P[i, (4 * i + 1) % 9] = 1
    assert orc.det_mod(P, qs[0]) == smith.det_bareiss(P.tolist()) % qs[0]
    S = np.array([[1, 2, 3], [2, 4, 6], [7, 8, 10]], dtype=np.int64)
    assert orc.det_mod(S, qs[0]) == 0
    T = np.array([[3, 1], [0, 5]], dtype=np.int64)  # det 15: zero modulo 3 only
    assert orc.det_mod(T, 3) == 0 and orc.det_mod(T, qs[1]) == 15
    assert orc.det_mod(np.zeros((0, 0), dtype=np.int64), qs[0]) == 1


def test_numpy_planted_construction_matches_python():
    # the numpy construction performs the same operations as the plain one
    import numpy as np
    for n, seed in [(5, 1), (40, 2), (64, 0)]:
        s = [1] * (n - 3) + [2, 6, 30]
        assert np.array_equal(inputs.smith_known_matrix_np(seed, s), np.array(inputs.smith_known_matrix(seed, s)))
    chain = inputs.divisibility_chain(3, "c", 6)
    assert all(b % a == 0 for a, b in zip(chain, chain[1:]))
    batch = inputs.batched_smith_workload(0, 6, 32, 64)
    for n, bits, A, s in batch:
        assert A.shape == (n, n) and int(np.abs(A).max()).bit_length() <= bits
    n, bits, A, s = batch[1]
    assert smith.smith_form(A.tolist()) == s  # a planted item's Smith form is its s
