"""Pins for the lifting oracle: the digits and residual satisfy the defining
identity with Python integers, match an independent route (the recurrence
X_i = C R_i mod p, R_(i+1) = (R_i - A X_i) / p with C = A^-1 mod p from
sympy), and a diagonal system has closed-form digits.  CPU only."""
import random

import sympy

from oracle import lifting


def _rand(rng, n, m, bits):
    while True:
        A = [[rng.randint(-(1 << bits), 1 << bits) for _ in range(n)] for _ in range(n)]
        if sympy.Matrix(A).det() % 16777213:
            B = [[rng.randint(-(1 << 40), 1 << 40) for _ in range(m)] for _ in range(n)]
            return A, B


def test_identity_and_digit_range():
    rng = random.Random(1)
    p = 16777213  # a prime below 2^24
    for n, m, k in [(3, 2, 4), (7, 3, 6), (12, 1, 3)]:
        A, B = _rand(rng, n, m, 20)
        X, R = lifting.lift(A, B, p, k)
        S = [[sum(X[i][r][c] * p ** i for i in range(k)) for c in range(m)] for r in range(n)]
        for r in range(n):
            for c in range(m):
                assert sum(A[r][l] * S[l][c] for l in range(n)) + p ** k * R[r][c] == B[r][c]
        assert all(0 <= v < p for D in X for row in D for v in row)


def test_matches_the_recurrence():
    rng = random.Random(2)
    p = 1000003
    n, m, k = 6, 2, 5
    A, B = _rand(rng, n, m, 10)
    C = sympy.Matrix(A).inv_mod(p)
    R = [row[:] for row in B]
    want = []
    for _ in range(k):
        Xi = [[int(sum(C[r, l] * R[l][c] for l in range(n))) % p for c in range(m)] for r in range(n)]
        want.append(Xi)
        R = [[(R[r][c] - sum(A[r][l] * Xi[l][c] for l in range(n))) // p for c in range(m)] for r in range(n)]
    X, Rk = lifting.lift(A, B, p, k)
    assert X == want and Rk == R


def test_diagonal_closed_form():
    # A = 3 I, B = 1: X = 1/3, whose p-adic digits are those of (p^k - 1) / 3 ... for p = 7:
    # 1/3 = 5 + 4*7 + 4*7^2 + ... (3 * 5 = 15 = 1 + 2*7, then 3 * 4 + 2 = 14 = 0 + 2*7, ...)
    X, R = lifting.lift([[3]], [[1]], 7, 4)
    assert [D[0][0] for D in X] == [5, 4, 4, 4]
    assert 3 * (5 + 4 * 7 + 4 * 49 + 4 * 343) + 7 ** 4 * R[0][0] == 1


def test_inverse_mod_p_and_recurrence_match_definition():
    import numpy as np
    rng = random.Random(3)
    p = 16777213
    for n, m, k in [(4, 2, 3), (9, 3, 5)]:
        A, B = _rand(rng, n, m, 20)
        C = lifting.inverse_mod_p(A, p)
        assert ((C @ (np.array(A, dtype=np.int64) % p)) % p == np.eye(n, dtype=np.int64)).all()
        X, R = lifting.lift(A, B, p, k)
        X2, R2 = lifting.lift_recurrence(A, B, p, k, C)
        assert [D.tolist() for D in X2] == X and R2.tolist() == R
