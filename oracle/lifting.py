"""Oracle for p-adic (Dixon) lifting (test infrastructure only, plain Python integers).

The paper's Phase 2 projections and Phase 1 solve linear systems over Q by
p-adic lifting (Section 2: "via an integrality certification procedure";
the lifting whose initialization computes A^-1 mod p is discussed in the
adaptive batch sizing of Section 3).  For a nonsingular integer A (n x n)
with p not dividing det A and an integer B (n x m), the solution
X = A^-1 B has a unique p-adic expansion X = sum_i X_i p^i with digit
matrices X_i in [0, p); after k digits the residual R_k satisfies
    A (sum_(i<k) X_i p^i) + p^k R_k = B.
``lift`` returns (X_0, ..., X_(k-1)) and R_k from that definition: the digits
of A^-1 B mod p^k (A^-1 mod p^k by sympy) and R_k by exact division.
Pinned by ``tests/test_oracle_lifting.py``.
"""
from __future__ import annotations

import sympy


def lift(A, B, p: int, k: int):
    """Digits [k][n][m] (ints in [0, p)) and the residual R_k [n][m] (ints)."""
    n, m = len(A), len(B[0])
    pk = p ** k
    Ainv = sympy.Matrix(A).inv_mod(pk)
    X = (Ainv * sympy.Matrix(B)).applyfunc(lambda v: int(v) % pk)
    digits = []
    rest = [[int(X[i, j]) for j in range(m)] for i in range(n)]
    for _ in range(k):
        digits.append([[v % p for v in row] for row in rest])
        rest = [[v // p for v in row] for row in rest]
    Xk = [[int(X[i, j]) for j in range(m)] for i in range(n)]
    R = []
    for i in range(n):
        row = []
        for j in range(m):
            t = B[i][j] - sum(A[i][l] * Xk[l][j] for l in range(n))
            assert t % pk == 0
            row.append(t // pk)
        R.append(row)
    return digits, R
