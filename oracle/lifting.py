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


def inverse_mod_p(A, p: int):
    """A^-1 mod p (int64 [n][n] in [0, p)) by Gauss-Jordan elimination over GF(p),
    p < 2^31 so that every product fits int64.  ValueError if p divides det A."""
    import numpy as np
    n = len(A)
    M = np.concatenate([np.array(A, dtype=np.int64) % p, np.eye(n, dtype=np.int64)], axis=1)
    for k in range(n):
        piv = next((i for i in range(k, n) if M[i, k]), None)
        if piv is None:
            raise ValueError("singular modulo p")
        if piv != k:
            M[[k, piv]] = M[[piv, k]]
        M[k] = M[k] * pow(int(M[k, k]), p - 2, p) % p
        f = M[:, k].copy()
        f[k] = 0
        M = (M - np.outer(f, M[k]) % p) % p
    return M[:, n:].copy()


def lift_recurrence(A, B, p: int, k: int, C):
    """The same digits and residual as ``lift`` by the recurrence
    X_i = C R_i mod p, R_(i+1) = (R_i - A X_i) / p (C = A^-1 mod p), exact in
    int64 while n p^2 and n max|A| p stay below 2^62 (checked)."""
    import numpy as np
    A = np.asarray(A, dtype=np.int64)
    R = np.asarray(B, dtype=np.int64).copy()
    C = np.asarray(C, dtype=np.int64)
    n = A.shape[0]
    amax = int(np.abs(A).max()) if A.size else 0
    if n * p * p >= (1 << 62) or n * max(amax, 1) * p >= (1 << 61) or int(np.abs(R).max(initial=0)) >= (1 << 61):
        raise ValueError("outside the int64 range of the recurrence")
    digits = []
    for _ in range(k):
        X = (C @ (R % p)) % p
        digits.append(X)
        T = R - A @ X
        assert not (T % p).any()
        R = T // p
    return digits, R
