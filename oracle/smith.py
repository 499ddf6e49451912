"""Oracle for the Smith form (test infrastructure only, plain Python integers).

The problem the paper states: for a nonsingular integer matrix A (n x n) find
its Smith form diag(s_1, ..., s_n), s_i > 0 and s_i | s_(i+1), with
prod s_i = |det A| (Section 2).  The paper's massager algorithm is one way to
reach it; this module reaches the same unique result by elimination:

- ``det_bareiss``: the exact determinant by Bareiss' fraction-free elimination
  (every division is exact).
- ``smith_form``: with d = |det A|, d Z^n lies in the lattice of A's columns
  (d A^-1 = +-adj(A) is integral), so the Smith form of A equals that of A
  over Z/dZ, with s_i = gcd(e_i, d) for the diagonal e_i found there.  Over
  Z/dZ the diagonal is reached by 2 x 2 unimodular steps from extended gcds on
  rows and columns, then a divisibility fix-up (Section 2's invariant factors
  are unique, so any elimination order gives them).
- ``det_mod``: det A mod q by Gaussian elimination over GF(q).

Slow and meant for small n.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the bench's CPU baseline may use it.  Pinned by ``tests/test_oracle_smith.py``.
"""
from __future__ import annotations

from math import gcd


class SingularMatrix(ValueError):
    pass


def det_bareiss(A) -> int:
    """Exact det A for a square integer matrix (lists of ints)."""
    M = [list(map(int, row)) for row in A]
    n = len(M)
    if any(len(r) != n for r in M):
        raise ValueError("square matrix required")
    sign, prev = 1, 1
    for k in range(n - 1):
        if M[k][k] == 0:
            for i in range(k + 1, n):
                if M[i][k] != 0:
                    M[k], M[i] = M[i], M[k]
                    sign = -sign
                    break
            else:
                return 0
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev  # exact
            M[i][k] = 0
        prev = M[k][k]
    return sign * M[n - 1][n - 1] if n else 1


def _xgcd(a: int, b: int):
    """(g, x, y) with a x + b y = g = gcd(a, b) >= 0."""
    x0, y0, x1, y1 = 1, 0, 0, 1
    while b:
        q, a, b = a // b, b, a - (a // b) * b
        x0, x1 = x1, x0 - q * x1
        y0, y1 = y1, y0 - q * y1
    if a < 0:
        a, x0, y0 = -a, -x0, -y0
    return a, x0, y0


def smith_form(A):
    """[s_1, ..., s_n] of a nonsingular integer matrix (SingularMatrix otherwise)."""
    n = len(A)
    d = abs(det_bareiss(A))
    if d == 0:
        raise SingularMatrix("det A = 0")
    if d == 1:
        return [1] * n
    M = [[int(a) % d for a in row] for row in A]

    def rows(i, k, a, b, c, e):  # (row_k, row_i) <- (a row_k + b row_i, c row_k + e row_i), det = 1
        rk, ri = M[k], M[i]
        M[k] = [(a * x + b * y) % d for x, y in zip(rk, ri)]
        M[i] = [(c * x + e * y) % d for x, y in zip(rk, ri)]

    def cols(j, k, a, b, c, e):
        for row in M:
            x, y = row[k], row[j]
            row[k], row[j] = (a * x + b * y) % d, (c * x + e * y) % d

    diag = []
    for k in range(n):
        while True:
            # a pivot with the smallest gcd with d (0 counts as d) at (k, k)
            best = None
            for i in range(k, n):
                for j in range(k, n):
                    g = gcd(M[i][j], d)
                    if best is None or g < best[0]:
                        best = (g, i, j)
            _, bi, bj = best
            M[k], M[bi] = M[bi], M[k]
            for row in M:
                row[k], row[bj] = row[bj], row[k]
            # A pivot that divides an entry clears it by subtracting a multiple
            # (cofactors 1, 0), which leaves the pivot's row and column alone;
            # otherwise the extended-gcd step puts gcd(pivot, entry) < pivot at
            # (k, k).  The pivot thus only decreases, so the sweeps end.
            changed = True
            while changed:
                changed = False
                for i in range(k + 1, n):  # clear column k below the pivot
                    if M[i][k]:
                        if M[k][k] and M[i][k] % M[k][k] == 0:
                            rows(i, k, 1, 0, -(M[i][k] // M[k][k]), 1)
                        else:
                            g, x, y = _xgcd(M[k][k], M[i][k])
                            rows(i, k, x, y, -(M[i][k] // g), M[k][k] // g)
                        changed = True
                for j in range(k + 1, n):  # clear row k right of the pivot
                    if M[k][j]:
                        if M[k][k] and M[k][j] % M[k][k] == 0:
                            cols(j, k, 1, 0, -(M[k][j] // M[k][k]), 1)
                        else:
                            g, x, y = _xgcd(M[k][k], M[k][j])
                            cols(j, k, x, y, -(M[k][j] // g), M[k][k] // g)
                        changed = True
            # the pivot's gcd with d must divide every remaining entry's
            p = gcd(M[k][k], d)
            bad = next(((i, j) for i in range(k + 1, n) for j in range(k + 1, n) if M[i][j] % p), None)
            if bad is None:
                break
            M[k] = [(x + y) % d for x, y in zip(M[k], M[bad[0]])]  # add that row and start over
        diag.append(gcd(M[k][k], d))
    return diag


def det_mod(A, q: int) -> int:
    """det A mod q (q prime) by Gaussian elimination over GF(q), in [0, q)."""
    M = [[int(a) % q for a in row] for row in A]
    n = len(M)
    det = 1
    for k in range(n):
        piv = next((i for i in range(k, n) if M[i][k]), None)
        if piv is None:
            return 0
        if piv != k:
            M[k], M[piv] = M[piv], M[k]
            det = -det
        det = det * M[k][k] % q
        inv = pow(M[k][k], q - 2, q)
        for i in range(k + 1, n):
            if M[i][k]:
                f = M[i][k] * inv % q
                M[i] = [(x - f * y) % q for x, y in zip(M[i], M[k])]
    return det % q
