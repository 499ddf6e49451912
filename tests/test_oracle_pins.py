"""Pins for the oracle: each check ties an oracle function to something other
than itself (Python integers, sympy, closed forms, brute force on tiny inputs,
invariants).  CPU only.
"""
import numpy as np
import pytest
import sympy
from sympy.ntheory.modular import crt as sympy_crt

from paper_2605_19254_gb300 import inputs

EDGE_1 = [0, 1, -1, 2, -2, (1 << 63) - 1, -(1 << 63), (1 << 20), -(1 << 20), 12345678901234]


def _edge_ints(W):
    top = 64 * W - 1
    vals = [0, 1, -1, (1 << top) - 1, -(1 << top), (1 << 64) - 1, -(1 << 64), 1 << 63, -(1 << 63) - 1]
    return [v for v in vals if -(1 << top) <= v < (1 << top)]


# --------------------------------------------------------------------------- basis

def test_primes_below_match_sympy(orc):
    for bound in [1 << 26, 1 << 16, 1482912, 100]:
        got = [int(p) for p in orc.primes_below(bound, 12)]
        want, p = [], bound
        for _ in range(12):
            p = sympy.prevprime(p)
            want.append(p)
            if p == 2:
                break
        assert got == want[: len(got)]
        assert len(got) == min(12, len(want))


def test_is_prime_matches_sympy(orc):
    for n in list(range(0, 2000)) + [67108859, 67108861, 2**31 - 1, 2**32 - 5, 2**32 - 1]:
        assert orc.is_prime(n) == sympy.isprime(n), n


def test_basis_minimal_and_covering(orc):
    # |C| <= 4096 * 2^20 * 2^511 = 2^543 for the 4096 x 4096 by 4096 x 256 product
    pr = [int(p) for p in orc.basis(1 << 26, 543)]
    assert len(pr) == 21
    chain, p = [], 1 << 26
    for _ in range(21):
        p = sympy.prevprime(p)
        chain.append(p)
    assert pr == chain and pr[-1] == 67108529
    M = 1
    for p in pr:
        M *= p
    assert M > 2 ** 544 and (M - 1) // 2 >= 2 ** 543
    M_short = M // pr[-1]
    assert M_short <= 2 ** 544  # one prime fewer would not cover the bound
    # every bound bit count gives a covering, minimal basis
    for bits in [0, 1, 25, 26, 63, 100, 200]:
        pr = [int(p) for p in orc.basis(1 << 16, bits)]
        M = 1
        for p in pr:
            M *= p
        assert (M - 1) // 2 >= 2 ** bits
        assert M // pr[-1] <= 2 ** (bits + 1)


def test_fp64_prime_cap_is_maximal(orc):
    lim = 2 ** 53 - 1
    for n in [1, 2, 53, 101, 1009, 4096, 10007, 2 ** 20]:
        p = orc.fp64_prime_cap(n)
        assert n * (p - 1) ** 2 + (p - 1) < lim
        assert n * p ** 2 + p >= lim
    # float estimate of the closed form p ~ 1 + sqrt(2^53 / n)
    assert abs(orc.fp64_prime_cap(4096) - (1 + (2 ** 53 / 4096) ** 0.5)) < 2
    assert sympy.prevprime(orc.fp64_prime_cap(4096) + 1) == 1482907


# --------------------------------------------------------------------------- reduce

@pytest.mark.parametrize("W", [1, 2, 8])
def test_reduce_matches_python_mod(orc, W):
    X = inputs.random_words(1, f"red{W}", (9, 7), W)
    edge = orc.ints_to_words(np.array(_edge_ints(W), dtype=object).reshape(1, -1), W)
    primes = [int(p) for p in orc.primes_below(1 << 26, 5)] + [3, 65521, 2147483647]
    for mat in (X, edge):
        res = orc.reduce(mat, primes)
        vals = orc.words_to_ints(mat)
        for i, p in enumerate(primes):
            want = np.vectorize(lambda v: v % p, otypes=[object])(vals)
            assert (res[i].astype(object) == want).all()


def test_reduce_int64_small_is_identity_mod(orc):
    a = np.array([[0, 1, -1, 1 << 20, -(1 << 20), 67108858]], dtype=np.int64)
    res = orc.reduce(inputs.int64_to_words(a), [67108859])
    assert res[0].tolist() == [[0, 1, 67108858, 1 << 20, 67108859 - (1 << 20), 67108858]]


# --------------------------------------------------------------------------- matmul

def _py_matmul(a, b):
    M, K = a.shape
    N = b.shape[1]
    return np.array([[sum(a[m, k] * b[k, n] for k in range(K)) for n in range(N)] for m in range(M)],
                    dtype=object)


@pytest.mark.parametrize("shape,Wa,Wb", [((3, 5, 2), 1, 8), ((1, 1, 1), 2, 2), ((4, 9, 6), 8, 1),
                                          ((2, 17, 3), 3, 5)])
def test_matmul_bruteforce(orc, shape, Wa, Wb):
    M, K, N = shape
    A = inputs.random_words(7, "mA", (M, K), Wa)
    B = inputs.random_words(7, "mB", (K, N), Wb)
    # plant extremes into the first row / column
    A[0, 0] = orc.ints_to_words([-(1 << (64 * Wa - 1))], Wa)[0]
    B[0, -1] = orc.ints_to_words([-(1 << (64 * Wb - 1))], Wb)[0]
    Wc = Wa + Wb + 1
    C = orc.matmul(A, B, Wc)
    want = _py_matmul(orc.words_to_ints(A), orc.words_to_ints(B))
    assert (orc.words_to_ints(C) == want).all()


def test_matmul_closed_forms(orc):
    # ones(M, K) times rows all equal to x  ->  K * x in every row
    M, K, N = 3, 11, 4
    x = orc.words_to_ints(inputs.random_words(3, "x", (N,), 8))
    A = inputs.int64_to_words(np.ones((M, K), dtype=np.int64))
    B = orc.ints_to_words(np.array([list(x)] * K, dtype=object), 8)
    C = orc.words_to_ints(orc.matmul(A, B, 9))
    assert all(C[m, n] == K * x[n] for m in range(M) for n in range(N))
    # identity times B is B
    eye = inputs.int64_to_words(np.eye(K, dtype=np.int64))
    Bw = inputs.random_words(4, "b", (K, N), 8)
    assert (orc.matmul(eye, Bw, 8) == Bw).all()
    # the most negative operands: 4 * (-2^63)(-2^511) = 2^576, exactly word 9 set
    A = orc.ints_to_words(np.array([[-(1 << 63)] * 4], dtype=object), 1)
    B = orc.ints_to_words(np.array([[-(1 << 511)]] * 4, dtype=object), 8)
    C = orc.matmul(A, B, 10)
    assert C[0, 0].tolist() == [0] * 9 + [1]
    _, ok = orc.matmul(A, B, 9, allow_overflow=True)
    assert not ok
    # a sign pattern whose products cancel to zero
    A = inputs.int64_to_words(np.array([[5, -5, 7, -7]], dtype=np.int64))
    B = orc.ints_to_words(np.array([[1 << 300], [1 << 300], [-(1 << 500)], [-(1 << 500)]], dtype=object), 8)
    assert orc.words_to_ints(orc.matmul(A, B, 9))[0, 0] == 0


def test_matmul_freivalds(orc):
    M, K, N = 40, 33, 12
    A = inputs.rns_matmul_workload(5, M, K, N, 20, 8)[0]
    B = inputs.random_words(5, "fB", (K, N), 8)
    C = orc.words_to_ints(orc.matmul(A, B, 9))
    a, b = orc.words_to_ints(A), orc.words_to_ints(B)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = [int(t) for t in rng.integers(-1000, 1000, N)]
        bv = [sum(b[k, n] * v[n] for n in range(N)) for k in range(K)]
        lhs = [sum(a[m, k] * bv[k] for k in range(K)) for m in range(M)]
        rhs = [sum(C[m, n] * v[n] for n in range(N)) for m in range(M)]
        assert lhs == rhs


# --------------------------------------------------------------------------- residue gemm

def test_residue_gemm_matches_exact_product(orc):
    M, K, N = 6, 29, 5
    A, B = inputs.rns_matmul_workload(11, M, K, N, 20, 8)
    primes = [int(p) for p in orc.basis(1 << 26, 20 + 511 + 5)]
    C = orc.words_to_ints(orc.matmul(A, B, 9))
    Ares = orc.reduce(A, primes)
    Bres = orc.reduce(B, primes)
    got = orc.residue_gemm(Ares, Bres, primes)
    for i, p in enumerate(primes):
        assert (got[i].astype(object) == np.vectorize(lambda v: v % p, otypes=[object])(C)).all()
    # centered representatives and a shared A (stride 0) give the same residues
    a_small = inputs.words_low_int64(A).astype(np.int32)
    got_shared = orc.residue_gemm(a_small, Bres, primes)
    assert (got_shared == got).all()
    pr = np.array(primes, dtype=np.int64)[:, None, None]
    Bc = Bres.astype(np.int64)
    Bc = np.where(Bc > (pr - 1) // 2, Bc - pr, Bc).astype(np.int32)
    assert (orc.residue_gemm(Ares, Bc, primes) == got).all()


def test_residue_gemm_bruteforce_extremes(orc):
    p = 67108859
    h = (p - 1) // 2
    for val_a, val_b in [(h, h), (-h, h), (p - 1, p - 1), (-(p - 1), p - 1)]:
        K = 37
        A = np.full((2, K), val_a, dtype=np.int32)
        B = np.full((1, K, 3), val_b, dtype=np.int32)
        got = orc.residue_gemm(A, B, [p])
        assert (got == (K * val_a * val_b) % p).all()


# --------------------------------------------------------------------------- crt

def test_crt_roundtrip_and_endpoints(orc):
    primes = [int(p) for p in orc.basis(1 << 26, 543)]
    M = 1
    for p in primes:
        M *= p
    h = (M - 1) // 2
    vals = [0, 1, -1, h, -h, h - 1, -h + 1, 2 ** 543, -(2 ** 543)]
    vals += list(orc.words_to_ints(inputs.random_words(2, "crt", (20,), 8)))
    X = orc.ints_to_words(np.array(vals, dtype=object).reshape(1, -1), 9)
    r = orc.reduce(X, primes)
    back = orc.words_to_ints(orc.crt(r, primes, 9))
    assert list(back[0]) == vals


def test_crt_matches_sympy_on_random_residues(orc):
    primes = [int(p) for p in orc.primes_below(1 << 26, 7)]
    rng = np.random.default_rng(3)
    r = np.stack([rng.integers(0, p, 16) for p in primes]).astype(np.int32)
    got = orc.words_to_ints(orc.crt(r, primes, 4))
    for e in range(16):
        want = sympy_crt(primes, [int(r[i, e]) for i in range(len(primes))], symmetric=True)[0]
        assert got[e] == want
        for i, p in enumerate(primes):
            assert got[e] % p == r[i, e]


def test_crt_rejects_bad_basis(orc):
    with pytest.raises(orc.OracleError):
        orc.crt(np.zeros((2, 3), dtype=np.int32), [7, 9], 2)
    with pytest.raises(orc.OracleError):
        orc.crt(np.zeros((2, 3), dtype=np.int32), [7, 7], 2)


# --------------------------------------------------------------------------- digits

def test_balanced_digits_unique_and_exact(orc):
    # brute force over every pair (lower digit in [-128, 127], top in [-128, 128])
    d0, d1 = np.meshgrid(np.arange(-128, 128), np.arange(-128, 129), indexing="ij")
    vals = (d0 + 256 * d1).ravel()
    assert np.unique(vals).size == vals.size  # unique representation
    got = orc.balanced_digits(vals, 2)
    assert (got[0] == d0.ravel()).all() and (got[1] == d1.ravel()).all()
    # coverage of 3 digits: every centred residue of a prime below 2^24
    r = np.concatenate([inputs.uniform_int(9, "dig", (1000,), -(1 << 23), 1 << 23),
                        np.array([(1 << 23) - 1, -(1 << 23) + 1, 8421247, -8421247])])
    dg = orc.balanced_digits(r, 3)
    assert dg[:2].min() >= -128 and dg[:2].max() <= 127 and np.abs(dg[2]).max() <= 128
    assert (sum(dg[u].astype(np.int64) << (8 * u) for u in range(3)) == r).all()
    for bad in [8421248, -8421505]:
        with pytest.raises(orc.OracleError):
            orc.balanced_digits(np.array([bad]), 3)
    with pytest.raises(orc.OracleError):
        orc.balanced_digits(np.array([1 << 20]), 2)
