"""GPU parity of the Smith-form driver (Section 2's three phases) and of its
two eliminations over Z/(m), bit-exact against the oracle.

- smith_local (the last iteration of Phase 2, one prime power at a time)
  against the oracle's Smith form: counts[t] = #{i : q^t | s_i}.
- det_mod (Phase 3's check) against the oracle's elimination over GF(q),
  itself pinned to the exact Bareiss determinant.
- smith_form against the oracle's Smith form (pinned to sympy and brute force
  over minors) on random matrices and the paper's test matrices
  A_ij = i^j mod n; against the known s of matrices built as U diag(s) V
  (the constructed workload of n = 64, and larger n); at n = 1009 on the
  paper's test matrix by the divisibility chain, prod s_i = +-det A modulo
  primes (the oracle's determinant) and the size the paper prints for s_n;
  the restart when Phase 3 rejects a candidate; singular input.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import smith  # noqa: E402
from paper_2605_19254_gb300 import inputs  # noqa: E402

FORMS = {"fp64": 0, "limb": 1}
Q62 = 4611686018427387847  # a prime below 2^62
Q31 = 2147483647


@pytest.fixture(scope="module")
def smf():
    from paper_2605_19254_gb300 import build, smf as _smf
    build.build()
    assert torch.cuda.is_available()
    return _smf


@pytest.fixture(scope="module", params=list(FORMS))
def ctx(request, smf):
    c = smf.Context(0, FORMS[request.param])
    yield c
    c.destroy()


@pytest.fixture(scope="module")
def lctx(smf):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    yield c
    c.destroy()


def _t(A, device=False):
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.int64))[..., None].copy())
    return t.cuda() if device else t


def _bits(A):
    return max(1, int(np.abs(np.asarray(A, dtype=np.int64)).max()).bit_length())


def _counts(s, q, e):
    return [sum(1 for v in s if v % q ** t == 0) for t in range(e + 1)]


# --------------------------------------------------------------------------- local Smith form

@pytest.mark.parametrize("n,seed,tail", [(30, 1, [2, 4, 12, 24, 24 * 9]), (90, 2, [3, 9, 27, 27 * 5, 27 * 25]),
                                         (257, 3, [2, 2, 6, 6 * 64, 6 * 64 * 7])])
def test_smith_local_matches_oracle(lctx, n, seed, tail):
    s = [1] * (n - len(tail)) + tail
    A = inputs.smith_known_matrix(seed, s, n)
    for q, e in [(2, 8), (3, 4), (5, 3), (7, 1), (11, 2), (2, 1), (3, 1)]:  # e = 1: modulo q itself
        assert lctx.smith_local(_t(A, device=bool(seed % 2)), q, e) == _counts(s, q, e), (q, e)


def test_smith_local_joint_prime_powers(lctx):
    # several prime powers in one joint column loop (the last iteration of Phase 2)
    n = 120
    tail = [2, 6, 6 * 5, 6 * 25 * 7, 6 * 25 * 49 * 11, 6 * 25 * 49 * 121 * 13]
    s = [1] * (n - len(tail)) + tail
    A = inputs.smith_known_matrix(8, s, n)
    qs, es = [2, 3, 5, 7, 11, 13], [3, 2, 2, 2, 2, 1]
    got = lctx.smith_local(_t(A, device=True), qs, es)
    assert got == [_counts(s, q, e) for q, e in zip(qs, es)]
    B = inputs.uniform_int(6, "LS", (30, 30), -40, 40)
    sb = smith.smith_form(B.tolist())
    qs = [2, 3, 5, 7, 11, 13, 17, 19, 23]  # beyond eight lanes: sixteen
    assert lctx.smith_local(_t(B), qs, [4] * len(qs)) == [_counts(sb, q, 4) for q in qs]
    assert lctx.smith_local(_t(B), [2, 1000003], [40, 2]) == [_counts(sb, 2, 40), _counts(sb, 1000003, 2)]


def test_smith_local_random_and_wide_moduli(lctx):
    # random matrices against the oracle's Smith form; q^e above 2^31 (64-bit arithmetic)
    for n, seed in [(12, 4), (25, 5)]:
        A = inputs.uniform_int(seed, "LS", (n, n), -40, 40)
        s = smith.smith_form(A.tolist())
        for q, e in [(2, 40), (3, 25), (2, 3), (2, 1), (3, 1)]:
            assert lctx.smith_local(_t(A), q, e) == _counts(s, q, e)
    A = np.diag([1, 1, 1 << 35, 3]).astype(np.int64)
    A[0, 3] = 5
    s = smith.smith_form(A.tolist())
    assert lctx.smith_local(_t(A), 2, 40) == _counts(s, 2, 40)
    assert lctx.smith_local(_t(np.zeros((0, 0))), 2, 3) == [0, 0, 0, 0]


# --------------------------------------------------------------------------- det mod q

@pytest.mark.parametrize("n", [1, 2, 50, 300, 1009])
def test_det_mod_matches_oracle(lctx, orc, n):
    A = inputs.uniform_int(n, "DM", (n, n), -(1 << 20), 1 << 20)
    for q in (Q62, Q31, 1000003):
        assert lctx.det_mod(_t(A, device=n % 2 == 0), q) == orc.det_mod(A, q), q
    # several primes in lockstep (Phase 3's form): four 31-bit primes, then six (two loops)
    qs = [2147483647, 2147483629, 2147483587, 2147483579]
    assert lctx.det_mod(_t(A), qs) == [orc.det_mod(A, q) for q in qs]
    qs6 = qs + [1000003, 1000033]
    assert lctx.det_mod(_t(A), qs6) == [orc.det_mod(A, q) for q in qs6]


def test_det_mod_blocked(lctx, orc):
    # above 2560 the determinants run by panels of 16 columns (pivot search and
    # panel update per column, the panel's pivot rows, one trailing pass per
    # panel): four 31-bit primes in lockstep against the oracle, a ragged last
    # panel (n = 2600), and a column with no joint unit pivot, which falls back
    # to the column loop and then to one prime at a time
    n = 2600
    A = inputs.uniform_int(n, "DB", (n, n), -(1 << 20), 1 << 20)
    qs = [2147483647, 2147483629, 2147483587, 2147483579]
    assert lctx.det_mod(_t(A), qs) == [orc.det_mod(A, q) for q in qs]
    C = np.eye(n, dtype=np.int64)
    C[0, 0] = 1000003  # zero modulo 1000003 only: det = 1000003
    assert lctx.det_mod(_t(C), [Q31, 1000003]) == [1000003, 0]


@pytest.fixture(scope="module")
def pctx(smf):
    # every elimination of this context by panels of 16 columns, whatever its size
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    c.set_elim_panels(1)
    yield c
    c.destroy()


def test_local_forms_and_dets_by_panels_match_oracle(pctx, orc):
    # the panel elimination at every size: local forms whose deferred columns
    # stay live across panels (planted factors; columns with no unit modulo q
    # from the start), ragged last panels, lockstep groups of four, two and one
    # 32-bit lanes next to 64-bit ones; determinants, with the fallback to the
    # column loop; the whole Smith form; against the oracle
    for n, seed, tail in [(30, 1, [2, 4, 12, 24, 24 * 9]), (257, 3, [2, 2, 6, 6 * 64, 6 * 64 * 7]),
                          (100, 4, [2] * 20 + [6] * 10 + [30] * 3)]:
        s = [1] * (n - len(tail)) + tail
        A = inputs.smith_known_matrix(seed, s, n)
        for q, e in [(2, 8), (3, 4), (5, 3), (7, 1), (2, 1), (2, 40)]:
            assert pctx.smith_local(_t(A), q, e) == _counts(s, q, e), (n, q, e)
        qs, es = [2, 3, 5, 7, 11, 13], [3, 2, 2, 2, 2, 1]
        assert pctx.smith_local(_t(A, device=True), qs, es) == [_counts(s, q, e) for q, e in zip(qs, es)], n
    B = inputs.uniform_int(7, "LP", (40, 40), -40, 40)
    B[:, [0, 3, 17, 33]] *= 2
    B[:, [5, 20]] *= 3
    sb = smith.smith_form(B.tolist())
    qs = [2, 3, 5, 7, 11, 13, 17, 19, 23]
    assert pctx.smith_local(_t(B), qs, [4] * len(qs)) == [_counts(sb, q, 4) for q in qs]
    for n in (1, 17, 50, 300):
        A = inputs.uniform_int(n, "DM", (n, n), -(1 << 20), 1 << 20)
        qs = [2147483647, 2147483629, 2147483587, 2147483579]
        assert pctx.det_mod(_t(A), qs) == [orc.det_mod(A, q) for q in qs], n
        assert pctx.det_mod(_t(A), 1000003) == orc.det_mod(A, 1000003), n
    C = np.eye(40, dtype=np.int64)
    C[0, 0] = 1000003  # zero modulo 1000003 only: det = 1000003
    assert pctx.det_mod(_t(C), [Q31, 1000003]) == [1000003, 0]
    A = inputs.vandermonde_mod(53)
    got, _, _ = pctx.smith_form(_t(A), seed=3, a_bits=_bits(A))
    assert got == smith.smith_form(A.tolist())
    with pytest.raises(Exception):
        pctx.set_elim_panels(-1)


def test_local_forms_by_panels_at_n_2600(lctx):
    # from 1536 columns on the local forms run by panels by default: four prime
    # powers in one lockstep loop on a planted U diag(s) V, against the known s
    n = 2600
    tail = [2] * 30 + [6] * 20 + [30] * 10 + [210] * 5 + [420] * 2
    s = [1] * (n - len(tail)) + tail
    A = inputs.smith_known_matrix_np(12, s, n)
    qs, es = [2, 3, 5, 7], [3, 2, 2, 1]
    assert lctx.smith_local(_t(A), qs, es) == [_counts(s, q, e) for q, e in zip(qs, es)]
    assert lctx.smith_local(_t(A), 3, 2) == _counts(s, 3, 2)  # one lane


def test_det_mod_singular_and_pivots(lctx, orc):
    A = inputs.uniform_int(7, "DM", (40, 40), -9, 9)
    A[5] = 3 * A[11]
    assert lctx.det_mod(_t(A), Q62) == 0
    B = inputs.uniform_int(8, "DM", (40, 40), -9, 9)
    B[:, 0] = 0
    B[39, 0] = 1  # column 0's only pivot sits in the last row
    assert lctx.det_mod(_t(B), Q31) == orc.det_mod(B, Q31)
    C = np.diag([1000003, 1, 1]).astype(np.int64)  # zero modulo 1000003 only
    assert lctx.det_mod(_t(C), 1000003) == 0 and lctx.det_mod(_t(C), Q31) == 1000003
    # in lockstep: the joint loop finds no pivot for column 0 and falls back per prime
    assert lctx.det_mod(_t(C), [Q31, 1000003, 1000033]) == [1000003, 0, 1000003]


# --------------------------------------------------------------------------- the Smith form

def _check_chain(s):
    assert all(v > 0 for v in s)
    assert all(b % a == 0 for a, b in zip(s, s[1:]))


def test_smith_form_constructed_config(ctx):
    # the constructed workload: A = U diag(s) V, U and V products of 4n elementary
    # operations with multipliers in [-3, 3], s = 58 ones then 2, 6, 12, 60, 120, 840
    n = 64
    tail = [2, 6, 12, 60, 120, 840]
    s = [1] * (n - len(tail)) + tail
    A = inputs.smith_known_matrix(0, s)
    got, secs, attempts = ctx.smith_form(_t(A), seed=1, a_bits=_bits(A))
    assert got == s
    assert len(secs) == 4 and secs[3] >= secs[0] > 0


@pytest.mark.parametrize("n,bits,seed", [(1, 5, 1), (2, 3, 2), (12, 20, 3), (25, 6, 4), (40, 8, 5), (33, 1, 6),
                                         (20, 40, 7)])  # 40-bit entries: a small lifting prime
def test_smith_form_matches_oracle_random(ctx, n, bits, seed):
    while True:
        A = inputs.uniform_int(seed, "SF", (n, n), -(1 << bits), 1 << bits)
        if smith.det_bareiss(A.tolist()):
            break
        seed += 100
    got, _, _ = ctx.smith_form(_t(A), seed=seed, a_bits=bits)
    assert got == smith.smith_form(A.tolist())


@pytest.mark.parametrize("n", [23, 53])
def test_smith_form_papers_test_matrices(ctx, n):
    # A_ij = i^j mod n (Section 4): several invariant factors above 2^62 (n = 53:
    # 112, 68 and 66 bits) ahead of a run of small ones
    A = inputs.vandermonde_mod(n)
    got, _, _ = ctx.smith_form(_t(A), seed=3, a_bits=_bits(A))
    assert got == smith.smith_form(A.tolist())


def test_smith_form_papers_primes_3_to_53(ctx):
    # Section 4.2's verification sweep over the test matrices A_ij = i^j mod n for
    # every prime n from 3 to 53: the divisibility chain, the oracle's Smith form
    # (itself pinned to sympy), and prod s_i = |det A| (exact, fraction-free)
    for n in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53):
        A = inputs.vandermonde_mod(n)
        got, _, _ = ctx.smith_form(_t(A), seed=n, a_bits=_bits(A))
        _check_chain(got)
        assert got == smith.smith_form(A.tolist()), n
        assert math.prod(got) == abs(smith.det_bareiss(A.tolist())), n


@pytest.mark.parametrize("n,tail,ops", [
    (100, [2, 2, 4, 4 * 3, 4 * 3 * 5, 4 * 3 * 5 * 49, 4 * 3 * 5 * 49 * 11], 100),
    (256, [3] * 20 + [9, 9 * 64, 9 * 64 * 1009], 96),  # 21 invariant factors divisible by 3
])
def test_smith_form_planted(ctx, n, tail, ops):
    s = [1] * (n - len(tail)) + tail
    A = inputs.smith_known_matrix(5, s, ops)
    got, _, _ = ctx.smith_form(_t(A, device=True), seed=2, a_bits=_bits(A))
    assert got == s


def test_smith_form_papers_matrix_1009(lctx, orc):
    # n = 1009: the divisibility chain, prod s_i = +-det A (one sign) modulo
    # primes from the oracle's elimination, and s_n of 4083 bits (Section 4)
    A = inputs.vandermonde_mod(1009)
    got, secs, _ = lctx.smith_form(_t(A), seed=1, a_bits=10)
    _check_chain(got)
    assert got[-1].bit_length() == 4083
    signs = set()
    for q in (Q62, 4611686018427387817, 2305843009213693951):
        prod = 1
        for v in got:
            prod = prod * (v % q) % q
        d = orc.det_mod(A, q)
        assert d in (prod, (q - prod) % q)
        signs.add(1 if d == prod else -1)
    assert len(signs) == 1
    assert sum(1 for v in got if v > 1) > 0


def test_smith_form_restarts_when_phase3_rejects(lctx, smf):
    A = inputs.vandermonde_mod(23)
    want = smith.smith_form(A.tolist())
    lctx.debug_inject(smf.SMF_INJECT_WRONG_SMITH)
    got, _, attempts = lctx.smith_form(_t(A), seed=4, a_bits=5)
    assert got == want and attempts == 2
    lctx.debug_inject(smf.SMF_INJECT_WRONG_SMITH_ALWAYS)
    with pytest.raises(smf.SmfError) as e:
        lctx.smith_form(_t(A), seed=4, a_bits=5)
    assert e.value.code == smf.SMF_E_RETRY_EXHAUSTED
    got, _, attempts = lctx.smith_form(_t(A), seed=4, a_bits=5)  # the flag cleared
    assert got == want and attempts == 1


def test_smith_form_singular_and_errors(lctx, smf):
    A = inputs.uniform_int(9, "SF", (20, 20), -50, 50)
    A[7] = A[2] - A[3]
    with pytest.raises(smf.SmfError) as e:
        lctx.smith_form(_t(A), a_bits=8)
    assert e.value.code == smf.SMF_E_SINGULAR
    with pytest.raises(smf.SmfError) as e:
        lctx.smith_form(_t(np.zeros((1, 1))), a_bits=1)
    assert e.value.code == smf.SMF_E_SINGULAR
    assert lctx.smith_form(_t([[-7]]), a_bits=3)[0] == [7]


def test_fp64_peak_probe(lctx):
    # the FP64 form's roofline: a plausible FP64 FMA rate for a GB300 (nominal 1.25 TFLOP/s)
    t = lctx.fp64_peak()
    assert 0.3 < t < 10.0


def test_smith_form_dense_random_10007(lctx):
    # the dense random n = 10007 workload (entries in [-100, 100]): the divisibility
    # chain, and prod s_i = +-det A (one sign for all) modulo the eight primes below
    # 2^62 whose determinants the oracle wrote to tests/golden/config3_det_mod.txt
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "config3_det_mod.txt")
    rows = [line.split() for line in open(path) if not line.startswith("#")]
    n, bound, seed = int(rows[0][1]), int(rows[0][3]), int(rows[0][5])
    dets = [(int(q), int(d)) for q, d in rows[1:]]
    assert len(dets) == 8
    A = inputs.smith_dense_matrix(n, bound, seed)
    got, secs, _ = lctx.smith_form(_t(A), seed=1, a_bits=7)
    assert len(got) == n
    _check_chain(got)
    signs = set()
    for q, d in dets:
        prod = 1
        for v in got:
            prod = prod * (v % q) % q
        assert d in (prod, (q - prod) % q), q
        signs.add(1 if d == prod else -1)
    assert len(signs) == 1
