"""The host big integers of the Smith-form driver (csrc/bignat.h), the
word-size modular arithmetic of its eliminations (csrc/modarith.h, compiled
here for the host), its word-size number theory (csrc/numtheory.h: the
primality test, the factoring of Phase 2's word-size modulus) and Phase 2's
Smith form of the projection over Z/(s) (csrc/pairing_smith.h), against
Python's integers, closed forms and sympy, on the CPU.

Phases 1 and 2 rebuild the lifting's p-adic values by Horner's rule (one digit
at a time, and by halves with shared powers of p), multiply them (schoolbook,
Karatsuba above 32 limbs), reduce them (Knuth's long division, Barrett's
reduction), invert units and reconstruct fractions (extended Euclid with
Lehmer's quotient runs).  tests/bignat_harness.cpp calls those routines on
lines of hexadecimal numbers; each case here checks its output with Python's
arbitrary-precision arithmetic, on edge values (zero, one, limb and word
boundaries, the add-back step of long division), the size thresholds of the
fast paths and random values.
"""
import math
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2605_19254_gb300", "csrc")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("bignat") / "bignat_harness")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "bignat_harness.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)

    def _run(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        out = r.stdout.splitlines()
        assert len(out) == len(lines)
        return out
    return _run


def h(x: int) -> str:
    return ("-" if x < 0 else "") + format(abs(x), "x")


def val(s: str) -> int:
    return -int(s[1:], 16) if s.startswith("-") else int(s, 16)


def rnd(rng, limbs: int) -> int:
    return rng.getrandbits(32 * limbs) if limbs else 0


EDGE = [0, 1, 2, (1 << 32) - 1, 1 << 32, (1 << 32) + 1, (1 << 64) - 1, 1 << 64, (1 << 96) - 1,
        0x80000000 << 64, (1 << 1024) - 1, 1 << 1023]


def test_products_sums_and_compare(run):
    rng = random.Random(1)
    pairs = [(a, b) for a in EDGE for b in EDGE]
    # around the Karatsuba threshold (32 limbs), unbalanced operands, large sizes
    for la, lb in [(31, 31), (32, 32), (33, 33), (33, 32), (64, 64), (65, 40), (100, 3), (257, 256),
                   (1193, 1193), (1500, 700)]:
        pairs.append((rnd(rng, la), rnd(rng, lb)))
        pairs.append(((1 << 32 * la) - 1, (1 << 32 * lb) - 1))  # every limb all ones: longest carries
    lines = []
    for a, b in pairs:
        lines += [f"mul {h(a)} {h(b)}", f"add {h(a)} {h(b)}", f"cmp {h(a)} {h(b)}",
                  f"sub {h(max(a, b))} {h(min(a, b))}"]
    out = run(lines)
    for i, (a, b) in enumerate(pairs):
        assert val(out[4 * i]) == a * b, (a.bit_length(), b.bit_length())
        assert val(out[4 * i + 1]) == a + b
        assert int(out[4 * i + 2]) == (a > b) - (a < b)
        assert val(out[4 * i + 3]) == max(a, b) - min(a, b)


def test_signed_sums(run):
    rng = random.Random(2)
    vals = [0, 1, -1, 5, -5, (1 << 64), -(1 << 64)] + [rng.getrandbits(200) * rng.choice((1, -1)) for _ in range(8)]
    pairs = [(a, b) for a in vals for b in vals]
    out = run([f"iadd {h(a)} {h(b)}" for a, b in pairs])
    for (a, b), o in zip(pairs, out):
        assert val(o) == a + b and not (o.startswith("-") and val(o) == 0)


def test_long_division(run):
    rng = random.Random(3)
    cases = []
    for a in EDGE:
        for b in EDGE[1:]:
            cases.append((a, b))
    for la, lb in [(2, 1), (5, 2), (40, 39), (80, 33), (300, 150), (1200, 600), (3, 3), (10, 20)]:
        for _ in range(3):
            b = rnd(rng, lb) | 1
            cases.append((rnd(rng, la), b))
    # the add-back step of Algorithm D: a divisor whose top limbs make the trial
    # quotient one too large (b = 0x8000...0001 00..., a just below a multiple of b)
    for lb in (2, 3, 5):
        b = (0x80000000 << 32 * (lb - 1)) | 1
        for q in (0xFFFFFFFF, 0x7FFFFFFF, (1 << 64) - 1):
            cases += [(b * q - 1, b), (b * q, b), (b * q + b - 1, b)]
        b2 = ((1 << 32 * lb) - 1) ^ (1 << 31)
        cases += [(b2 * 0xFFFFFFFE + b2 - 1, b2), ((1 << 32 * (lb + 2)) - 1, b2)]
    out = run([f"divmod {h(a)} {h(b)}" for a, b in cases])
    for (a, b), o in zip(cases, out):
        q, r = map(val, o.split())
        assert (q, r) == divmod(a, b), (a.bit_length(), b.bit_length())


def test_gcd_xgcd_inverse_and_modular_helpers(run):
    rng = random.Random(4)
    pairs = [(0, 5), (5, 0), (1, 1), (12, 18), (2 ** 64, 2 ** 32 * 3), ((1 << 127) - 1, (1 << 89) - 1)]
    for bits in (60, 64, 65, 128, 1000, 5000):
        g = rng.getrandbits(bits // 3) | 1
        pairs.append((g * rng.getrandbits(bits), g * rng.getrandbits(bits)))
        pairs.append((rng.getrandbits(bits), rng.getrandbits(bits // 2) | 1))
    lines = []
    for a, b in pairs:
        lines += [f"gcd {h(a)} {h(b)}", f"xgcd {h(a)} {h(b)}"]
    out = run(lines)
    for i, (a, b) in enumerate(pairs):
        assert val(out[2 * i]) == math.gcd(a, b)
        g, x, y = map(val, out[2 * i + 1].split())
        assert g == math.gcd(a, b) and x * a + y * b == g
    # inverses modulo composite and prime moduli of word size and far above it (Lehmer rounds)
    mods = [7, 2 ** 61 - 1, 3 ** 40, (2 ** 127 - 1) * (2 ** 89 - 1), rng.getrandbits(4000) | 1,
            rng.getrandbits(40000) | 1]
    cases = []
    for m in mods:
        for a in (1, 2, 3, m - 1, m + 1, rng.getrandbits(m.bit_length() + 40)):
            cases.append((a, m))
    out = run([f"inv {h(a)} {h(m)}" for a, m in cases])
    for (a, m), o in zip(cases, out):
        if math.gcd(a, m) == 1:
            assert val(o) == pow(a, -1, m) and 0 <= val(o) < m
        else:
            assert o == "none"
    # mod_of (signed), mul_mod, sub_mod
    m = rng.getrandbits(300) | 1
    lines, want = [], []
    for v in (0, 1, -1, m, -m, 5 * m + 3, -(5 * m + 3), rng.getrandbits(700), -rng.getrandbits(700)):
        lines.append(f"modof {h(v)} {h(m)}")
        want.append(v % m)
    for _ in range(5):
        a, b = rng.randrange(m), rng.randrange(m)
        lines += [f"mulmod {h(a)} {h(b)} {h(m)}", f"submod {h(a)} {h(b)} {h(m)}"]
        want += [a * b % m, (a - b) % m]
    assert [val(o) for o in run(lines)] == want


def test_barrett_reciprocal(run):
    # mu = floor(B^(2n) / m): long division up to 48 limbs, above it the
    # reciprocal of the top half, a Newton step and the exact correction; every
    # size across the threshold and its recursion, moduli whose top limb is 1
    # (the largest relative error of the top-half estimate) or all ones
    rng = random.Random(8)
    ms = []
    for n in list(range(1, 120)) + [127, 128, 129, 200, 255, 256, 257, 500, 1000, 1023, 3700, 7350]:
        top = 1 << (32 * (n - 1))
        ms += [rnd(rng, n) | (1 << (32 * n - 1)), top, top + 1, (1 << (32 * n)) - 1,
               top + (1 << (32 * (n - 1))) - 1 if n > 1 else 1, top | rnd(rng, n - 1)]
    out = run([f"recip {h(m)}" for m in ms])
    for m, o in zip(ms, out):
        n = (m.bit_length() + 31) // 32
        assert val(o) == (1 << (64 * n)) // m, m.bit_length()


def test_barrett_reduction(run):
    rng = random.Random(5)
    cases = []
    for n in (1, 2, 3, 17, 60, 400, 3700):  # limbs of m; 3700 limbs: a 118,000-bit modulus
        top = 1 << (32 * n)
        for m in (rnd(rng, n) | (1 << (32 * n - 1)), (1 << (32 * (n - 1))) + 1 if n > 1 else 3, top - 1):
            for x in (0, 1, m - 1, m, m + 1, 2 * m, top * top - 1, m * (top - 1) + m - 1, rng.randrange(top * top)):
                if x < top * top:
                    cases.append((m, x))
    # inputs whose quotient estimate falls two short (the most Algorithm 14.42
    # allows, so the reduction must correct twice): moduli just above a limb
    # boundary, the inputs found by computing the estimate
    def short_by(m, x):
        n = (m.bit_length() + 31) // 32
        q = ((x >> (32 * (n - 1))) * ((1 << (64 * n)) // m)) >> (32 * (n + 1))
        return (x - q * m) // m
    for n in (2, 3):
        hits = 0
        for _ in range(100000):  # a few hundred draws suffice
            m = (1 << (32 * (n - 1))) + rng.getrandbits(8) + 1
            x = rng.randrange(1 << (64 * n))
            if short_by(m, x) == 2:
                cases.append((m, x))
                hits += 1
                if hits == 3:
                    break
        assert hits == 3
    out = run([f"barrett {h(m)} {h(x)}" for m, x in cases])
    for (m, x), o in zip(cases, out):
        assert val(o) == x % m, (m.bit_length(), x.bit_length())


def test_horner_one_digit_at_a_time_and_by_halves(run):
    rng = random.Random(6)
    lines, want = [], []
    # lifting primes (24-bit and word-size ones), digit sums as the driver forms them
    # (up to 2^54), lengths around the block of 128 digits and its doublings
    for p, cbits in [(16777213, 54), (16777213, 24), (251, 38), (3, 10), (2147483647, 31), (65521, 48)]:
        for k in (0, 1, 2, 5, 127, 128, 129, 255, 256, 257, 1000, 3584):
            c = [rng.getrandbits(cbits) for _ in range(k)]
            if k >= 3:
                c[-1] = (1 << cbits) - 1  # the largest digit in the top group
            z = sum(ct * p ** t for t, ct in enumerate(c))
            body = f"{p:x} {cbits:x} {k:x} " + " ".join(format(x, "x") for x in c)
            lines += ["horner " + body, "hsplit " + body]
            want += [z, z]
    # p^k by binary powering: exponents 0 and 1, powers of two and one below them,
    # the size of the n = 10007 Smith form's modulus (9800 digits of a 24-bit p)
    for p, k in [(3, 0), (3, 1), (3, 2), (16777213, 100), (2, 1000), (251, 4095), (251, 4096), (251, 4097),
                 (65521, 1), (2147483647, 777), (16777213, 9800)]:
        lines.append(f"pow {p:x} {k:x}")
        want.append(p ** k)
    assert [val(o) for o in run(lines)] == want


def test_rational_reconstruction_planted(run):
    rng = random.Random(7)
    lines, want = [], []
    for nb, db in [(10, 10), (64, 64), (200, 150), (3000, 2500)]:
        P = (1 << (nb + db + 2)) + rng.getrandbits(nb + db) | 1
        while True:
            b = rng.getrandbits(db) | 1
            if math.gcd(b, P) == 1:
                break
        a = rng.getrandbits(nb - 1) * rng.choice((1, -1))
        g = math.gcd(a, b)
        u = a * pow(b, -1, P) % P
        lines.append(f"rr {h(u)} {h(P)} {nb:x} {db:x}")
        want.append((a // g, b // g))
    # no fraction within the bounds: a value whose reconstruction needs a larger denominator
    P = (1 << 64) + 13
    lines.append(f"rr {h(pow(3, -1, P) * 2 ** 40 % P)} {h(P)} {8:x} {8:x}")
    want.append(None)
    out = run(lines)
    for o, w in zip(out, want):
        if w is None:
            assert o == "none"
        else:
            num, den = map(val, o.split())
            assert (num, den) == w


def _word_moduli(rng):
    # the eliminations' moduli: primes below 2^31 (Phase 3's, and the largest
    # 31-bit one), prime powers q^e below 2^31 (Phase 2's local forms), small ones
    ms = [2, 3, 4, 5, 7, 8, 9, 25, 27, 49, 1024, 3 ** 19, 5 ** 13, 7 ** 11, 2 ** 30, 2 ** 31 - 1,
          2147483629, 2147483587, 2147483579, 1000003, 65521, 16777213]
    ms += [rng.randrange(2, 1 << 31) for _ in range(20)]
    return ms


def test_word_inverse_and_reciprocal_product(run):
    rng = random.Random(9)
    lines, want = [], []
    for m in _word_moduli(rng):
        units = [a for a in (1, 2, 3, m - 1, m - 2, m // 2, m // 2 + 1, (m + 1) // 3) if 0 < a < m]
        units += [rng.randrange(1, m) for _ in range(40)]
        for a in units:
            if math.gcd(a, m) == 1:
                lines.append(f"inv32 {a:x} {m:x}")
                want.append(pow(a, -1, m))
        for a, b in [(0, 0), (m - 1, m - 1), (m - 1, 1), (m - 2, m - 1)] + \
                [(rng.randrange(m), rng.randrange(m)) for _ in range(40)]:
            lines.append(f"mulmod32 {a:x} {b:x} {m:x}")
            want.append(a * b % m)
    # every unit of a few small moduli, exhaustively
    for m in (2, 3, 4, 9, 16, 27, 97, 125, 256, 343, 1009):
        for a in range(1, m):
            if math.gcd(a, m) == 1:
                lines.append(f"inv32 {a:x} {m:x}")
                want.append(pow(a, -1, m))
            lines.append(f"mulmod32 {a:x} {m - a:x} {m:x}")
            want.append(a * (m - a) % m)
    assert [val(o) for o in run(lines)] == want


def test_word_primality_and_factoring(run):
    sympy = pytest.importorskip("sympy")
    rng = random.Random(10)
    # primality: every n below 3000; strong pseudoprimes to the first several
    # prime bases and Carmichael numbers (composite); primes and composites near
    # 2^31, 2^62 and 2^64
    ns = list(range(3000))
    ns += [561, 1105, 1729, 41041, 825265, 321197185, 3215031751, 2152302898747, 3474749660383,
           341550071728321, 3825123056546413051]
    ns += [2 ** 31 - 1, 2 ** 31 + 11, 2 ** 61 - 1, 2 ** 62 - 57, 2 ** 64 - 59, 2 ** 64 - 1, (2 ** 31 - 1) ** 2,
           4611686018427387847]
    ns += [rng.getrandbits(62) | 1 for _ in range(200)]
    out = run([f"isprime {n:x}" for n in ns])
    for n, o in zip(ns, out):
        assert o == ("1" if sympy.isprime(n) else "0"), n
    # factoring below 2^62 (the word-size moduli of Phase 2): smooth numbers,
    # squares and cubes of primes above the trial bound, semiprimes of two
    # 31-bit primes, prime powers of small primes, random values
    p31 = [int(sympy.prevprime(2 ** 31 - k * 1000)) for k in range(4)]
    ns = [1, 2, 4, 6, 999, 1000, 1009 * 1013, 1013 ** 2, 1013 ** 3, 65521 ** 3, 2 ** 61, 3 ** 39, 2 ** 61 - 1,
          p31[0] * p31[1], p31[2] ** 2, 2 * 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23 * 29 * 31 * 37 * 41 * 43 * 47,
          840 * 1000003 * 1000033, 2 ** 20 * 3 ** 10 * 5 ** 5 * 7 ** 3]
    ns += [rng.getrandbits(rng.randrange(2, 62)) | 1 for _ in range(150)]
    out = run([f"factor {n:x}" for n in ns])
    for n, o in zip(ns, out):
        got = [] if o == "-" else sorted(int(x, 16) for x in o.split())
        want = sorted(p for p, e in sympy.factorint(n).items() for _ in range(e))
        assert got == want, n
    # word powers modulo 62-bit moduli
    cases = [(0, 0, 7), (5, 0, 1), (2, 61, 2 ** 61 - 1), (3, 2 ** 62 - 58, 2 ** 62 - 57)]
    cases += [(rng.getrandbits(64), rng.getrandbits(64), rng.getrandbits(62) | 1) for _ in range(50)]
    out = run([f"powmod {a:x} {e:x} {m:x}" for a, e, m in cases])
    for (a, e, m), o in zip(cases, out):
        assert val(o) == pow(a, e, m)


def _planted(rng, rows, cols, e, ops=None):
    """U diag(e) V over the integers (rows x cols), U and V products of
    elementary operations: its integer invariant factors are e (a divisibility
    chain, zeros last)."""
    Y = [[e[i] if i == j and i < len(e) else 0 for j in range(cols)] for i in range(rows)]
    for _ in range(ops if ops is not None else 3 * (rows + cols)):
        i, k = rng.sample(range(rows), 2) if rows > 1 else (0, 0)
        c = rng.randint(-3, 3)
        if i != k:
            Y[i] = [x + c * y for x, y in zip(Y[i], Y[k])]
        j, l = rng.sample(range(cols), 2) if cols > 1 else (0, 0)
        c = rng.randint(-3, 3)
        if j != l:
            for row in Y:
                row[j] += c * row[l]
    return Y


def _psmith_line(Y, s):
    rows, cols = len(Y), len(Y[0])
    return f"psmith {rows:x} {cols:x} {s:x} " + " ".join(format(x % s, "x") for row in Y for x in row)


def _psmith_want(e, s, rows, cols):
    # over Z/(s) the invariant factors are d_i = gcd(e_i, s) (e_i = 0 beyond the
    # rank); each pivot stands for s / d_i, and the loop ends (complete) at the
    # first d_i = s
    d = [math.gcd(e[i] if i < len(e) else 0, s) for i in range(min(rows, cols))]
    inv = []
    for di in d:
        if di == s:
            return True, inv
        inv.append(s // di)
    return False, inv


def test_projection_smith_form_over_z_mod_s(run):
    sympy = pytest.importorskip("sympy")
    from sympy.matrices.normalforms import smith_normal_form
    rng = random.Random(11)
    cases = []
    s1 = 2 ** 5 * 3 ** 3 * 5 * 7
    cases.append((_planted(rng, 6, 6, [1, 2, 6, 12, 0, 0]), [1, 2, 6, 12, 0, 0], s1))
    cases.append(([[2, 3], [3, 2]], [1, 5], 6))  # no unit entry modulo 6: Bezout steps
    cases.append(([[2, 3, 0], [0, 2, 3]], [1, 1], 6))
    cases.append((_planted(rng, 5, 3, [2, 6, 30]), [2, 6, 30], 2 ** 4 * 3 ** 2 * 5 ** 2))
    cases.append((_planted(rng, 3, 5, [1, 3, 0]), [1, 3, 0], 3 ** 7))
    # wide moduli (threads on): a 2000-bit s and a 16 x 16 block, a 20 x 12 one
    big = sympy.nextprime(1 << 1000) * sympy.nextprime(1 << 990) * 2 ** 8 * 3 ** 5
    e16 = [1] * 8 + [2, 6, 6, 12, 2 ** 8 * 3, 2 ** 8 * 3 ** 5, 0, 0]
    cases.append((_planted(rng, 16, 16, e16), e16, big))
    e20 = [1] * 6 + [3, 3 * 2 ** 7, 3 * 2 ** 7 * int(sympy.nextprime(1 << 1000))] + [0] * 3
    cases.append((_planted(rng, 20, 12, e20), e20, big))
    lines = [_psmith_line(Y, s) for Y, e, s in cases]
    wants = [_psmith_want(e, s, len(Y), len(Y[0])) for Y, e, s in cases]
    # unplanted blocks: the integer invariant factors from sympy
    for rows, cols, s in [(4, 4, 360), (5, 3, 2 ** 6 * 3 ** 3), (6, 6, 2 * 3 * 5 * 7 * 11 * 13), (3, 3, 7 ** 5)]:
        Y = [[rng.randrange(s) for _ in range(cols)] for _ in range(rows)]
        snf = smith_normal_form(sympy.Matrix(Y), domain=sympy.ZZ)
        e = sorted(abs(int(snf[i, i])) for i in range(min(rows, cols)))
        e = [v for v in e if v] + [v for v in e if not v]  # the chain, zeros last
        lines.append(_psmith_line(Y, s))
        wants.append(_psmith_want(e, s, rows, cols))
    out = run(lines)
    for o, (complete, inv) in zip(out, wants):
        assert o != "fail"
        parts = o.split()
        assert parts[0] == ("1" if complete else "0") and [int(x, 16) for x in parts[1:]] == inv, (o[:80], inv)
