"""The seeded input generators that the oracle checks, the GPU tests and the
bench share (paper_2605_19254_gb300/inputs.py), on the CPU.

- The counter-based splitmix64 streams equal the published generator run as a
  state machine (Steele, Lea and Flood, 2014; restated here with Python
  integers): draw j of the stream with key k is the (j+1)-th output of the
  generator seeded with k.
- uniform_int stays in its closed range and covers both ends; the words of
  random_words and int64_to_words are two's complement values of the stated
  width; log_uniform_int stays in [lo, hi]; the test matrices A_ij = i^j mod n
  and the planted U diag(s) V constructions have the stated form.
"""
import numpy as np
import pytest

from paper_2605_19254_gb300 import inputs

MASK = (1 << 64) - 1


def reference_splitmix64(seed: int, count: int):
    x = seed & MASK
    out = []
    for _ in range(count):
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("key", [0, 1, 0x9E3779B97F4A7C15, MASK, 1234567890123456789])
def test_streams_are_the_published_generator(key):
    ref = reference_splitmix64(key, 40)
    assert [int(v) for v in inputs.splitmix64(key, 40)] == ref
    assert [int(v) for v in inputs.splitmix64(key, 15, offset=25)] == ref[25:]


def test_stream_keys_differ_by_seed_and_tag():
    keys = {inputs.stream_seed(s, t) for s in range(4) for t in ("A", "B", "dense10007", "batch_n")}
    assert len(keys) == 16
    assert inputs.stream_seed(7, "A") == inputs.stream_seed(7, "A")


def test_uniform_int_range_and_coverage():
    for lo, hi in [(-5, 5), (0, 0), (-(1 << 20), 1 << 20), (-100, 100), (3, 2 ** 40)]:
        a = inputs.uniform_int(3, "U", (20000,), lo, hi)
        assert a.dtype == np.int64 and a.min() >= lo and a.max() <= hi
        if hi - lo <= 10:
            assert set(np.unique(a)) == set(range(lo, hi + 1))
    a = inputs.uniform_int(4, "U", (200000,), -100, 100)
    counts = np.bincount(a + 100, minlength=201)
    assert counts.min() > 0.8 * 200000 / 201 and counts.max() < 1.2 * 200000 / 201
    with pytest.raises(ValueError):
        inputs.uniform_int(0, "U", (3,), 5, 4)


def test_word_layouts_are_twos_complement():
    a = np.array([0, 1, -1, 2 ** 62, -(2 ** 63)], dtype=np.int64)
    w = inputs.int64_to_words(a, 3)
    for x, row in zip(a.tolist(), w):
        v = sum(int(row[j]) << (64 * j) for j in range(3))
        assert (v - (1 << 192) if v >> 191 else v) == x
    assert np.array_equal(inputs.words_low_int64(w), a)
    r = inputs.random_words(5, "B", (1000,), 8)
    tops = r[:, 7] >> np.uint64(63)
    assert r.shape == (1000, 8) and 400 < int(tops.sum()) < 600  # signs of 512-bit values, about half negative
    for kind, value in [("min", -(1 << 511)), ("max", (1 << 511) - 1), ("minus1", -1), ("zero", 0)]:
        e = inputs.extreme_words(kind, (2, 3), 8)
        v = sum(int(e[1, 2, j]) << (64 * j) for j in range(8))
        assert (v - (1 << 512) if v >> 511 else v) == value


def test_log_uniform_sizes_and_test_matrices():
    n = inputs.log_uniform_int(1, "batch_n", 5000, 32, 1024)
    assert n.min() >= 32 and n.max() <= 1024
    # log-uniform: about half the draws below the geometric mean sqrt(32 * 1024) = 181
    assert 0.45 < float((n < 181).mean()) < 0.55
    A = inputs.vandermonde_mod(7)
    assert A.tolist()[0] == [1, 0, 0, 0, 0, 0, 0]  # 0^0 = 1
    assert all(A[i, j] == pow(i, j, 7) for i in range(1, 7) for j in range(7))
    s = [1, 1, 2, 6]
    P = inputs.smith_known_matrix(3, s, 12)
    assert round(abs(np.linalg.det(np.array(P, dtype=float)))) == 12  # |det U diag(s) V| = prod s
    assert np.array_equal(np.array(P, dtype=np.int64), inputs.smith_known_matrix_np(3, s, 12))
