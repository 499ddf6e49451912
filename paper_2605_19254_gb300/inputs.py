"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module holds random-number generation and data layout only: none of the
RNS arithmetic.  The generator is splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", 2014) used as a counter-based
generator: draw ``j`` of stream ``s`` is the splitmix64 output for state
``s + (j + 1) * 0x9E3779B97F4A7C15``.  Streams are derived from a user seed
and a tag so that each tensor of a workload has its own stream.

Integer layout: a big-integer matrix is a uint64 array ``[rows, cols, W]``
holding W little-endian 64-bit words of the two's complement value per entry.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, tag: str) -> int:
    """A 64-bit stream key from a user seed and a tensor tag."""
    h = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for ch in tag.encode():
            h = _mix(h + _GAMMA * np.uint64(ch + 1))
    return int(h)


def splitmix64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of the stream with the given key (uint64)."""
    j = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + j * _GAMMA
        return _mix(z)


def uniform_int(seed: int, tag: str, shape, lo: int, hi: int) -> np.ndarray:
    """int64 array uniform on [lo, hi] (inclusive), by rejection on masked draws."""
    n = int(np.prod(shape))
    span = hi - lo + 1
    if span <= 0 or span > (1 << 62):
        raise ValueError("range")
    bits = (span - 1).bit_length()
    mask = np.uint64((1 << bits) - 1)
    key = stream_seed(seed, tag)
    out = np.empty(n, dtype=np.int64)
    filled = 0
    offset = 0
    while filled < n:
        want = max(1024, int((n - filled) * 2.2))
        d = splitmix64(key, want, offset) & mask
        offset += want
        d = d[d < np.uint64(span)]
        take = min(d.shape[0], n - filled)
        out[filled:filled + take] = d[:take].astype(np.int64) + lo
        filled += take
    return out.reshape(shape)


def random_words(seed: int, tag: str, shape, W: int) -> np.ndarray:
    """[*shape, W] uint64: uniform signed integers in [-2^(64W-1), 2^(64W-1))."""
    n = int(np.prod(shape)) * W
    return splitmix64(stream_seed(seed, tag), n).reshape(tuple(shape) + (W,))


def int64_to_words(a: np.ndarray, W: int = 1) -> np.ndarray:
    """Sign-extend an int64 array to [..., W] two's complement words."""
    a = np.asarray(a, dtype=np.int64)
    out = np.empty(a.shape + (W,), dtype=np.uint64)
    out[..., 0] = a.view(np.uint64)
    ext = np.where(a < 0, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
    for j in range(1, W):
        out[..., j] = ext
    return out


def words_low_int64(w: np.ndarray) -> np.ndarray:
    """Lowest word of [..., W] words reinterpreted as int64 (exact when W=1)."""
    return np.ascontiguousarray(w[..., 0]).view(np.int64)


# ---------------------------------------------------------------------------
# Workloads with the paper's shapes (RNS matmul of an n x n small-entry matrix
# by an n x m big-entry matrix, Section 3.1 and the lifting products).
# ---------------------------------------------------------------------------

def rns_matmul_workload(seed: int, M: int, K: int, N: int, a_bits: int, b_words: int):
    """A: M x K int64 uniform in [-2^a_bits, 2^a_bits] (as [M, K, 1] words);
    B: K x N uniform signed (64 b_words)-bit integers ([K, N, b_words] words)."""
    A = uniform_int(seed, "A", (M, K), -(1 << a_bits), 1 << a_bits)
    B = random_words(seed, "B", (K, N), b_words)
    return int64_to_words(A, 1), B


def extreme_words(kind: str, shape, W: int) -> np.ndarray:
    """Adversarial constant matrices: 'min' = -2^(64W-1), 'max' = 2^(64W-1)-1,
    'minus1' = -1, 'zero' = 0."""
    out = np.zeros(tuple(shape) + (W,), dtype=np.uint64)
    if kind == "min":
        out[..., W - 1] = np.uint64(1 << 63)
    elif kind == "max":
        out[...] = np.uint64(0xFFFFFFFFFFFFFFFF)
        out[..., W - 1] = np.uint64(0x7FFFFFFFFFFFFFFF)
    elif kind == "minus1":
        out[...] = np.uint64(0xFFFFFFFFFFFFFFFF)
    elif kind != "zero":
        raise ValueError(kind)
    return out


def log_uniform_int(seed: int, tag: str, count: int, lo: int, hi: int) -> np.ndarray:
    """count integers round(exp(U(ln lo, ln hi))), U from 53-bit draws."""
    u = (splitmix64(stream_seed(seed, tag), count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    n = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def batched_shapes(seed: int, count: int = 512, lo: int = 32, hi: int = 1024, ks=(7, 20)):
    """(n_i, k_i) of a batch of square matrices: n log-uniform in [lo, hi], k
    cycling through ks (the batched Smith-form workload's sizes)."""
    n = log_uniform_int(seed, "batch_n", count, lo, hi)
    return [(int(n[i]), int(ks[i % len(ks)])) for i in range(count)]


def batched_workload(seed: int, count: int = 512, r: int = 128, b_words: int = 8, lo: int = 32, hi: int = 1024,
                     ks=(7, 20)):
    """Products A_i B_i of the batch: A_i n_i x n_i with entries uniform in
    [-2^k_i, 2^k_i], B_i n_i x r uniform signed (64 b_words)-bit integers (the
    big-entry right-hand block of the lifting products).  Returns a list of
    (n_i, k_i, A_i words, B_i words)."""
    out = []
    for i, (n, k) in enumerate(batched_shapes(seed, count, lo, hi, ks)):
        A, B = rns_matmul_workload(stream_seed(seed, f"batch{i}"), n, n, r, k, b_words)
        out.append((n, k, A, B))
    return out


def unimodular_ops(seed: int, tag: str, n: int, count: int, lo: int = -3, hi: int = 3):
    """`count` elementary operations (i, j, c): add c times line j to line i,
    i != j uniform, c uniform in [lo, hi] (zero allowed: a no-op)."""
    ij = uniform_int(seed, tag + "ij", (count, 2), 0, n - 2)
    c = uniform_int(seed, tag + "c", (count,), lo, hi)
    ops = []
    for k in range(count):
        i = int(ij[k, 0])
        j = int(ij[k, 1])
        j = j + 1 if j >= i else j  # j uniform over the other n - 1 lines
        ops.append((i, j, int(c[k])))
    return ops


def smith_known_matrix(seed: int, s, ops_per_side=None):
    """A = U diag(s) V with U, V products of elementary operations (the
    constructed test matrices of the Smith-form configs): rows of diag(s) get
    U's operations, columns get V's.  Python integers, row-major lists."""
    n = len(s)
    count = 4 * n if ops_per_side is None else ops_per_side
    A = [[int(s[i]) if i == j else 0 for j in range(n)] for i in range(n)]
    for i, j, c in unimodular_ops(seed, "U", n, count):
        if c:
            A[i] = [a + c * b for a, b in zip(A[i], A[j])]
    for i, j, c in unimodular_ops(seed, "V", n, count):
        if c:
            for row in A:
                row[i] += c * row[j]
    return A


def vandermonde_mod(n: int) -> np.ndarray:
    """The paper's test matrices (Section 4): A_ij = i^j mod n for 0 <= i, j < n
    (0^0 = 1), int64 [n, n]; nonsingular for prime n."""
    A = np.empty((n, n), dtype=np.int64)
    i = np.arange(n, dtype=np.int64)
    col = np.ones(n, dtype=np.int64) % max(n, 1)
    for j in range(n):
        A[:, j] = col
        col = col * i % n
    return A


def smith_dense_matrix(n: int, bound: int, seed: int = 0) -> np.ndarray:
    """A dense random n x n int64 matrix with entries uniform in [-bound, bound]
    (the paper's largest Smith-form dimension is n = 10007; its random
    counterpart takes bound = 100, int32-sized entries)."""
    return uniform_int(seed, f"dense{n}", (n, n), -bound, bound)


def smith_known_matrix_np(seed: int, s, ops_per_side=None) -> np.ndarray:
    """smith_known_matrix with numpy int64 rows (the same operations in the same
    order, so the same matrix), for large n; raises OverflowError if an entry
    would leave [-2^62, 2^62]."""
    n = len(s)
    count = 4 * n if ops_per_side is None else ops_per_side
    A = np.zeros((n, n), dtype=np.int64)
    A[np.arange(n), np.arange(n)] = np.asarray([int(v) for v in s], dtype=np.int64)
    lim = 1 << 62
    for i, j, c in unimodular_ops(seed, "U", n, count):
        if c:
            A[i] += c * A[j]
            if np.abs(A[i]).max() >= lim:
                raise OverflowError("entries beyond 2^62")
    for i, j, c in unimodular_ops(seed, "V", n, count):
        if c:
            A[:, i] += c * A[:, j]
            if np.abs(A[:, i]).max() >= lim:
                raise OverflowError("entries beyond 2^62")
    return A


def divisibility_chain(seed: int, tag: str, count: int, factors=(1, 2, 3, 5)):
    """`count` integers s_1 | s_2 | ... : s_1 = 2 and each next one the previous
    times a factor drawn uniformly from `factors`."""
    out, cur = [], 2
    f = uniform_int(seed, tag, (count,), 0, len(factors) - 1)
    for t in range(count):
        if t:
            cur *= factors[int(f[t])]
        out.append(cur)
    return out


def batched_smith_workload(seed: int, count: int = 512, lo: int = 32, hi: int = 1024, ks=(7, 20)):
    """The batched Smith-form workload: `count` matrices, n log-uniform in
    [lo, hi]; even items uniform in [-2^k, 2^k] (k cycling through ks), odd items
    U diag(s) V built like the constructed workload (elementary operations with
    multipliers in [-3, 3]; 2n per side, which keeps entries below 2^40 at
    n = 1024) with s ending in a random divisibility chain of 4 to 8 factors.
    Returns (n, bits, A, planted s or None) per item."""
    out = []
    for i, (n, k) in enumerate(batched_shapes(seed, count, lo, hi, ks)):
        sd = stream_seed(seed, f"smith{i}")
        if i % 2 == 0:
            A = uniform_int(sd, "A", (n, n), -(1 << k), 1 << k)
            out.append((n, k + 1, A, None))
        else:
            tail = divisibility_chain(sd, "s", int(uniform_int(sd, "t", (1,), 4, 8)[0]))
            s = [1] * (n - len(tail)) + tail
            A = smith_known_matrix_np(sd, s, 2 * n)
            out.append((n, max(1, int(np.abs(A).max()).bit_length()), A, s))
    return out
