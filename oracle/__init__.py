"""Oracle for the RNS exact integer matrix product (test infrastructure only).

A plain CPU implementation of what the hot path computes, written from the
paper ("A C implementation of the Smith massager algorithm", Section 3.1):
reduction modulo word-size primes, the per-prime residue products, CRT
reconstruction, conversion between RNS bases, and the exact schoolbook
product the RNS route must reproduce.
The arithmetic lives in ``oracle.c`` (plain C, OpenMP over rows); this module
only marshals numpy arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and imports nothing from it.

Parity status: every entry point here is pinned by ``tests/test_oracle_*.py``
(``-m "not gpu"``) against Python integers, sympy, closed forms and brute
force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

ORC_OK = 0
ORC_E_OVERFLOW = 1
ORC_E_INVALID = 2
ORC_E_NOMEM = 3


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            i32 = ctypes.c_int
            u64 = ctypes.c_uint64
            lib.orc_is_prime.argtypes = [u64]
            lib.orc_primes_below.argtypes = [u64, i32, P]
            lib.orc_fp64_prime_cap.argtypes = [u64]
            lib.orc_fp64_prime_cap.restype = u64
            lib.orc_basis.argtypes = [u64, i32, i32, P]
            lib.orc_reduce.argtypes = [P, i64, i64, i64, i32, P, i32, P]
            lib.orc_matmul.argtypes = [P, i64, i64, i64, i32, P, i64, i64, i32, P, i64, i32]
            lib.orc_residue_gemm.argtypes = [P, i64, P, i64, i64, i64, P, i32, P]
            lib.orc_crt.argtypes = [P, i64, P, i32, P, i32]
            lib.orc_balanced_digits.argtypes = [P, i64, i32, P]
            lib.orc_det_mod.argtypes = [P, i64, i64, u64, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# representation helpers (two's complement words <-> Python ints)
# --------------------------------------------------------------------------

def words_to_ints(w: np.ndarray) -> np.ndarray:
    """[..., W] uint64 two's complement words -> object array of Python ints."""
    w = np.asarray(w, dtype=np.uint64)
    W = w.shape[-1]
    flat = w.reshape(-1, W)
    out = np.empty(flat.shape[0], dtype=object)
    for e in range(flat.shape[0]):
        v = 0
        for j in range(W - 1, -1, -1):
            v = (v << 64) | int(flat[e, j])
        if v >> (64 * W - 1):
            v -= 1 << (64 * W)
        out[e] = v
    return out.reshape(w.shape[:-1])


def ints_to_words(x, W: int) -> np.ndarray:
    """Object/int array of Python ints -> [..., W] uint64 two's complement."""
    x = np.asarray(x, dtype=object)
    flat = x.reshape(-1)
    out = np.zeros((flat.shape[0], W), dtype=np.uint64)
    lim = 1 << (64 * W - 1)
    mask = (1 << 64) - 1
    for e in range(flat.shape[0]):
        v = int(flat[e])
        if not (-lim <= v < lim):
            raise OverflowError(f"{v} does not fit in {W} words")
        v &= (1 << (64 * W)) - 1
        for j in range(W):
            out[e, j] = (v >> (64 * j)) & mask
    return out.reshape(x.shape + (W,))


# --------------------------------------------------------------------------
# basis (Section 3.1: a run of consecutive primes just under the bound)
# --------------------------------------------------------------------------

def is_prime(n: int) -> bool:
    return bool(_load().orc_is_prime(int(n)))


def primes_below(bound: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    k = _load().orc_primes_below(int(bound), int(count), _ptr(out))
    return out[:k]


def fp64_prime_cap(n: int) -> int:
    """Largest p with n (p-1)^2 + (p-1) < 2^53 - 1 (Section 3.1)."""
    return int(_load().orc_fp64_prime_cap(int(n)))


def basis(bound: int, bits: int, cap: int = 4096) -> np.ndarray:
    """Primes descending below ``bound`` until their product exceeds 2^(bits+1)."""
    out = np.zeros(cap, dtype=np.uint32)
    L = _load().orc_basis(int(bound), int(bits), int(cap), _ptr(out))
    if L < 0:
        raise OracleError("basis: not enough primes below bound")
    return out[:L].copy()


# --------------------------------------------------------------------------
# the path
# --------------------------------------------------------------------------

def reduce(X: np.ndarray, primes) -> np.ndarray:
    """X: [rows, cols, W] uint64 -> residues [L, rows, cols] int32 in [0, p)."""
    X = np.ascontiguousarray(X, dtype=np.uint64)
    if X.ndim == 2:
        X = X[:, :, None]
    rows, cols, W = X.shape
    pr = np.ascontiguousarray(primes, dtype=np.uint32)
    out = np.zeros((pr.shape[0], rows, cols), dtype=np.int32)
    rc = _load().orc_reduce(_ptr(X), rows, cols, cols, W, _ptr(pr), pr.shape[0], _ptr(out))
    if rc != ORC_OK:
        raise OracleError(f"reduce: status {rc}")
    return out


def matmul(A: np.ndarray, B: np.ndarray, Wc: int, allow_overflow: bool = False):
    """Exact C = A B.  A: [M, K, Wa], B: [K, N, Wb] uint64 words -> [M, N, Wc]."""
    A = np.ascontiguousarray(A, dtype=np.uint64)
    B = np.ascontiguousarray(B, dtype=np.uint64)
    if A.ndim == 2:
        A = A[:, :, None]
    if B.ndim == 2:
        B = B[:, :, None]
    M, K, Wa = A.shape
    K2, N, Wb = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = np.zeros((M, N, Wc), dtype=np.uint64)
    rc = _load().orc_matmul(_ptr(A), M, K, K, Wa, _ptr(B), N, N, Wb, _ptr(C), N, Wc)
    if rc == ORC_E_OVERFLOW and allow_overflow:
        return C, False
    if rc != ORC_OK:
        raise OracleError(f"matmul: status {rc}")
    return (C, True) if allow_overflow else C


def residue_gemm(A: np.ndarray, B: np.ndarray, primes) -> np.ndarray:
    """C_i = A_i B_i mod p_i.  A: [L, M, K] or [M, K] (shared), B: [L, K, N] int32."""
    pr = np.ascontiguousarray(primes, dtype=np.uint32)
    L = pr.shape[0]
    A = np.ascontiguousarray(A, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    if A.ndim == 2:
        M, K = A.shape
        stride = 0
    else:
        _, M, K = A.shape
        stride = M * K
    _, K2, N = B.shape
    if K != K2 or B.shape[0] != L:
        raise ValueError("shape mismatch")
    C = np.zeros((L, M, N), dtype=np.int32)
    rc = _load().orc_residue_gemm(_ptr(A), stride, _ptr(B), M, N, K, _ptr(pr), L, _ptr(C))
    if rc != ORC_OK:
        raise OracleError(f"residue_gemm: status {rc}")
    return C


def crt(residues: np.ndarray, primes, W: int) -> np.ndarray:
    """residues [L, ...] canonical -> [..., W] words of the symmetric CRT value."""
    r = np.ascontiguousarray(residues, dtype=np.int32)
    pr = np.ascontiguousarray(primes, dtype=np.uint32)
    L = pr.shape[0]
    shape = r.shape[1:]
    count = int(np.prod(shape)) if shape else 1
    out = np.zeros((count, W), dtype=np.uint64)
    rc = _load().orc_crt(_ptr(r), count, _ptr(pr), L, _ptr(out), W)
    if rc != ORC_OK:
        raise OracleError(f"crt: status {rc}")
    return out.reshape(shape + (W,))


def base_convert(residues: np.ndarray, primes_from, primes_to) -> np.ndarray:
    """Section 3.1, conversion between RNS bases.

    residues [L, ...] canonical modulo ``primes_from`` -> [L', ...] canonical
    modulo ``primes_to``, for the integers x they represent taken as the
    symmetric representative in [-(M-1)/2, (M-1)/2], M = prod primes_from.
    Written as the definition of the conversion: CRT reconstruction in the
    first basis, then reduction in the second (the paper's Lagrange shortcut
    with a floating-point correction must reach this same result)."""
    pf = [int(p) for p in np.asarray(primes_from).ravel()]
    bits = sum(p.bit_length() for p in pf) + 1
    W = bits // 64 + 1
    r = np.ascontiguousarray(residues, dtype=np.int32)
    shape = r.shape[1:]
    X = crt(r.reshape(r.shape[0], -1), primes_from, W)  # [count, W]
    out = reduce(X[:, None, :], primes_to)              # [L', count, 1]
    return out.reshape((out.shape[0],) + shape)


def balanced_digits(r: np.ndarray, t: int) -> np.ndarray:
    """Signed ints [...] -> [t, ...] balanced base-256 digits in [-128, 127]."""
    r = np.ascontiguousarray(r, dtype=np.int64)
    out = np.zeros((t,) + r.shape, dtype=np.int32)
    rc = _load().orc_balanced_digits(_ptr(r), r.size, t, _ptr(out))
    if rc != ORC_OK:
        raise OracleError(f"balanced_digits: status {rc}")
    return out


def det_mod(A: np.ndarray, q: int) -> int:
    """det A mod q for a square int64 matrix and a prime q < 2^63 (Section 2:
    the invariant factors multiply to |det A|), by Gaussian elimination over
    GF(q) in C with OpenMP over the rows of each step."""
    A = np.ascontiguousarray(A, dtype=np.int64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix required")
    out = np.zeros(1, dtype=np.uint64)
    rc = _load().orc_det_mod(_ptr(A), A.shape[0], A.shape[0], int(q), _ptr(out))
    if rc != ORC_OK:
        raise OracleError(f"det_mod: status {rc}")
    return int(out[0])
