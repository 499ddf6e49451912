"""GPU parity of the Smith-form driver's first phase and its initialization.

inverse_mod_p (Gauss-Jordan over GF(p) on the device) is compared with the
oracle's elimination (pinned by C A = I mod p) element by element, and with
the defining identity where the oracle is too slow.  largest_invariant_factor
is compared with the oracle's Smith form (pinned against sympy and brute
force over minors) on random matrices (s_n close to det A: the lifting runs
to Hadamard's precision), and with the planted s_n of matrices A = U diag(s) V
built from elementary operations up to n = 1024 and the paper's test matrices
(s_n far below det A: the lifting stops early)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lifting, smith  # noqa: E402
from paper_2605_19254_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def smf():
    from paper_2605_19254_gb300 import build, smf as _smf
    build.build()
    assert torch.cuda.is_available()
    return _smf


@pytest.fixture(scope="module")
def ctx(smf):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    yield c
    c.destroy()


def _words(x, W=1):
    if W == 1 and isinstance(x, np.ndarray) and x.dtype == np.int64:
        return torch.from_numpy(np.ascontiguousarray(x)[..., None]).cuda()
    x = np.asarray(x, dtype=object)
    out = np.zeros(x.shape + (W,), dtype=np.uint64)
    for idx, v in np.ndenumerate(x):
        v = int(v) % (1 << (64 * W))
        for w in range(W):
            out[idx + (w,)] = (v >> (64 * w)) & ((1 << 64) - 1)
    return torch.from_numpy(out.view(np.int64)).cuda()


def _inverse(ctx, pb, A, bits, W=1):
    n = len(A)
    C = torch.full((n, n), -1, dtype=torch.int32, device="cuda")
    ctx.inverse_mod_p(pb, _words(A, W), C, a_bits=bits)
    ctx.status_sync()
    return C.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n,bits", [(1, 20), (7, 20), (100, 30), (257, 60), (300, 20)])
def test_inverse_mod_p_matches_oracle(ctx, n, bits):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    seed = n
    while True:
        A = inputs.uniform_int(seed, "IA", (n, n), -(1 << bits), 1 << bits)
        try:
            want = lifting.inverse_mod_p(A.tolist(), p)
            break
        except ValueError:
            seed += 1
    assert np.array_equal(_inverse(ctx, pb, A, bits), want)
    pb.destroy()


def test_inverse_mod_p_pivots_and_wide_entries(ctx):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    # a permutation whose pivots lie more than 1024 rows below the diagonal
    n = 1100
    perm = [(i + 1030) % n for i in range(n)]  # column j has its one in row perm^-1(j)
    A = np.zeros((n, n), dtype=np.int64)
    for i in range(n):
        A[i, perm[i]] = 1
    assert np.array_equal(_inverse(ctx, pb, A, 1), A.T)
    # 100-bit entries (two words): the oracle inverts A mod p
    n = 40
    rng = np.random.default_rng(5)
    Abig = [[int(rng.integers(-(1 << 50), 1 << 50)) * (1 << 50) + int(rng.integers(0, 1 << 50)) for _ in range(n)]
            for _ in range(n)]
    want = lifting.inverse_mod_p([[v % p for v in r] for r in Abig], p)
    assert np.array_equal(_inverse(ctx, pb, Abig, 101, W=2), want)
    pb.destroy()


def test_inverse_mod_p_identity_at_n_1500(ctx):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    n = 1500
    A = inputs.uniform_int(77, "IA", (n, n), -(1 << 20), 1 << 20)
    C = _inverse(ctx, pb, A, 20)
    assert C.min() >= 0 and C.max() < p
    rows = np.random.default_rng(2).choice(n, 48, replace=False)
    assert ((C[rows] @ (A % p)) % p == np.eye(n, dtype=np.int64)[rows]).all()
    pb.destroy()


def test_inverse_mod_p_identity_at_n_5003(ctx):
    # the size of the largest Phase 1 run in the bench: 40 panels of 128 columns
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    n = 5003
    A = inputs.uniform_int(55, "IA", (n, n), -(1 << 20), 1 << 20)
    C = _inverse(ctx, pb, A, 20)
    assert C.min() >= 0 and C.max() < p
    rows = np.random.default_rng(3).choice(n, 16, replace=False)
    assert ((C[rows] @ (A % p)) % p == np.eye(n, dtype=np.int64)[rows]).all()
    pb.destroy()


@pytest.mark.parametrize("n", [50, 300])  # one-column launches; panels with a product update
def test_inverse_mod_p_singular_is_reported(ctx, smf, n):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    A = inputs.uniform_int(3, "IA", (n, n), -(1 << 20), 1 << 20)
    A[17] = A[4]  # singular over Z
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    ctx.inverse_mod_p(pb, _words(A), C, a_bits=20)
    with pytest.raises(smf.SmfError) as e:
        ctx.status_sync()
    assert e.value.code == smf.SMF_E_SINGULAR
    B = A.copy()
    B[17] = p * inputs.uniform_int(4, "IB", (n,), 1, 9)  # nonsingular over Z, singular mod p
    ctx.inverse_mod_p(pb, _words(B), C, a_bits=30)
    with pytest.raises(smf.SmfError) as e:
        ctx.status_sync()
    assert e.value.code == smf.SMF_E_SINGULAR
    # the context is usable afterwards
    A2 = inputs.uniform_int(8, "IA", (30, 30), -(1 << 20), 1 << 20)
    assert np.array_equal(_inverse(ctx, pb, A2, 20), lifting.inverse_mod_p(A2.tolist(), p))
    pb.destroy()


def _lif(ctx, A, bits, m=32, seed=1):
    At = torch.from_numpy(np.asarray(A, dtype=np.int64)[..., None].copy())
    s, secs = ctx.largest_invariant_factor(At, m=m, seed=seed, a_bits=bits)
    return s


def test_largest_invariant_factor_one_by_one(ctx, smf):
    assert _lif(ctx, [[-6]], 3) == 6
    assert _lif(ctx, [[1]], 1) == 1
    assert _lif(ctx, [[16777213 * 5]], 27) == 16777213 * 5  # p | det: the next prime is taken
    with pytest.raises(smf.SmfError) as e:
        _lif(ctx, [[0]], 1)
    assert e.value.code == smf.SMF_E_SINGULAR


@pytest.mark.parametrize("n,bits,seed", [(12, 20, 1), (30, 20, 2), (40, 8, 3)])
def test_largest_invariant_factor_matches_oracle(ctx, n, bits, seed):
    A = inputs.uniform_int(seed, "SA", (n, n), -(1 << bits), 1 << bits)
    want = smith.smith_form(A.tolist())[-1]
    assert _lif(ctx, A, bits) == want


@pytest.mark.parametrize("n,s_tail,ops", [
    (64, [2, 6, 12, 60, 120, 840], 256),                 # the constructed Smith-form workload: prod s = 870,912,000
    (200, [3, 3 * 2 ** 10, 3 * 2 ** 10 * 1009], 200),     # three non-trivial factors (28-bit entries)
    (1024, [6, 60, 2 ** 9 * 3 * 5 * 7 * 11], 1024),       # n = 1024
    (2048, [6, 60, 2 ** 9 * 3 * 5 * 7 * 11], 2048),       # n = 2048 (24-bit entries)
    (3001, [6, 60, 2 ** 9 * 3 * 5 * 7 * 11], 3001),       # above 3000: two lifting chunks queued per checkpoint
])
def test_largest_invariant_factor_planted(ctx, n, s_tail, ops):
    assert all(b % a == 0 for a, b in zip(s_tail, s_tail[1:]))  # diag(s) is in Smith form
    s = [1] * (n - len(s_tail)) + s_tail
    A = np.array(inputs.smith_known_matrix(11, s, ops), dtype=np.int64)
    bits = int(np.abs(A).max()).bit_length()
    assert _lif(ctx, A, bits) == s_tail[-1]


def test_largest_invariant_factor_host_and_device_operands_and_errors(ctx, smf):
    A = inputs.uniform_int(9, "SA", (20, 20), -(1 << 20), 1 << 20)
    want = smith.smith_form(A.tolist())[-1]
    Ad = torch.from_numpy(A[..., None].copy()).cuda()
    s, secs = ctx.largest_invariant_factor(Ad, m=16, seed=4, a_bits=20)
    assert s == want and len(secs) == 4 and secs[3] >= secs[1] >= 0
    sing = A.copy()
    sing[3] = 2 * sing[5]
    with pytest.raises(smf.SmfError) as e:
        _lif(ctx, sing, 21)
    assert e.value.code == smf.SMF_E_SINGULAR
    with pytest.raises(smf.SmfError) as e:  # n |A| beyond 64-bit residuals even with a small prime
        _lif(ctx, A, 52)
    assert e.value.code == smf.SMF_E_BOUND
    # 40-bit entries: a lifting prime below 2^16 keeps the residuals in 64-bit words
    W = inputs.uniform_int(10, "SA", (16, 16), -(1 << 40), 1 << 40)
    assert _lif(ctx, W, 40) == smith.smith_form(W.tolist())[-1]


def test_largest_invariant_factor_papers_test_matrices(ctx):
    # A_ij = i^j mod n (Section 4): against the oracle at n = 53; at n = 1009
    # against the size the paper prints for s_n (4083 bits, Section 4)
    A = inputs.vandermonde_mod(53)
    assert _lif(ctx, A, 6) == smith.smith_form(A.tolist())[-1]
    s = _lif(ctx, inputs.vandermonde_mod(1009), 10)
    assert s.bit_length() == 4083


@pytest.mark.parametrize("form,p_max", [("fp64", 0), ("limb", 1 << 26)])
def test_inverse_mod_p_one_column_path_at_large_n(smf, form, p_max):
    # n > 256 without the blocked form: the FP64 form, and a prime near 2^26 whose
    # residues take four digits (beyond the limb products)
    c = smf.Context(0, smf.SMF_FORM_FP64 if form == "fp64" else smf.SMF_FORM_INT8LIMB)
    try:
        pb = c.basis_create(10, p_max)
        p = int(pb.primes[0])
        n = 300
        A = inputs.uniform_int(21, "IA", (n, n), -(1 << 20), 1 << 20)
        want = lifting.inverse_mod_p(A.tolist(), p)
        assert np.array_equal(_inverse(c, pb, A, 20), want)
        pb.destroy()
    finally:
        c.destroy()
