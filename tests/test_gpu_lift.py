"""GPU parity of p-adic lifting against the oracle's recurrence (pinned to
the definition A^-1 B mod p^k), bit-exact, in both forms: the digits X_i and
the residual R_k; a wrong inverse is reported by the remainder check; a bound
that does not fit 64-bit residuals is refused."""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lifting  # noqa: E402
from paper_2605_19254_gb300 import inputs  # noqa: E402

FORMS = {"fp64": 0, "limb": 1}


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


def _system(seed, n, m, p, a_bits=20, b_bits=40):
    while True:
        A = inputs.uniform_int(seed, "LA", (n, n), -(1 << a_bits), 1 << a_bits)
        try:
            C = lifting.inverse_mod_p(A.tolist(), p)
            break
        except ValueError:
            seed += 1
    B = inputs.uniform_int(seed, "LB", (n, m), -(1 << b_bits), 1 << b_bits)
    return A, B, C


def _words(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.int64)[..., None]).cuda()


@pytest.mark.parametrize("n,m,k", [(5, 1, 4), (64, 3, 12), (150, 20, 6)])
def test_lift_matches_oracle(ctx, n, m, k):
    pb = ctx.basis_create(10)  # one prime, the largest below the form's bound
    p = int(pb.primes[0])
    A, B, C = _system(n + m, n, m, p)
    want_X, want_R = lifting.lift_recurrence(A, B, p, k, C)
    X = torch.full((k, n, m), -1, dtype=torch.int32, device="cuda")
    R = torch.zeros((n, m, 1), dtype=torch.int64, device="cuda")
    Ad, Bd = _words(A), _words(B)
    ctx.padic_lift(pb, Ad, torch.from_numpy(C.astype(np.int32)).cuda(), Bd, k, X, R, a_bits=20, b_bits=40)
    ctx.status_sync()
    got_X = X.cpu().numpy()
    for i in range(k):
        assert np.array_equal(got_X[i], want_X[i]), f"digit {i}"
    assert np.array_equal(R.cpu().numpy()[..., 0], want_R)
    if n <= 5:  # and the defining identity, in Python integers
        S = sum(got_X[i].astype(object) * p ** i for i in range(k))
        lhs = np.array(A, dtype=object).dot(S) + p ** k * want_R.astype(object)
        assert (lhs == np.array(B, dtype=object)).all()
    pb.destroy()


def test_lift_reports_a_wrong_inverse_and_bounds(ctx, smf):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    n, m, k = 16, 2, 3
    A, B, C = _system(7, n, m, p)
    bad = C.copy()
    bad[3, 5] = (bad[3, 5] + 1) % p
    X = torch.zeros((k, n, m), dtype=torch.int32, device="cuda")
    R = torch.zeros((n, m, 1), dtype=torch.int64, device="cuda")
    ctx.padic_lift(pb, _words(A), torch.from_numpy(bad.astype(np.int32)).cuda(), _words(B), k, X, R, a_bits=20,
                   b_bits=40)
    with pytest.raises(smf.SmfError) as e:
        ctx.status_sync()
    assert e.value.code == smf.SMF_E_INVALID
    ctx.status_sync()  # the status word was cleared: the context is usable
    with pytest.raises(smf.SmfError) as e:  # 40-bit A with a 24/26-bit p and n = 16: beyond 62 bits
        ctx.padic_lift(pb, _words(A), torch.from_numpy(C.astype(np.int32)).cuda(), _words(B), k, X, R, a_bits=40,
                       b_bits=40)
    assert e.value.code == smf.SMF_E_BOUND
    pb.destroy()


# (p_max, a_bits, n, m, k).  The limb form's step kernels take the residue
# products' K-split partials and the product basis of A X_i as the plan gives
# them: a 10-bit p (two-digit C R_i, one product prime); a 6-bit A (one-digit
# A X_i product, two primes); a 28-bit A that no prime holds centred (per-prime
# A digits, three primes); n = 150 (K splits in both products).
@pytest.mark.parametrize("p_max,a_bits,n,m,k", [(1 << 10, 6, 40, 3, 5), (0, 6, 96, 5, 4), (0, 28, 64, 7, 3),
                                                 (0, 20, 150, 65, 3)])
def test_lift_digit_and_basis_widths(ctx, p_max, a_bits, n, m, k):
    pb = ctx.basis_create(7, p_max)  # one prime: 7 + 2 bits fit a 10-bit prime
    p = int(pb.primes[0])
    A, B, C = _system(3 * n + m, n, m, p, a_bits, 40)
    want_X, want_R = lifting.lift_recurrence(A, B, p, k, C)
    X = torch.full((k, n, m), -1, dtype=torch.int32, device="cuda")
    R = _words(B)  # in place: R is B
    ctx.padic_lift(pb, _words(A), torch.from_numpy(C.astype(np.int32)).cuda(), R, k, X, R, a_bits=a_bits,
                   b_bits=40)
    ctx.status_sync()
    got_X = X.cpu().numpy()
    for i in range(k):
        assert np.array_equal(got_X[i], want_X[i]), f"digit {i}"
    assert np.array_equal(R.cpu().numpy()[..., 0], want_R)
    pb.destroy()


def test_lift_zero_steps_copies_b(ctx):
    pb = ctx.basis_create(10)
    p = int(pb.primes[0])
    A, B, C = _system(11, 12, 4, p)
    X = torch.full((1, 12, 4), -1, dtype=torch.int32, device="cuda")
    R = torch.zeros((12, 4, 1), dtype=torch.int64, device="cuda")
    ctx.padic_lift(pb, _words(A), torch.from_numpy(C.astype(np.int32)).cuda(), _words(B), 0, X, R, a_bits=20,
                   b_bits=40)
    ctx.status_sync()
    assert np.array_equal(R.cpu().numpy()[..., 0], B)
    assert (X.cpu().numpy() == -1).all()
    pb.destroy()


def _inverse_mod_p_torch(A, p, dev):
    """A^-1 mod p by Gauss-Jordan over GF(p) with torch int64 ops (an input of
    the call, checked below by C A = I mod p; the oracle's own routine is too
    slow at n = 1024)."""
    n = A.shape[0]
    M = torch.cat([torch.from_numpy(A % p).to(dev), torch.eye(n, dtype=torch.int64, device=dev)], dim=1)
    for k in range(n):
        piv = k + int(torch.nonzero(M[k:, k])[0, 0])
        if piv != k:
            M[[k, piv]] = M[[piv, k]]
        M[k] = M[k] * pow(int(M[k, k]), p - 2, p) % p
        f = M[:, k].clone()
        f[k] = 0
        M = (M - torch.outer(f, M[k]) % p) % p
    return M[:, n:].cpu().numpy()


def test_lift_full_size_limb(smf):
    # the bench's lifting workload: 1024 x 1024 (20-bit) by 1024 x 64 (40-bit), 16 steps, limb form
    c = smf.Context(0, FORMS["limb"])
    try:
        pb = c.basis_create(10)
        p = int(pb.primes[0])
        n, m, k = 1024, 64, 16
        A = inputs.uniform_int(9, "LA", (n, n), -(1 << 20), 1 << 20)
        B = inputs.uniform_int(9, "LB", (n, m), -(1 << 40), 1 << 40)
        C = _inverse_mod_p_torch(A, p, "cuda")
        rows = np.random.default_rng(1).choice(n, 64, replace=False)  # a wrong C also fails the remainder check
        assert ((C[rows] @ (A % p)) % p == np.eye(n, dtype=np.int64)[rows]).all()
        want_X, want_R = lifting.lift_recurrence(A, B, p, k, C)
        X = torch.full((k, n, m), -1, dtype=torch.int32, device="cuda")
        R = torch.zeros((n, m, 1), dtype=torch.int64, device="cuda")
        c.padic_lift(pb, _words(A), torch.from_numpy(C.astype(np.int32)).cuda(), _words(B), k, X, R, a_bits=20,
                     b_bits=40)
        c.status_sync()
        got_X = X.cpu().numpy()
        for i in range(k):
            assert np.array_equal(got_X[i], want_X[i]), f"digit {i}"
        assert np.array_equal(R.cpu().numpy()[..., 0], want_R)
        pb.destroy()
    finally:
        c.destroy()
