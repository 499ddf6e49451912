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


def _system(seed, n, m, p):
    while True:
        A = inputs.uniform_int(seed, "LA", (n, n), -(1 << 20), 1 << 20)
        try:
            C = lifting.inverse_mod_p(A.tolist(), p)
            break
        except ValueError:
            seed += 1
    B = inputs.uniform_int(seed, "LB", (n, m), -(1 << 40), 1 << 40)
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
