"""GPU parity of the conversion between RNS bases (Section 3.1) against the
oracle's base_convert, bit-exact.  Random canonical residues represent, by
the CRT bijection, uniformly random integers over the whole symmetric range;
the endpoints +-(M-1)/2 (where the fp32 estimate of alpha is too close to
call and the exact settlement runs) are appended from Python integers."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _prod(ps):
    m = 1
    for p in ps:
        m *= int(p)
    return m


def _residues(seed, primes, count):
    """[L, count] canonical residues: uniform per prime, then special values."""
    P = [int(p) for p in primes]
    M = _prod(P)
    H = (M - 1) // 2
    special = [H, -H, H - 1, -H + 1, 0, 1, -1, M // P[0], -(M // P[0]), H // 2, -(H // 2)]
    r = np.stack([inputs.uniform_int(seed, f"r{i}", (count,), 0, p - 1) for i, p in enumerate(P)]).astype(np.int32)
    extra = np.array([[x % p for x in special] for p in P], dtype=np.int32)
    return np.ascontiguousarray(np.concatenate([r, extra], axis=1))


def _convert(ctx, src, dst, r_in):
    rin = torch.from_numpy(r_in).cuda()
    rout = torch.full((len(dst.primes), r_in.shape[1]), -1, dtype=torch.int32, device="cuda")
    ctx.base_convert(src, dst, rin, rout)
    ctx.status_sync()
    return rout.cpu().numpy()


@pytest.mark.parametrize("src_bits,src_pmax,dst_bits,count", [
    (543, 0, 543, 3000),             # 23 -> 23 primes below 2^24, disjoint
    (100, 1 << 20, 543, 700),        # 6 small primes -> 23
    (543, 0, 60, 1000),              # 23 -> 3 primes below the source's
    (1200, 1 << 26, 1230, 513),      # 47 -> 48 primes below 2^26 (the largest kernel)
])
def test_base_convert_matches_oracle(ctx, orc, src_bits, src_pmax, dst_bits, count):
    src = ctx.basis_create(src_bits, src_pmax)
    dst = ctx.basis_create(dst_bits, min(src.primes))  # primes below the source's: disjoint
    try:
        r_in = _residues(src_bits + count, src.primes, count)
        got = _convert(ctx, src, dst, r_in)
        want = orc.base_convert(r_in, src.primes, dst.primes)
        assert np.array_equal(got, want)
    finally:
        src.destroy()
        dst.destroy()


def test_base_convert_identity_and_shared_primes(ctx, orc):
    src = ctx.basis_create(543)
    try:
        r_in = _residues(3, src.primes, 1000)
        assert np.array_equal(_convert(ctx, src, src, r_in), r_in)
    finally:
        src.destroy()


def test_base_convert_errors(ctx, smf):
    src = ctx.basis_create(543)
    big = ctx.basis_create(1300, 1 << 26)  # 50 primes: beyond the kernel's 48
    try:
        rin = torch.zeros((len(src.primes), 10), dtype=torch.int32)  # host memory
        rout = torch.zeros((len(src.primes), 10), dtype=torch.int32, device="cuda")
        with pytest.raises(smf.SmfError) as e:
            ctx.base_convert(src, src, rin, rout)
        assert e.value.code == smf.SMF_E_INVALID
        assert len(big.primes) > 48
        rb = torch.zeros((len(big.primes), 10), dtype=torch.int32, device="cuda")
        with pytest.raises(smf.SmfError) as e:
            ctx.base_convert(big, src, rb, rout)
        assert e.value.code == smf.SMF_E_UNSUPPORTED
        empty = torch.zeros((len(src.primes), 0), dtype=torch.int32, device="cuda")
        ctx.base_convert(src, src, empty, empty.clone())
    finally:
        src.destroy()
        big.destroy()


def test_base_convert_full_size_sampled(ctx, orc):
    # the 4096 x 256 residue matrix of the product workload, 23 -> 23 primes,
    # in the launch the bench times; sampled columns against the oracle
    src = ctx.basis_create(543)
    dst = ctx.basis_create(543, min(src.primes))
    try:
        n = 4096 * 256
        r_in = _residues(11, src.primes, n)
        got = _convert(ctx, src, dst, r_in)
        rng = np.random.default_rng(2)
        cols = np.unique(np.concatenate([rng.choice(n, 3000, replace=False), np.arange(n, r_in.shape[1])]))
        want = orc.base_convert(np.ascontiguousarray(r_in[:, cols]), src.primes, dst.primes)
        assert np.array_equal(got[:, cols], want)
    finally:
        src.destroy()
        dst.destroy()
