"""GPU parity on edge shapes and sizes, bit-exact against the oracle: single
entries, K = 1, 1024-bit B (a 44-prime basis: the widest CRT fast path),
grouped calls of one product, and conversions of one entry or from a
one-prime basis."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def _wc(a_bits, Wb, K):
    return ((a_bits or 63) + 64 * Wb - 1 + int(np.ceil(np.log2(max(K, 2)))) + 2 + 63) // 64


@pytest.mark.parametrize("M,K,N,a_bits,Wb", [(1, 1, 1, 20, 1), (1, 1, 1, 0, 8), (300, 1, 70, 20, 8),
                                             (1, 700, 1, 20, 8), (70, 90, 40, 20, 16), (33, 1, 5, 0, 16)])
def test_rns_matmul_edges(ctx, orc, M, K, N, a_bits, Wb):
    if a_bits:
        A = inputs.rns_matmul_workload(40 + M, M, K, N, a_bits, 1)[0]
    else:
        A = inputs.random_words(40 + M, "eA", (M, K), 1)
    B = inputs.random_words(40 + K, "eB", (K, N), Wb)
    Wc = _wc(a_bits, Wb, K)
    C = torch.full((M, N, Wc), 7, dtype=torch.int64, device="cuda")
    ctx.rns_matmul(_dev(A), _dev(B), C, a_bits=a_bits)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, Wc))


def test_rns_matmul_extreme_wide_entries(ctx, orc):
    # -2^1023 and 2^1023 - 1 entries in B, +-2^20 in A: the largest magnitudes of a 16-word product
    M, K, N = 20, 40, 12
    A = inputs.int64_to_words(np.where(np.arange(M * K).reshape(M, K) % 2 == 0, 1 << 20, -(1 << 20)), 1)
    B = inputs.extreme_words("min", (K, N), 16)
    B[:, ::2] = inputs.extreme_words("max", (K, (N + 1) // 2), 16)
    Wc = _wc(20, 16, K)
    C = torch.zeros((M, N, Wc), dtype=torch.int64, device="cuda")
    ctx.rns_matmul(_dev(A), _dev(B), C, a_bits=20)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, Wc))


def test_grouped_single_and_mostly_empty(ctx, orc):
    A, B = inputs.rns_matmul_workload(77, 50, 60, 9, 20, 8)
    Wc = _wc(20, 8, 60)
    C = torch.zeros((50, 9, Wc), dtype=torch.int64, device="cuda")
    ctx.rns_matmul_grouped([_dev(A)], [_dev(B)], [C], a_bits=20)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, Wc))
    # one 1 x 1 x 1 product among empty ones
    A1, B1 = inputs.rns_matmul_workload(78, 1, 1, 1, 20, 8)
    W1 = _wc(20, 8, 1)
    As = [torch.zeros((0, 4, 1), dtype=torch.int64, device="cuda"), _dev(A1),
          torch.zeros((3, 0, 1), dtype=torch.int64, device="cuda")]
    Bs = [torch.zeros((4, 2, 8), dtype=torch.int64, device="cuda"), _dev(B1),
          torch.zeros((0, 5, 8), dtype=torch.int64, device="cuda")]
    Cs = [torch.zeros((0, 2, W1), dtype=torch.int64, device="cuda"), torch.full((1, 1, W1), 7, dtype=torch.int64,
                                                                                 device="cuda"),
          torch.full((3, 5, W1), 7, dtype=torch.int64, device="cuda")]
    ctx.rns_matmul_grouped(As, Bs, Cs, a_bits=20)
    ctx.status_sync()
    assert np.array_equal(Cs[1].cpu().numpy().view(np.uint64), orc.matmul(A1, B1, W1))
    assert int(Cs[2].abs().sum()) == 0  # K = 0: the zero product


def test_base_convert_single_entry_and_one_prime_basis(smf, orc):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    try:
        src = c.basis_create(543)
        dst = c.basis_create(543, min(src.primes))
        one = c.basis_create(10)  # a single prime: every residue is its own symmetric value
        assert len(one.primes) == 1
        r = np.array([[int(p) - 1] for p in src.primes], dtype=np.int32)  # x = -1
        out = torch.empty((len(dst.primes), 1), dtype=torch.int32, device="cuda")
        c.base_convert(src, dst, torch.from_numpy(r).cuda(), out)
        c.status_sync()
        assert np.array_equal(out.cpu().numpy(), orc.base_convert(r, src.primes, dst.primes))
        assert all(int(v) == int(q) - 1 for v, q in zip(out.cpu().numpy()[:, 0], dst.primes))
        p0 = int(one.primes[0])
        h = p0 // 2
        edge = [0, 1, 2, h - 1, h, h + 1, p0 - 2, p0 - 1]
        r1 = np.concatenate([edge, inputs.uniform_int(3, "one", (3000,), 0, p0 - 1)]).astype(np.int32)[None, :]
        out1 = torch.empty((len(dst.primes), r1.shape[1]), dtype=torch.int32, device="cuda")
        c.base_convert(one, dst, torch.from_numpy(r1).cuda(), out1)
        c.status_sync()
        assert np.array_equal(out1.cpu().numpy(), orc.base_convert(r1, one.primes, dst.primes))
        for b in (src, dst, one):
            b.destroy()
    finally:
        c.destroy()


@pytest.mark.parametrize("M,K,N", [(1024, 4096, 16), (300, 1100, 5), (128, 200, 64)])
def test_skinny_residue_gemm_split_k(smf, orc, M, K, N):
    # few output tiles: the K range is split across CTAs and the partial
    # residues summed mod p (limb form, non-shared A)
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    try:
        b = c.basis_create(60)  # three primes below 2^24
        primes = np.array(b.primes, dtype=np.uint32)
        L = len(primes)
        Ar = np.stack([inputs.uniform_int(5 + i, "sa", (M, K), 0, int(p) - 1) for i, p in enumerate(primes)])
        Br = np.stack([inputs.uniform_int(6 + i, "sb", (K, N), 0, int(p) - 1) for i, p in enumerate(primes)])
        want = orc.residue_gemm(Ar, Br, primes)
        A = torch.from_numpy(Ar.astype(np.int32)).cuda()
        B = torch.from_numpy(Br.astype(np.int32)).cuda()
        C = torch.full((L, M, N), -1, dtype=torch.int32, device="cuda")
        ws = torch.empty(c.residue_gemm_workspace(b, M, N, K, False), dtype=torch.uint8, device="cuda")
        c.residue_gemm(b, A, M * K, B, C, M, N, K, workspace=ws)
        c.status_sync()
        assert np.array_equal(C.cpu().numpy(), want)
        b.destroy()
    finally:
        c.destroy()


def test_split_k_below_one_wave(smf, orc):
    # 79 row tiles of one prime (between half a wave and a wave of SMs): the K
    # range splits three ways, 237 units in two waves (the lifting's C R_i at
    # n near 10^4 has this shape)
    M, K, N = 10007, 1000, 32
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    try:
        b = c.basis_create(20)  # one prime below 2^24
        primes = np.array(b.primes, dtype=np.uint32)
        assert len(primes) == 1
        Ar = inputs.uniform_int(15, "wa", (1, M, K), 0, int(primes[0]) - 1)
        Br = inputs.uniform_int(16, "wb", (1, K, N), 0, int(primes[0]) - 1)
        want = orc.residue_gemm(Ar, Br, primes)
        C = torch.full((1, M, N), -1, dtype=torch.int32, device="cuda")
        ws = torch.empty(c.residue_gemm_workspace(b, M, N, K, False), dtype=torch.uint8, device="cuda")
        c.residue_gemm(b, torch.from_numpy(Ar.astype(np.int32)).cuda(), M * K,
                       torch.from_numpy(Br.astype(np.int32)).cuda(), C, M, N, K, workspace=ws)
        c.status_sync()
        assert np.array_equal(C.cpu().numpy(), want)
        b.destroy()
    finally:
        c.destroy()


@pytest.mark.parametrize("M,K,N", [(512, 4096, 8), (129, 3000, 3)])
def test_skinny_rns_matmul_split_k(smf, orc, M, K, N):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    try:
        A, B = inputs.rns_matmul_workload(90 + N, M, K, N, 20, 8)
        Wc = _wc(20, 8, K)
        C = torch.zeros((M, N, Wc), dtype=torch.int64, device="cuda")
        c.rns_matmul(_dev(A), _dev(B), C, a_bits=20)
        c.status_sync()
        got = C.cpu().numpy().view(np.uint64)
        rows = np.unique(np.append(np.random.default_rng(0).choice(M, 40, replace=False), M - 1))
        assert np.array_equal(got[rows], orc.matmul(A[rows], B, Wc))
    finally:
        c.destroy()


# --------------------------------------------------------------------------- declared entry bounds

def _bound_case(seed, M, K, N):
    A, B = inputs.rns_matmul_workload(seed, M, K, N, 20, 8)
    A[0, 0, 0] = np.uint64(1 << 20)  # both ends of [-2^20, 2^20] are inside the bound
    A[1, 1, 0] = np.int64(-(1 << 20)).view(np.uint64)
    return A, B


@pytest.mark.parametrize("K", [304, 300])  # the 8-entry digit split, and the generic reduce (K % 8 != 0)
def test_entry_beyond_declared_bound_is_reported(ctx, smf, orc, K):
    M, N = 200, 40
    A, B = _bound_case(31, M, K, N)
    C = torch.zeros((M, N, 9), dtype=torch.int64, device="cuda")
    ctx.rns_matmul(_dev(A), _dev(B), C, a_bits=20)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, 9))
    for bad in (1 << 20) + 1, -(1 << 20) - 1, 1 << 40:
        A2 = A.copy()
        A2[57, K - 3, 0] = np.int64(bad).view(np.uint64)
        ctx.rns_matmul(_dev(A2), _dev(B), C, a_bits=20)
        with pytest.raises(smf.SmfError) as e:
            ctx.status_sync()
        assert e.value.code == smf.SMF_E_BOUND, bad
    # B declared 30 bits, one entry of 31 bits; the other words are sign extension
    Bs = inputs.int64_to_words(inputs.uniform_int(32, "bB", (K, N), -(1 << 30), 1 << 30), 8)
    C2 = torch.zeros((M, N, 2), dtype=torch.int64, device="cuda")
    ctx.rns_matmul(_dev(A), _dev(Bs), C2, a_bits=20, b_bits=30)
    ctx.status_sync()
    assert np.array_equal(C2.cpu().numpy().view(np.uint64), orc.matmul(A, Bs, 2))
    for bad in (1 << 30) + 1, -(1 << 31), 1 << 100:
        B2 = Bs.copy()
        B2[K - 1, N - 1] = inputs.int64_to_words(np.array([0]), 8)[0]
        if bad == 1 << 100:
            B2[K - 1, N - 1, 1] = np.uint64(1 << 36)
        else:
            B2[K - 1, N - 1] = inputs.int64_to_words(np.array([bad]), 8)[0]
        ctx.rns_matmul(_dev(A), _dev(B2), C2, a_bits=20, b_bits=30)
        with pytest.raises(smf.SmfError) as e:
            ctx.status_sync()
        assert e.value.code == smf.SMF_E_BOUND, bad
    # the context computes exactly afterwards
    ctx.rns_matmul(_dev(A), _dev(B), C, a_bits=20)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, 9))


def test_entry_beyond_declared_bound_in_a_grouped_call(smf, orc):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    shapes = [(40, 7), (130, 20), (70, 20)]
    items = [inputs.rns_matmul_workload(40 + i, n, n, 16, k, 8) for i, (n, k) in enumerate(shapes)]
    Cs = [torch.zeros((n, 16, 9), dtype=torch.int64, device="cuda") for n, _ in shapes]
    As = [_dev(A) for A, _ in items]
    Bs = [_dev(B) for _, B in items]
    c.rns_matmul_grouped(As, Bs, Cs, a_bits=[k for _, k in shapes])
    c.status_sync()
    for (A, B), C in zip(items, Cs):
        assert np.array_equal(C.cpu().numpy().view(np.uint64), orc.matmul(A, B, 9))
    A1 = items[1][0].copy()
    A1[129, 0, 0] = np.uint64((1 << 20) + 1)  # the last entry of the second item's split units
    c.rns_matmul_grouped([As[0], _dev(A1), As[2]], Bs, Cs, a_bits=[k for _, k in shapes])
    with pytest.raises(smf.SmfError) as e:
        c.status_sync()
    assert e.value.code == smf.SMF_E_BOUND
    c.destroy()
