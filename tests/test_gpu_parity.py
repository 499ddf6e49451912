"""GPU parity: every step of the CUDA path against the oracle, bit-exact.

All inputs are seeded synthetic matrices from paper_2605_19254_gb300.inputs;
expected values come only from the oracle.  Sizes span several tiles with
ragged tails; the last tests run the 4096 x 4096 by 4096 x 256 product at full
size and compare every output entry.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19254_gb300 import inputs  # noqa: E402

FORMS = {"fp64": 0, "limb": 1}


def dev(words: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda()


def host_words(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


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


# --------------------------------------------------------------------------- basis (a0)

def test_basis_matches_oracle(smf, orc):
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    for bits, pmax in [(543, 1 << 26), (543, 1 << 24), (100, 1 << 16), (0, 1 << 26), (3000, 1 << 26)]:
        b = c.basis_create(bits, pmax)
        assert b.primes == [int(p) for p in orc.basis(pmax, bits)]
        b.destroy()
    c.destroy()


# --------------------------------------------------------------------------- rns_reduce (a1, a2)

@pytest.mark.parametrize("shape,W", [((37, 300), 1), ((130, 70), 8), ((5, 9), 2), ((64, 33), 9), ((1, 1), 3)])
def test_rns_reduce(ctx, orc, shape, W):
    X = inputs.random_words(21, f"rr{W}", shape, W)
    X[0, 0] = inputs.extreme_words("min", (1,), W)[0]
    X[-1, -1] = inputs.extreme_words("max", (1,), W)[0]
    if shape[1] > 2:
        X[0, 1] = inputs.extreme_words("minus1", (1,), W)[0]
        X[0, 2] = 0
    b = ctx.basis_create(64 * W + 40)
    L = len(b.primes)
    out = torch.empty((L,) + shape, dtype=torch.int32, device="cuda")
    ctx.rns_reduce(b, dev(X), out)
    torch.cuda.synchronize()
    want = orc.reduce(X, b.primes)
    assert np.array_equal(out.cpu().numpy(), want)
    b.destroy()


# --------------------------------------------------------------------------- residue_gemm (a3, a4, a5)

def _residues(orc, primes, M, N, K, seed, shared_a_bits=None):
    A = inputs.random_words(seed, "gA", (M, K), 1)
    B = inputs.random_words(seed, "gB", (K, N), 8)
    Br = orc.reduce(B, primes)
    if shared_a_bits is not None:
        a = inputs.uniform_int(seed, "gAs", (M, K), -(1 << shared_a_bits), 1 << shared_a_bits).astype(np.int32)
        return a, Br
    return orc.reduce(A, primes), Br


@pytest.mark.parametrize("M,N,K", [(300, 70, 1500), (128, 32, 64), (129, 33, 65), (7, 5, 1), (200, 96, 2049)])
def test_residue_gemm(ctx, orc, M, N, K):
    b = ctx.basis_create(200)
    primes = b.primes
    Ar, Br = _residues(orc, primes, M, N, K, seed=M + N + K)
    want = orc.residue_gemm(Ar, Br, primes)
    ws_n = ctx.residue_gemm_workspace(b, M, N, K, False)
    ws = torch.empty(max(ws_n, 1), dtype=torch.uint8, device="cuda")
    C = torch.empty((len(primes), M, N), dtype=torch.int32, device="cuda")
    ctx.residue_gemm(b, torch.from_numpy(Ar).cuda(), M * K, torch.from_numpy(Br).cuda(), C, M, N, K, ws)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy(), want)
    b.destroy()


def test_residue_gemm_shared_a_and_centred_inputs(ctx, orc):
    M, N, K = 260, 40, 1100
    b = ctx.basis_create(300)
    primes = b.primes
    a, Br = _residues(orc, primes, M, N, K, seed=5, shared_a_bits=20)
    pr = np.array(primes, dtype=np.int64)[:, None, None]
    Bc = np.where(Br > (pr - 1) // 2, Br - pr, Br).astype(np.int32)  # centred representatives
    want = orc.residue_gemm(a, Br, primes)
    ws = torch.empty(max(ctx.residue_gemm_workspace(b, M, N, K, True), 1), dtype=torch.uint8, device="cuda")
    C = torch.empty((len(primes), M, N), dtype=torch.int32, device="cuda")
    ctx.residue_gemm(b, torch.from_numpy(a).cuda(), 0, torch.from_numpy(Bc).cuda(), C, M, N, K, ws)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy(), want)
    b.destroy()


@pytest.mark.parametrize("va,vb", [("h", "h"), ("-h", "h"), ("-h", "-h"), ("p-1", "1-p")])
def test_residue_gemm_extremes(ctx, orc, va, vb):
    # every residue at the edge of the exactness bounds, K across two fold blocks
    M, N, K = 130, 34, 2050
    b = ctx.basis_create(100)
    primes = b.primes
    L = len(primes)

    def fill(v, shape):
        out = np.empty((L,) + shape, dtype=np.int64)
        for i, p in enumerate(primes):
            out[i] = {"h": (p - 1) // 2, "-h": -((p - 1) // 2), "p-1": p - 1, "1-p": 1 - p}[v]
        return out.astype(np.int32)

    Ar, Br = fill(va, (M, K)), fill(vb, (K, N))
    want = orc.residue_gemm(Ar, Br, primes)
    ws = torch.empty(max(ctx.residue_gemm_workspace(b, M, N, K, False), 1), dtype=torch.uint8, device="cuda")
    C = torch.empty((L, M, N), dtype=torch.int32, device="cuda")
    ctx.residue_gemm(b, torch.from_numpy(Ar).cuda(), M * K, torch.from_numpy(Br).cuda(), C, M, N, K, ws)
    ctx.status_sync()
    assert np.array_equal(C.cpu().numpy(), want)
    b.destroy()


def test_limb_digit_extremes_fill_accumulator(smf, orc):
    # A = -128 and B = -(p-1)/2 (top digit -128): the products of the top digits
    # are +2^14 and each fold block of 1024 of them sums to exactly 2^24
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    b = c.basis_create(40, 1 << 16)
    primes = b.primes
    M, N, K = 128, 32, 4096
    L = len(primes)
    a = np.full((M, K), -128, dtype=np.int32)  # shared A
    Br = np.empty((L, K, N), dtype=np.int32)
    for i, p in enumerate(primes):
        Br[i] = -((p - 1) // 2)
    want = orc.residue_gemm(a, Br, primes)
    ws = torch.empty(c.residue_gemm_workspace(b, M, N, K, True), dtype=torch.uint8, device="cuda")
    C = torch.empty((L, M, N), dtype=torch.int32, device="cuda")
    c.residue_gemm(b, torch.from_numpy(a).cuda(), 0, torch.from_numpy(Br).cuda(), C, M, N, K, ws)
    c.status_sync()
    assert np.array_equal(C.cpu().numpy(), want)
    c.destroy()


@pytest.mark.parametrize("va,vb", [(-1015936, -8355968), (-1015936, 8355968), (1015936, -8355968)])
def test_limb_fold_block_from_digit_bounds(smf, orc, va, vb):
    # |A| <= 2^20 caps A's top digit at 16, so a fold block spans 7 K steps
    # (448 products) instead of 5.  A = -1015936 has digits (-128, -128, -15) and
    # B = -8355968, its own centred residue for every prime below 2^24, has
    # (-128, -128, -127): every product of a diagonal has the same sign and the
    # busiest diagonal reaches 448 * 34560 = 0.92 * 2^24 per block.
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    M, N, K = 130, 70, 3 * 448 + 13
    A = np.full((M, K), va, dtype=np.int64)
    B = np.full((K, N), vb, dtype=np.int64)
    Aw = inputs.int64_to_words(A, 1)
    Bw = inputs.int64_to_words(B, 1)
    want = orc.matmul(Aw, Bw, 2)
    C = torch.zeros((M, N, 2), dtype=torch.int64, device="cuda")
    c.rns_matmul(dev(Aw), dev(Bw), C, a_bits=20)
    c.status_sync()
    assert np.array_equal(host_words(C), want)
    c.destroy()


def test_residue_gemm_long_k_folds(smf, orc):
    # K beyond 64 fold blocks of 320 products: the drain reduces its running
    # sums modulo each column's prime mid-tile
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    b = c.basis_create(60)
    primes = b.primes
    L = len(primes)
    M, N, K = 130, 50, 20544 + 77
    rng = np.random.default_rng(17)
    a = rng.integers(-(1 << 20), (1 << 20) + 1, (M, K)).astype(np.int32)  # shared A
    Br = np.stack([rng.integers(0, p, (K, N)) for p in primes]).astype(np.int32)
    want = orc.residue_gemm(a, Br, primes)
    ws = torch.empty(c.residue_gemm_workspace(b, M, N, K, True), dtype=torch.uint8, device="cuda")
    C = torch.empty((L, M, N), dtype=torch.int32, device="cuda")
    c.residue_gemm(b, torch.from_numpy(a).cuda(), 0, torch.from_numpy(Br).cuda(), C, M, N, K, ws)
    c.status_sync()
    assert np.array_equal(C.cpu().numpy(), want)
    c.destroy()


# --------------------------------------------------------------------------- crt_reconstruct (a6)

def test_crt_roundtrip_and_random(ctx, orc):
    b = ctx.basis_create(543)
    primes = b.primes
    M_ = 1
    for p in primes:
        M_ *= p
    h = (M_ - 1) // 2
    vals = [0, 1, -1, h, -h, h - 1, -h + 1] + list(orc.words_to_ints(inputs.random_words(3, "c", (90,), 8)))
    X = orc.ints_to_words(np.array(vals, dtype=object).reshape(1, -1), 9)
    r = orc.reduce(X, primes)
    out = torch.zeros((1, len(vals), 9), dtype=torch.int64, device="cuda")
    ctx.crt_reconstruct(b, torch.from_numpy(r).cuda(), out)
    torch.cuda.synchronize()
    assert np.array_equal(host_words(out), X)
    # uniformly random residues (any value in [0, M)) against the oracle's CRT
    rng = np.random.default_rng(4)
    R = np.stack([rng.integers(0, p, (33, 17)) for p in primes]).astype(np.int32)
    out = torch.zeros((33, 17, 9), dtype=torch.int64, device="cuda")
    ctx.crt_reconstruct(b, torch.from_numpy(R).cuda(), out)
    torch.cuda.synchronize()
    assert np.array_equal(host_words(out), orc.crt(R, primes, 9))
    b.destroy()


@pytest.mark.parametrize("bits", [543, 100, 1200])
def test_crt_near_half_modulus(ctx, orc, bits):
    # values whose quotient estimate is ambiguous (|x| within M 2^-12 of M/2)
    # exercise the exact mixed-radix path next to ordinary values
    b = ctx.basis_create(bits)
    primes = b.primes
    M_ = 1
    for p in primes:
        M_ *= p
    h = (M_ - 1) // 2
    rng = np.random.default_rng(bits)
    span = M_ >> 11
    vals = []
    for _ in range(150):
        k = int(rng.integers(0, 1 << 62)) % span
        vals += [h - k, -h + k, k - span, (M_ >> 2) - k]
    W = (M_.bit_length() + 64) // 64 + 1
    X = orc.ints_to_words(np.array(vals, dtype=object).reshape(3, -1), W)
    r = orc.reduce(X, primes)
    out = torch.zeros(X.shape, dtype=torch.int64, device="cuda")
    ctx.crt_reconstruct(b, torch.from_numpy(r).cuda(), out)
    torch.cuda.synchronize()
    assert np.array_equal(host_words(out), X)
    b.destroy()


@pytest.mark.parametrize("bits", [300, 543, 700])
def test_crt_many_tiles_against_oracle(ctx, orc, bits):
    # 90000 entries (704 tiles of 128, the last one ragged): more tiles than the
    # persistent grid's blocks, so blocks take several; random residues (any value in
    # [0, M)) and values near +-M/2, whose quotient estimate is ambiguous, side by side
    b = ctx.basis_create(bits)
    primes = b.primes
    M_ = 1
    for p in primes:
        M_ *= p
    h = (M_ - 1) // 2
    W = (M_.bit_length() + 64) // 64 + 1
    rng = np.random.default_rng(bits + 7)
    R = np.stack([rng.integers(0, p, (300, 300)) for p in primes]).astype(np.int32)
    span = M_ >> 11
    near = []
    for _ in range(150):
        k = int(rng.integers(0, 1 << 62)) % span
        near += [h - k, -h + k]
    Xn = orc.ints_to_words(np.array(near, dtype=object).reshape(1, -1), W)
    Rn = orc.reduce(Xn, primes)
    R[:, 0, :] = Rn[:, 0, :]
    want = orc.crt(R, primes, W)
    out = torch.zeros((300, 300, W), dtype=torch.int64, device="cuda")
    ctx.crt_reconstruct(b, torch.from_numpy(R).cuda(), out)
    torch.cuda.synchronize()
    got = host_words(out)
    assert np.array_equal(got[0], Xn[0])
    assert np.array_equal(got, want)
    b.destroy()


def test_crt_rejects_short_output(ctx, smf):
    b = ctx.basis_create(543)
    out = torch.zeros((2, 2, 8), dtype=torch.int64, device="cuda")
    r = torch.zeros((len(b.primes), 2, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(smf.SmfError) as e:
        ctx.crt_reconstruct(b, r, out)
    assert e.value.code == smf.SMF_E_BOUND
    b.destroy()


# --------------------------------------------------------------------------- rns_matmul end to end

@pytest.mark.parametrize("M,K,N,a_bits,Wb", [(150, 300, 40, 20, 8), (129, 1100, 33, 20, 8), (64, 64, 64, 40, 2),
                                             (3, 5, 2, 63, 1), (200, 2100, 20, 30, 4)])
def test_rns_matmul(ctx, orc, M, K, N, a_bits, Wb):
    if a_bits >= 63:
        A = inputs.random_words(8, "eA", (M, K), 1)
        bits = 0
    else:
        A = inputs.rns_matmul_workload(8, M, K, N, a_bits, 1)[0]
        bits = a_bits
    B = inputs.random_words(8, "eB", (K, N), Wb)
    a_eff = bits if bits else 63
    Wc = (a_eff + 64 * Wb - 1 + int(np.ceil(np.log2(max(K, 2)))) + 2 + 63) // 64
    want = orc.matmul(A, B, Wc)
    C = torch.zeros((M, N, Wc), dtype=torch.int64, device="cuda")
    ctx.rns_matmul(dev(A), dev(B), C, a_bits=bits)
    ctx.status_sync()
    assert np.array_equal(host_words(C), want)


def test_rns_matmul_host_buffers(ctx, orc):
    M, K, N = 100, 700, 30
    A, B = inputs.rns_matmul_workload(2, M, K, N, 20, 8)
    want = orc.matmul(A, B, 9)
    At = torch.from_numpy(A.view(np.int64)).pin_memory()
    Bt = torch.from_numpy(B.view(np.int64)).pin_memory()
    C = torch.zeros((M, N, 9), dtype=torch.int64).pin_memory()
    ctx.rns_matmul(At, Bt, C, a_bits=20)
    ctx.status_sync()
    assert np.array_equal(C.numpy().view(np.uint64), want)


@pytest.mark.parametrize("where", ["host,host,host", "host,dev,dev", "dev,host,host", "dev,dev,host"])
def test_rns_matmul_chunked_host_pipeline(ctx, orc, where):
    # M > 1024 with A or C in host memory: the product runs as four row chunks
    # (128, 640, 404, 128 rows) whose copies overlap the other chunks' kernels
    M, K, N = 1300, 300, 40
    A, B = inputs.rns_matmul_workload(3, M, K, N, 20, 8)
    want = orc.matmul(A, B, 9)
    wa, wb, wc = where.split(",")

    def place(x, w):
        t = torch.from_numpy(np.ascontiguousarray(x).view(np.int64))
        return t.pin_memory() if w == "host" else t.cuda()

    At, Bt = place(A, wa), place(B, wb)
    C = place(np.zeros((M, N, 9), dtype=np.uint64), wc)
    for _ in range(2):  # a second call reuses the staging slots and events
        C.zero_()
        ctx.rns_matmul(At, Bt, C, a_bits=20)
        ctx.status_sync()
        assert np.array_equal(C.cpu().numpy().view(np.uint64), want)


@pytest.mark.parametrize("a_bits,M", [(7, 9856), (12, 9856), (7, 9893)])
def test_narrow_digit_product_wide_tiles(ctx, orc, a_bits, M):
    # a one- or two-digit shared A over two primes and 32 columns: 64-column
    # tiles fill one wave where 48-column ones need two, so the narrow-digit
    # kernel runs with BN = 64 (MMA N = 192); a ragged last row tile at M = 9893
    K, N = 256, 32
    A = inputs.rns_matmul_workload(90 + a_bits + M, M, K, N, a_bits, 1)[0]
    B = inputs.uniform_int(91 + M, "nB", (K, N), -(1 << 20), 1 << 20)
    B = inputs.int64_to_words(B, 1)
    Wc = 1
    want = orc.matmul(A, B, Wc)
    C = torch.full((M, N, Wc), 7, dtype=torch.int64, device="cuda")
    ctx.rns_matmul(dev(A), dev(B), C, a_bits=a_bits, b_bits=20)
    ctx.status_sync()
    diff = (host_words(C) != want).any(axis=-1)
    assert not diff.any(), f"{int(diff.sum())} entries differ, the first at {np.argwhere(diff)[:4].tolist()}"


GROUP_SHAPES = [(32, 32, 7), (100, 100, 20), (129, 129, 7), (300, 257, 20), (33, 64, 7), (64, 500, 20),
                (1, 5, 1), (0, 10, 3), (40, 0, 5)]


@pytest.mark.parametrize("a_bits", [20, 0, 6])
def test_rns_matmul_grouped(ctx, orc, a_bits):
    # products of uneven shapes in one call: in the limb form one launch runs the
    # residue products of all of them; 20-bit A shares its digits across primes,
    # full 64-bit A is reduced per prime, and 6-bit A (one digit, outside the
    # 3x3-digit kernel) runs the products one at a time
    As, Bs, Cs, wants = [], [], [], []
    for i, (M, K, N) in enumerate(GROUP_SHAPES):
        if a_bits:
            A = inputs.rns_matmul_workload(30 + i, M, K, N, a_bits, 1)[0]
        else:
            A = inputs.random_words(30 + i, "gA", (M, K), 1)
        B = inputs.random_words(30 + i, "gB", (K, N), 8)
        Wc = (((a_bits or 63) + 511 + 10) + 2 + 63) // 64
        wants.append(orc.matmul(A, B, Wc))
        As.append(dev(A))
        Bs.append(dev(B))
        Cs.append(torch.zeros((M, N, Wc), dtype=torch.int64, device="cuda"))
    for _ in range(2):  # the second call reuses the descriptor staging
        for C in Cs:
            C.fill_(7)  # every output, empty-K products included, is written
        ctx.rns_matmul_grouped(As, Bs, Cs, a_bits=a_bits)
        ctx.status_sync()
        for C, want in zip(Cs, wants):
            assert np.array_equal(host_words(C), want)


def test_rns_matmul_grouped_mixed_widths(ctx, orc):
    # per-item entry bounds (7, 20 and 40-bit A) and B of 1, 2, 3 and 8 words:
    # the transposed reduce runs one grouped launch per word count it takes
    # (1, 2, 4, 8) and the 3-word operand on its own
    shapes = [(70, 90, 9, 7, 1), (33, 200, 17, 20, 2), (128, 64, 64, 40, 3), (257, 129, 5, 7, 8),
              (16, 16, 16, 20, 8), (90, 300, 33, 40, 1)]
    As, Bs, Cs, wants, bits = [], [], [], [], []
    for i, (M, K, N, ab, Wb) in enumerate(shapes):
        A = inputs.rns_matmul_workload(60 + i, M, K, N, ab, 1)[0]
        B = inputs.random_words(60 + i, "mB", (K, N), Wb)
        Wc = (ab + 64 * Wb - 1 + int(np.ceil(np.log2(K))) + 2 + 63) // 64
        wants.append(orc.matmul(A, B, Wc))
        As.append(dev(A))
        Bs.append(dev(B))
        Cs.append(torch.full((M, N, Wc), 7, dtype=torch.int64, device="cuda"))
        bits.append(ab)
    ctx.rns_matmul_grouped(As, Bs, Cs, a_bits=bits)
    ctx.status_sync()
    for C, want in zip(Cs, wants):
        assert np.array_equal(host_words(C), want)


def test_rns_matmul_grouped_empty_and_host_operands(ctx, smf):
    ctx.rns_matmul_grouped([], [], [])
    assert ctx.rns_matmul_grouped_workspace([], [], []) == 0
    A = torch.zeros((4, 4, 1), dtype=torch.int64)
    B = torch.zeros((4, 4, 1), dtype=torch.int64, device="cuda")
    C = torch.zeros((4, 4, 3), dtype=torch.int64, device="cuda")
    with pytest.raises(smf.SmfError) as e:
        ctx.rns_matmul_grouped([A], [B], [C])
    assert e.value.code == smf.SMF_E_INVALID


def test_rns_matmul_errors(ctx, smf):
    A = torch.zeros((4, 5, 1), dtype=torch.int64, device="cuda")
    B = torch.zeros((6, 3, 8), dtype=torch.int64, device="cuda")
    C = torch.zeros((4, 3, 9), dtype=torch.int64, device="cuda")
    with pytest.raises(smf.SmfError) as e:
        ctx.rns_matmul(A, B, C)
    assert e.value.code == smf.SMF_E_INVALID
    B = torch.zeros((5, 3, 8), dtype=torch.int64, device="cuda")
    C = torch.zeros((4, 3, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(smf.SmfError) as e:
        ctx.rns_matmul(A, B, C)
    assert e.value.code == smf.SMF_E_BOUND


def test_rns_matmul_empty(ctx):
    A = torch.zeros((0, 5, 1), dtype=torch.int64, device="cuda")
    B = torch.zeros((5, 3, 8), dtype=torch.int64, device="cuda")
    C = torch.zeros((0, 3, 9), dtype=torch.int64, device="cuda")
    ctx.rns_matmul(A, B, C, a_bits=20)
    A = torch.zeros((4, 0, 1), dtype=torch.int64, device="cuda")
    B = torch.zeros((0, 3, 8), dtype=torch.int64, device="cuda")
    C = torch.full((4, 3, 9), 7, dtype=torch.int64, device="cuda")
    ctx.rns_matmul(A, B, C, a_bits=20)
    ctx.status_sync()
    assert int(C.abs().sum()) == 0


# --------------------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def full_size():
    M = K = 4096
    N = 256
    A, B = inputs.rns_matmul_workload(0, M, K, N, 20, 8)
    return A, B


@pytest.fixture(scope="module")
def full_size_want(orc, full_size):
    A, B = full_size
    return orc.matmul(A, B, 9)  # every entry, schoolbook over Z (about 16 s on 16 cores)


@pytest.mark.parametrize("form", list(FORMS) + ["limb_fused_crt"])
def test_full_size_every_entry(smf, full_size, full_size_want, form):
    # the bench's launch configuration: every one of the 4096 x 256 entries,
    # so every tile of the raster order and every tile spanning two primes;
    # limb_fused_crt: the residue product with the CRT in its epilogue
    A, B = full_size
    c = smf.Context(0, FORMS[form.split("_")[0]])
    if form == "limb_fused_crt":
        c.set_fused_crt(True)
    C = torch.zeros((4096, 256, 9), dtype=torch.int64, device="cuda")
    c.rns_matmul(dev(A), dev(B), C, a_bits=20)
    c.status_sync()
    diff = (host_words(C) != full_size_want).any(axis=-1)
    assert not diff.any(), f"{int(diff.sum())} entries differ, the first at {np.argwhere(diff)[:4].tolist()}"
    c.destroy()


def test_batched_full_size_sampled(smf, orc):
    # the 512-product batch (n log-uniform in [32, 1024], k = 7 / 20, B n x 128
    # of 512 bits) in one grouped call, as the bench times it; sampled entries of
    # the smallest, the largest and a spread of other products against the oracle
    batch = inputs.batched_workload(0, 512, 128, 8)
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    As, Bs, Cs, bits, Wcs = [], [], [], [], []
    for n, k, A, B in batch:
        Wc = (k + 511 + int(np.ceil(np.log2(n))) + 2 + 63) // 64
        As.append(dev(A))
        Bs.append(dev(B))
        Cs.append(torch.full((n, 128, Wc), 7, dtype=torch.int64, device="cuda"))
        bits.append(k)
        Wcs.append(Wc)
    c.rns_matmul_grouped(As, Bs, Cs, a_bits=bits)
    c.status_sync()
    ns = [b[0] for b in batch]
    rng = np.random.default_rng(1)
    picks = sorted({int(np.argmin(ns)), int(np.argmax(ns)), 0, 1, 511, *rng.choice(512, 6, replace=False).tolist()})
    for i in picks:
        n, k, A, B = batch[i]
        rows = np.unique(np.append(rng.choice(n, min(n, 4), replace=False), n - 1))
        cols = np.unique(np.append(rng.choice(128, 4, replace=False), 127))
        want = orc.matmul(A[rows], B[:, cols], Wcs[i])
        got = host_words(Cs[i])[rows][:, cols]
        assert np.array_equal(got, want), f"product {i} (n={n}, k={k})"
    c.destroy()


# --------------------------------------------------------------------------- failure detection

def test_bounded_wait_timeout_is_reported_and_context_recovers(smf, orc):
    # the copy-issuing warp stays idle: every wait on data gives up after about
    # two seconds, the kernel unwinds and the status reports the timeout
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    M, K, N = 256, 512, 96
    A, B = inputs.rns_matmul_workload(13, M, K, N, 20, 8)
    Ad, Bd = dev(A), dev(B)
    C = torch.zeros((M, N, 9), dtype=torch.int64, device="cuda")
    c.debug_inject(smf.SMF_INJECT_STALL_LOADS)
    c.rns_matmul(Ad, Bd, C, a_bits=20)
    with pytest.raises(smf.SmfError) as e:
        c.status_sync()
    assert e.value.code == smf.SMF_E_TIMEOUT
    # the flag cleared after one launch and the context still computes exactly
    c.rns_matmul(Ad, Bd, C, a_bits=20)
    c.status_sync()
    assert np.array_equal(host_words(C), orc.matmul(A, B, 9))
    c.destroy()
