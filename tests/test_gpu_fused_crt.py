"""GPU parity of the residue product with the CRT fused into its epilogue
(smf_set_fused_crt): every output entry against the oracle's schoolbook
product, on shapes with ragged row tiles, several column blocks per prime,
shared and per-prime A, and repeated calls (the per-unit counters restart).
The full-size case is in test_gpu_parity.py (test_full_size_every_entry).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19254_gb300 import inputs  # noqa: E402


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


# (M, K, N, bits of A, words of B): 20-bit A is shared across primes (N a
# multiple of 64 for the fused path), 0 = full 64-bit A reduced per prime (any
# N); one row tile, ragged row tiles, one to four column blocks per prime, a
# ragged column block.  Every shape has enough tiles to run without a K split
# (a product that splits K keeps the two kernels).
SHAPES = [(128, 64, 64, 20, 8), (300, 257, 128, 20, 8), (1000, 700, 192, 20, 4), (129, 1000, 256, 20, 8),
          (300, 90, 100, 0, 4), (1280, 200, 64, 0, 2)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_crt_matches_oracle(smf, orc, shape):
    M, K, N, ab, Wb = shape
    if ab:
        A = inputs.rns_matmul_workload(70 + M, M, K, N, ab, 1)[0]
    else:
        A = inputs.random_words(70 + M, "fA", (M, K), 1)
    B = inputs.random_words(70 + M, "fB", (K, N), Wb)
    Wc = ((ab or 63) + 64 * Wb - 1 + int(np.ceil(np.log2(K))) + 2 + 63) // 64
    want = orc.matmul(A, B, Wc)
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    c.set_fused_crt(True)
    Ad, Bd = dev(A), dev(B)
    C = torch.full((M, N, Wc), 7, dtype=torch.int64, device="cuda")
    c.profile_enable(True)
    for _ in range(2):  # the second call finds the counters of the first at L and restarts them
        C.fill_(7)
        c.rns_matmul(Ad, Bd, C, a_bits=ab)
        c.status_sync()
        prof = c.profile_read()
        assert prof["residue_gemm"][0] == 1 and prof["crt"][0] == 0  # one fused kernel, no CRT launch
        diff = (host_words(C) != want).any(axis=-1)
        assert not diff.any(), f"{int(diff.sum())} entries differ, the first at {np.argwhere(diff)[:4].tolist()}"
    c.destroy()


def test_fused_crt_timeout_ends_every_warp_and_context_recovers(smf, orc):
    # the copy-issuing warp stays idle: every wait on data gives up after about
    # two seconds; the drain warps agree on the failure at their shared barrier,
    # skip the counting and the reconstruction, and the kernel unwinds
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    c.set_fused_crt(True)
    M, K, N = 256, 512, 128
    A, B = inputs.rns_matmul_workload(14, M, K, N, 20, 8)
    Ad, Bd = dev(A), dev(B)
    C = torch.zeros((M, N, 9), dtype=torch.int64, device="cuda")
    c.debug_inject(smf.SMF_INJECT_STALL_LOADS)
    c.rns_matmul(Ad, Bd, C, a_bits=20)
    with pytest.raises(smf.SmfError) as e:
        c.status_sync()
    assert e.value.code == smf.SMF_E_TIMEOUT
    c.rns_matmul(Ad, Bd, C, a_bits=20)
    c.status_sync()
    assert np.array_equal(host_words(C), orc.matmul(A, B, 9))
    c.destroy()
