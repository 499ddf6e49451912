"""The allocation-free residue product, called through the C ABI.

smf_residue_gemm_noalloc serves callers that cannot call cudaMalloc (another
component owns the device allocator, or an allocation's implicit device
synchronisation is not allowed where they run): it keeps its scratch in a
fixed device array built into the library instead of a caller workspace.
These checks compare it with smf_residue_gemm, which takes a workspace, and
with the oracle's residue product, on two calls in a row (the second call sees
the first call's leftovers in the shared array; one call has per-prime
residues of A, the other one A shared by all primes), and check that an
oversized product is refused.  The file is named so that pytest collects it
last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def smf():
    from paper_2605_19254_gb300 import build, smf as _smf
    build.build()
    assert torch.cuda.is_available()
    return _smf


def _operands(seed, L, M, N, K, primes, shared):
    rng = np.random.default_rng(seed)
    if shared:
        A = rng.integers(-(1 << 20), (1 << 20) + 1, (M, K)).astype(np.int32)
    else:
        A = np.stack([rng.integers(0, p, (M, K)) for p in primes]).astype(np.int32)
    B = np.stack([rng.integers(-(p - 1), p, (K, N)) for p in primes]).astype(np.int32)
    return torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_noalloc_matches_workspace_entry_point_twice(smf, orc, form):
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB if form == "limb" else smf.SMF_FORM_FP64)
    basis = ctx.basis_create(120)
    primes = basis.primes
    L = len(primes)
    cases = [(300, 70, 1500, False, 1), (257, 45, 2100, True, 2)]  # two calls in a row, different shapes
    for M, N, K, shared, seed in cases:
        A, B = _operands(seed, L, M, N, K, primes, shared)
        stride = 0 if shared else M * K
        ws = torch.empty(max(ctx.residue_gemm_workspace(basis, M, N, K, shared), 1), dtype=torch.uint8,
                         device="cuda")
        want = torch.empty((L, M, N), dtype=torch.int32, device="cuda")
        ctx.residue_gemm(basis, A, stride, B, want, M, N, K, ws)
        got = torch.full((L, M, N), -1, dtype=torch.int32, device="cuda")
        ctx.residue_gemm_noalloc(basis, A, stride, B, got, M, N, K)
        ctx.status_sync()
        assert torch.equal(got, want)  # exact: the residues are integers
        # and the product itself, from the oracle (canonical residues)
        ref = orc.residue_gemm(A.cpu().numpy(), B.cpu().numpy(), primes)
        assert np.array_equal(got.cpu().numpy(), ref)
    basis.destroy()
    ctx.destroy()


def test_noalloc_rejects_oversized_product(smf):
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    basis = ctx.basis_create(543)
    L = len(basis.primes)
    M, N, K = 4096, 256, 4096  # B digit planes alone: 3 * L * 256 * 4096 * 2 bytes > 64 MiB
    A = torch.zeros((M, K), dtype=torch.int32, device="cuda")
    B = torch.zeros((L, K, N), dtype=torch.int32, device="cuda")
    C = torch.zeros((L, M, N), dtype=torch.int32, device="cuda")
    with pytest.raises(smf.SmfError) as e:
        ctx.residue_gemm_noalloc(basis, A, 0, B, C, M, N, K)
    assert e.value.code == smf.SMF_E_NOMEM
    assert "scratch" in smf.lib().smf_last_error(ctx.handle).decode()
    basis.destroy()
    ctx.destroy()


def test_noalloc_binding_rejects_short_or_foreign_buffers(smf):
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    basis = ctx.basis_create(120)
    L = len(basis.primes)
    M, N, K = 64, 16, 32
    A = torch.zeros((M, K), dtype=torch.int32, device="cuda")
    B = torch.zeros((L, K, N), dtype=torch.int32, device="cuda")
    C = torch.zeros((L, M, N), dtype=torch.int32, device="cuda")
    for args in ((A[:, :-1].contiguous(), B, C), (A, B[:-1], C), (A, B, C[:, :-1]), (A.cpu(), B, C),
                 (A.to(torch.int64), B, C), (A.t(), B, C)):
        with pytest.raises(ValueError):
            ctx.residue_gemm_noalloc(basis, args[0], 0, args[1], args[2], M, N, K)
    with pytest.raises(ValueError):  # per-prime A needs L planes
        ctx.residue_gemm_noalloc(basis, A, M * K, B, C, M, N, K)
    basis.destroy()
    ctx.destroy()
