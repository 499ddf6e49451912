"""GPU tests of the serving loop: jobs served in a mix (several batches,
arriving while others run, under an HBM budget) give bit for bit the results
of the same products computed alone, and the budget holds."""
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


def _jobs(seed, count, r=32, wb=8):
    ns = inputs.log_uniform_int(seed, "serve_n", count, 16, 600)
    out = []
    for i, n in enumerate(ns):
        n = int(n)
        k = (7, 20, 40)[i % 3]
        A, B = inputs.rns_matmul_workload(inputs.stream_seed(seed, f"job{i}"), n, n, r, k, wb)
        Wc = (k + 64 * wb - 1 + int(np.ceil(np.log2(max(n, 2)))) + 2 + 63) // 64
        out.append((n, k, A, B, Wc))
    return out


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_served_results_equal_alone(smf, orc, form):
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB if form == "limb" else smf.SMF_FORM_FP64)
    jobs = _jobs(3, 18 if form == "limb" else 6)
    As = [_dev(A) for _, _, A, _, _ in jobs]
    Bs = [_dev(B) for _, _, _, B, _ in jobs]
    alone = []
    for (n, k, _, _, Wc), A, B in zip(jobs, As, Bs):
        C = torch.zeros((n, 32, Wc), dtype=torch.int64, device="cuda")
        ctx.rns_matmul(A, B, C, a_bits=k)
        alone.append(C)
    ctx.status_sync()
    # a budget of about three of the larger jobs: the mix runs as several batches
    ws = sorted(ctx.rns_matmul_grouped_workspace([A], [B], [C], a_bits=k)
                for (n, k, _, _, Wc), A, B, C in zip(jobs, As, Bs, alone))
    budget = ws[-1] + ws[-2] + ws[-3]
    srv = smf.Server(ctx, budget, max_batch=5)
    try:
        mixed = [torch.full_like(C, 7) for C in alone]
        half = len(jobs) // 2
        ids = [srv.submit(A, B, C, a_bits=k) for (n, k, *_), A, B, C in zip(jobs[:half], As, Bs, mixed)]
        srv.step()  # the first wave is on the device ...
        peak = srv.stats()[2]
        ids += [srv.submit(A, B, C, a_bits=k)  # ... when the second arrives
                for (n, k, *_), A, B, C in zip(jobs[half:], As[half:], Bs[half:], mixed[half:])]
        steps = 0
        while True:
            launched = srv.step()
            q, running, in_use = srv.stats()
            peak = max(peak, in_use)
            assert in_use <= budget
            if q == 0 and running == 0:
                break
            steps += 1
            assert steps < 100000
            if launched == 0:
                torch.cuda.synchronize()
        states = [srv.job(j) for j in ids]
        assert all(s == smf.SMF_JOB_DONE and code == 0 for s, code, _ in states)
        starts = sorted({t[1] for _, _, t in states})
        assert len(starts) >= 2  # more than one batch
        for C, Cm in zip(alone, mixed):
            assert torch.equal(C, Cm)
        for i in (0, len(jobs) - 1):  # and against the oracle
            n, k, A, B, Wc = jobs[i]
            assert np.array_equal(mixed[i].cpu().numpy().view(np.uint64), orc.matmul(A, B, Wc))
    finally:
        srv.destroy()
        ctx.destroy()


def test_budget_and_errors(smf):
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    n, k, A, B, Wc = _jobs(5, 1)[0]
    A, B = _dev(A), _dev(B)
    C = torch.zeros((n, 32, Wc), dtype=torch.int64, device="cuda")
    need = ctx.rns_matmul_grouped_workspace([A], [B], [C], a_bits=k)
    small = smf.Server(ctx, max(1, need - 1), max_batch=4)
    try:
        with pytest.raises(smf.SmfError) as e:
            small.submit(A, B, C, a_bits=k)
        assert e.value.code == smf.SMF_E_NOMEM
    finally:
        small.destroy()
    with pytest.raises(smf.SmfError):
        smf.Server(ctx, 0)
    srv = smf.Server(ctx, need, max_batch=4)  # room for exactly one at a time
    try:
        Cs = [torch.zeros_like(C) for _ in range(3)]
        ids = [srv.submit(A, B, Ci, a_bits=k) for Ci in Cs]
        assert srv.step() == 1
        srv.drain()
        assert all(srv.job(j)[0] == smf.SMF_JOB_DONE for j in ids)
        assert srv.stats() == (0, 0, 0)
        for Ci in Cs[1:]:
            assert torch.equal(Ci, Cs[0])
    finally:
        srv.destroy()
        ctx.destroy()
