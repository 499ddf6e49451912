"""Serving Smith-form jobs: continuous batching on one GPU (the Smith form of
Sections 1-2 as a request stream).  A mix of jobs of different sizes and entry
widths, submitted in two waves (the second while the first runs) under a
budget of about three jobs, gives bit for bit the Smith forms of the same
matrices computed alone, and the oracle's where it is quick; the bytes in use
never exceed the budget; a job larger than the budget is refused."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import smith  # noqa: E402
from paper_2605_19254_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def smf():
    from paper_2605_19254_gb300 import build, smf as _smf
    build.build()
    assert torch.cuda.is_available()
    return _smf


def _jobs():
    out = []
    sizes = [(24, 7), (300, 20), (50, 40), (700, 7), (90, 20), (35, 40), (1200, 20), (64, 7)]
    for i, (n, k) in enumerate(sizes):
        if i % 3 == 2:  # some matrices with a planted Smith form
            s = [1] * (n - 3) + [6, 60, 60 * 7]
            A = np.array(inputs.smith_known_matrix(100 + i, s, n), dtype=np.int64)
        else:
            A = inputs.uniform_int(100 + i, "SV", (n, n), -(1 << k), 1 << k)
        out.append((A, int(np.abs(A).max()).bit_length(), 10 + i))
    return out


@pytest.mark.parametrize("form", ["limb", "fp64"])
def test_served_smith_forms_equal_alone(smf, form):
    fm = smf.SMF_FORM_INT8LIMB if form == "limb" else smf.SMF_FORM_FP64
    jobs = _jobs()
    if form == "fp64":
        jobs = [j for j in jobs if j[0].shape[0] <= 300]
    ctx = smf.Context(0, fm)
    alone = [ctx.smith_form(torch.from_numpy(A[..., None].copy()), seed=sd, a_bits=b)[0] for A, b, sd in jobs]
    ctx.destroy()
    for (A, b, sd), s in zip(jobs, alone):
        if A.shape[0] <= 40:
            assert s == smith.smith_form(A.tolist())
    biggest = max(A.shape[0] for A, _, _ in jobs)
    budget = 3 * (64 * biggest * biggest + (64 << 20))
    srv = smf.SmithServer(0, fm, budget, workers=3)
    try:
        half = len(jobs) // 2
        ids = [srv.submit(A, b, sd) for A, b, sd in jobs[:half]]
        peak = 0
        for _ in range(20):  # the second wave arrives while the first runs
            q, r, used = srv.stats()
            peak = max(peak, used)
            time.sleep(0.005)
        ids += [srv.submit(A, b, sd) for A, b, sd in jobs[half:]]
        while True:
            q, r, used = srv.stats()
            peak = max(peak, used)
            if q == 0 and r == 0:
                break
            time.sleep(0.002)
        srv.drain()
        assert peak <= budget
        for jid, (A, b, sd), want in zip(ids, jobs, alone):
            state, status, (t0, t1, t2) = srv.job(jid)
            assert state == smf.SMF_JOB_DONE and status == smf.SMF_OK
            assert t0 <= t1 <= t2
            assert srv.result(jid, A.shape[0]) == want
    finally:
        srv.destroy()


def test_smith_server_refuses_oversized_job(smf):
    srv = smf.SmithServer(0, smf.SMF_FORM_INT8LIMB, 80 << 20, workers=1)
    try:
        A = inputs.uniform_int(1, "SV", (600, 600), -100, 100)  # 64 n^2 + 64 MiB > 80 MiB
        with pytest.raises(smf.SmfError) as e:
            srv.submit(A, 7)
        assert e.value.code == smf.SMF_E_NOMEM
        small = inputs.uniform_int(2, "SV", (20, 20), -100, 100)
        jid = srv.submit(small, 7, 3)
        srv.drain()
        assert srv.result(jid, 20) == smith.smith_form(small.tolist())
    finally:
        srv.destroy()


def test_many_sizes_under_eight_workers(smf):
    """Jobs of many sizes under eight workers: every worker's context builds new
    RNS bases while the others' kernels and copies run, so each job depends on
    its bases being on the device before its first kernel reads them.  Every job
    ends done; the planted ones give their planted forms; random ones equal the
    same matrix computed alone."""
    batch = inputs.batched_smith_workload(5, count=128, lo=32, hi=384)
    srv = smf.SmithServer(0, smf.SMF_FORM_INT8LIMB, 0, workers=8)
    try:
        ids = [srv.submit(A, b, 1) for _, b, A, _ in batch]
        srv.drain()
        got = {}
        for jid, (n, b, A, s) in zip(ids, batch):
            state, status, _ = srv.job(jid)
            assert state == smf.SMF_JOB_DONE and status == smf.SMF_OK, (n, status, srv.message(jid))
            got[jid] = srv.result(jid, n)
            if s is not None:
                assert got[jid] == list(s)
    finally:
        srv.destroy()
    ctx = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    try:
        checked = 0
        for jid, (n, b, A, s) in zip(ids, batch):
            if s is None and checked < 12:
                alone = ctx.smith_form(torch.from_numpy(A[..., None].copy()), seed=1, a_bits=b)[0]
                assert got[jid] == alone
                checked += 1
        assert checked == 12
    finally:
        ctx.destroy()
