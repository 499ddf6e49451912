"""Replica path (one independent product per rank) on two CPU ranks over gloo."""
import os
import socket

import pytest

from paper_2605_19254_gb300 import replicas


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    import json

    import numpy as np
    import torch.distributed as dist

    from paper_2605_19254_gb300 import inputs, replicas as rp

    env = {"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)}
    re = rp.rank_env(env)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=re.rank, world_size=re.world_size)
    try:
        # each rank draws its own product
        A, B = inputs.rns_matmul_workload(rp.rank_seed(7, re.rank), 8, 16, 4, 20, 2)
        digest = int(np.bitwise_xor.reduce(A.view(np.uint64).ravel()) ^ np.bitwise_xor.reduce(B.ravel()))
        # a slow rank: rank r reports (r + 1) * 10 ms
        ms = rp.max_over_ranks(10.0 * (re.rank + 1), re.world_size)
        rate = rp.whole_job_rate(1000.0, re.world_size, ms * 1e-3)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "rate": rate, "digest": digest, "root": re.is_root}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import json

    import torch.multiprocessing as mp

    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    # every rank sees the slowest rank's time, and the same whole-job rate
    assert all(r["ms"] == 20.0 for r in res)
    assert all(r["rate"] == pytest.approx(1000.0 * ws / 0.020) for r in res)
    # the ranks computed different products; only rank 0 is the root
    assert res[0]["digest"] != res[1]["digest"]
    assert [r["root"] for r in res] == [True, False]


def test_rank_env_defaults_and_errors():
    e = replicas.rank_env({})
    assert (e.world_size, e.rank, e.local_rank, e.is_root) == (1, 0, 0, True)
    assert replicas.rank_env({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "1"}).local_rank == 1
    with pytest.raises(ValueError):
        replicas.rank_env({"WORLD_SIZE": "2", "RANK": "2"})
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.whole_job_rate(10.0, 3, 2.0) == 15.0
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1.0, 1, 0.0)


def _split_worker(rank, ws, M, port, out_dir):
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_2605_19254_gb300 import inputs, replicas as rp

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        # one product, the same on every rank; M not a multiple of the ranks (or
        # below their number: a rank with no rows)
        A, B = inputs.rns_matmul_workload(5, M, 20, 6, 20, 8)
        seen = []

        def product(a, b):  # this rank's row block, by the oracle
            seen.append(a.shape[0])
            return oracle.matmul(a, b, 9)

        C = rp.split_product(A, B, product, ws, rank)
        np.save(os.path.join(out_dir, f"c{rank}.npy"), C)
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), np.array(seen))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,M", [(2, 37), (3, 37), (3, 2)])
def test_row_block_split_on_gloo_ranks(tmp_path, orc, ws, M):
    pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp

    from paper_2605_19254_gb300 import inputs

    mp.spawn(_split_worker, args=(ws, M, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    A, B = inputs.rns_matmul_workload(5, M, 20, 6, 20, 8)
    want = orc.matmul(A, B, 9)
    C0 = np.load(tmp_path / "c0.npy")
    assert np.array_equal(C0, want)  # rank 0 gathered the whole product
    sizes = [int(np.load(tmp_path / f"rows{r}.npy")[0]) for r in range(ws)]
    assert sum(sizes) == M and max(sizes) - min(sizes) <= 1
    for r in range(1, ws):  # every other rank kept its own block
        m0, m1 = replicas.row_block(M, ws, r)
        assert np.array_equal(np.load(tmp_path / f"c{r}.npy"), want[m0:m1])


def test_row_block_bounds():
    for M in (0, 1, 5, 37, 4096):
        for ws in (1, 2, 3, 8):
            blocks = [replicas.row_block(M, ws, r) for r in range(ws)]
            assert blocks[0][0] == 0 and blocks[-1][1] == M
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            assert max(b - a for a, b in blocks) - min(b - a for a, b in blocks) <= 1
    with pytest.raises(ValueError):
        replicas.row_block(10, 2, 2)
