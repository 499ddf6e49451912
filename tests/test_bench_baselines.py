"""The paper-design host baseline timed by bench.py computes the exact product."""
import numpy as np

from paper_2605_19254_gb300 import inputs


def test_paper_design_baseline_is_exact(orc):
    import bench

    A, B = inputs.rns_matmul_workload(11, 9, 70, 5, 20, 3)
    got = bench.paper_design_matmul(A, B, 5)
    assert np.array_equal(got, orc.matmul(A, B, 5))
    # the prime bound of the paper's design: K (p-1)^2 + (p-1) < 2^53
    p = orc.fp64_prime_cap(4096)
    assert 4096 * (p - 1) ** 2 + (p - 1) < 2 ** 53 - 1 <= 4096 * p ** 2 + p
