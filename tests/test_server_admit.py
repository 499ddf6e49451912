"""The serving loop's admission rule on its own (host code of the library,
no GPU needed): queued jobs in arrival order are admitted while their
workspace fits what is left of the budget, at most max_batch of them."""
import pytest

from paper_2605_19254_gb300 import smf


def test_admits_in_order_and_lets_small_jobs_pass():
    # 100 left: job 0 (60) fits, job 1 (50) does not, job 2 (40) fits the rest
    assert smf.server_admit(100, [60, 50, 40, 1], 8) == [1, 0, 1, 0]
    # exact fit, then nothing left
    assert smf.server_admit(100, [100, 1], 8) == [1, 0]
    assert smf.server_admit(0, [0, 1], 8) == [1, 0]


def test_max_batch_and_empty_queue():
    assert smf.server_admit(1000, [1] * 5, 3) == [1, 1, 1, 0, 0]
    assert smf.server_admit(1000, [], 3) == []
    assert smf.server_admit(10, [11, 12], 3) == [0, 0]


def test_bad_arguments():
    with pytest.raises(ValueError):
        smf.server_admit(10, [1], -1)
