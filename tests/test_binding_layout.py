"""The Python binding's big-integer matrix descriptors (argument marshalling
only, no GPU): rows, columns, words per entry and the leading dimension read
from a tensor's strides, for contiguous tensors, row slices, size-one and
empty dimensions, and the layouts the library cannot take."""
import pytest

torch = pytest.importorskip("torch")

from paper_2605_19254_gb300.smf import bigmat  # noqa: E402


def test_contiguous_and_row_slices():
    t = torch.zeros((5, 7, 3), dtype=torch.int64)
    d = bigmat(t, 20)
    assert (d.rows, d.cols, d.ld, d.words, d.bits, d.on_device) == (5, 7, 7, 3, 20, 0)
    # columns 2..5 of every row: entries contiguous, rows 7 entries apart
    v = t[:, 2:6, :]
    d = bigmat(v)
    assert (d.rows, d.cols, d.ld, d.words) == (5, 4, 7, 3)
    assert d.data == v.data_ptr()


def test_size_one_and_empty_dimensions_carry_no_layout():
    # one row, or one word, whatever their strides
    t = torch.zeros((4, 6, 1), dtype=torch.int64)
    d = bigmat(t[..., :1])
    assert (d.rows, d.cols, d.ld, d.words) == (4, 6, 6, 1)
    row = torch.zeros((3, 9, 2), dtype=torch.int64)[1:2]
    d = bigmat(row)
    assert (d.rows, d.cols, d.ld, d.words) == (1, 9, 9, 2)
    col = torch.zeros((8, 1), dtype=torch.int64)[..., None]  # stride 0 on the new axis
    d = bigmat(col)
    assert (d.rows, d.cols, d.words) == (8, 1, 1)
    empty = torch.zeros((0, 5, 2), dtype=torch.int64)
    d = bigmat(empty)
    assert (d.rows, d.cols, d.ld, d.words) == (0, 5, 5, 2)


def test_layouts_the_library_cannot_take():
    t = torch.zeros((4, 6, 2), dtype=torch.int64)
    with pytest.raises(ValueError):
        bigmat(t.transpose(0, 1))  # entries not contiguous along a row
    with pytest.raises(ValueError):
        bigmat(t[:, :, ::2])  # every other word: entries one word wide but two words apart
    with pytest.raises(ValueError):
        bigmat(torch.zeros((4, 6), dtype=torch.int64))  # not [rows, cols, W]


class _DeviceLike:
    """What the residue product's operand checks read of a tensor (device,
    dtype, contiguity, entry count), so that they run without a GPU."""

    def __init__(self, n, cuda=True, dtype=None, contiguous=True):
        self._n, self.is_cuda, self._contiguous = n, cuda, contiguous
        self.dtype = torch.int32 if dtype is None else dtype

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._contiguous


def test_residue_product_operand_checks():
    # the binding refuses operands the C side could not check on the device:
    # wrong device, type or layout, or fewer entries than M, N, K and the
    # per-prime stride of A imply
    from paper_2605_19254_gb300.smf import Context

    class _Basis:
        primes = [101, 103, 107]

    check = Context._check_residue_operands
    L, M, N, K = 3, 4, 5, 6
    A, B, C = _DeviceLike(M * K), _DeviceLike(L * K * N), _DeviceLike(L * M * N)
    check(_Basis, A, 0, B, C, M, N, K)  # A shared by every prime
    check(_Basis, _DeviceLike((L - 1) * 2 * M * K + M * K), 2 * M * K, B, C, M, N, K)  # per-prime A, padded
    check(_Basis, _DeviceLike(0), 0, _DeviceLike(0), _DeviceLike(0), 0, N, 0)  # nothing to compute
    bad = [
        ((_DeviceLike(M * K - 1), 0, B, C), "A holds"),
        ((_DeviceLike(L * M * K - 1), M * K, B, C), "A holds"),
        ((A, 0, _DeviceLike(L * K * N - 1), C), "B holds"),
        ((A, 0, B, _DeviceLike(L * M * N - 1)), "C holds"),
        ((_DeviceLike(M * K, cuda=False), 0, B, C), "CUDA"),
        ((A, 0, _DeviceLike(L * K * N, dtype=torch.float32), C), "int32"),
        ((A, 0, B, _DeviceLike(L * M * N, dtype=torch.int64)), "int32"),
        ((A, 0, B, _DeviceLike(L * M * N, contiguous=False)), "contiguous"),
        ((A, -1, B, C), "negative"),
    ]
    for (a, stride, b, c), msg in bad:
        with pytest.raises(ValueError, match=msg):
            check(_Basis, a, stride, b, c, M, N, K)
    with pytest.raises(ValueError, match="negative"):
        check(_Basis, A, 0, B, C, -1, N, K)
