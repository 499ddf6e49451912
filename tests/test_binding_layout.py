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
