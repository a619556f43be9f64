"""Host-side packing of the batched solve: systems back to back, the queue's longest-first order."""
import numpy as np
import pytest

from paper_1406_5802_gb300.batch import pack_layout


def test_offsets_are_back_to_back():
    sizes = [3, 7, 1, 7, 5]
    offA, offv, order = pack_layout(sizes)
    assert offA.tolist() == [0, 9, 58, 59, 108]  # running sums of n_i^2
    assert offv.tolist() == [0, 3, 10, 11, 18]   # running sums of n_i
    assert order.tolist() == [1, 3, 4, 0, 2]     # decreasing n, ties in index order
    assert offA.dtype == np.int64 and offv.dtype == np.int64 and order.dtype == np.int32


def test_large_orders_do_not_overflow():
    offA, _, _ = pack_layout([4096] * 200)
    assert offA[-1] == 199 * 4096 * 4096  # beyond 2^31


@pytest.mark.parametrize("bad", [[], [0, 3], [[2, 3]]])
def test_bad_sizes_are_rejected(bad):
    with pytest.raises(ValueError):
        pack_layout(bad)
