"""Argument checks of the binding: the arrays of the allocation-free entry
point, and the graph's edge labels.

The library trusts the sizes it is given, so the binding checks dtype, length
and device of every array before the call; these checks run on the host and
are tested here without a GPU (CPU tensors fail the size and dtype checks
before the device check is reached)."""
import numpy as np
import pytest
import torch

from paper_1912_08453_gb300 import ccpm

TL = [5, 4, 6]
TE = [(0, 1), (1, 2)]


def arrays(n=100, m=300):
    return dict(row_ptr=torch.zeros(n + 1, dtype=torch.int64), col=torch.zeros(m, dtype=torch.int32),
                labels=torch.zeros(n, dtype=torch.uint8), omega=torch.zeros(n, dtype=torch.int32),
                ebits=torch.zeros((m + 31) // 32, dtype=torch.int32))


def call(a):
    return ccpm.lcc_fixpoint_noalloc(0, a["row_ptr"], a["col"], a["labels"], TL, TE, a["omega"], a["ebits"])


@pytest.mark.parametrize("name,bad,msg", [
    ("omega", torch.zeros(99, dtype=torch.int32), "omega holds 99"),
    ("ebits", torch.zeros(9, dtype=torch.int32), "ebits holds 9"),
    ("labels", torch.zeros(100, dtype=torch.int64), "labels must have dtype"),
    ("row_ptr", torch.zeros(101, dtype=torch.int32), "row_ptr must have dtype"),
    ("col", torch.zeros(300, dtype=torch.int64), "col must have dtype"),
    ("omega", torch.zeros(200, dtype=torch.int32)[::2], "contiguous"),
])
def test_bad_arrays_are_rejected_before_the_call(name, bad, msg):
    a = arrays()
    a[name] = bad
    with pytest.raises(ValueError, match=msg):
        call(a)


def test_host_tensors_are_rejected():
    with pytest.raises(ValueError, match="must be a tensor on cuda:0"):
        call(arrays())


@pytest.mark.parametrize("bad,msg", [
    (np.zeros(9, dtype=np.uint8), "hold 9 entries"),
    (np.zeros(10, dtype=np.int32), "uint8"),
    (torch.zeros(10, dtype=torch.int64), "uint8"),
    (np.zeros(20, dtype=np.uint8)[::2], "contiguous"),
])
def test_edge_label_arrays_are_checked(bad, msg):
    # the graph's edge labels: one uint8 per CSR entry, read m bytes at a time
    with pytest.raises(ValueError, match=msg):
        ccpm.check_edge_labels(bad, 10)
