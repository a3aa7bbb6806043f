"""Host logic of the Python binding that needs no GPU: the marshalling of a
batch of problems into the device addresses and lengths that
dpd_estimate_batched takes.  The tensor checks (complex64, CUDA, contiguous)
are replaced by a no-op so that CPU tensors stand in for device ones; the
address arithmetic is the same."""
import numpy as np
import pytest
import torch

import paper_1612_09001_gb300 as dpd


@pytest.fixture
def cpu_tensors_allowed(monkeypatch):
    monkeypatch.setattr(dpd, "_check_samples", lambda t, name: None)


def test_two_d_batch_gives_row_addresses(cpu_tensors_allowed):
    X = torch.zeros((5, 12), dtype=torch.complex64)
    addr, lens, dev = dpd._batch_pointers(X, "u")
    assert addr.dtype == np.uint64 and lens.dtype == np.int64
    assert [int(a) for a in addr] == [X.data_ptr() + 12 * 8 * i for i in range(5)]
    assert [int(n) for n in lens] == [12] * 5
    assert dev == X.device


def test_list_of_rows_matches_the_two_d_form(cpu_tensors_allowed):
    X = torch.zeros((4, 7), dtype=torch.complex64)
    a2, n2, _ = dpd._batch_pointers(X, "u")
    al, nl, _ = dpd._batch_pointers(list(X), "u")
    assert np.array_equal(a2, al) and np.array_equal(n2, nl)


def test_list_of_different_lengths(cpu_tensors_allowed):
    xs = [torch.zeros(n, dtype=torch.complex64) for n in (3, 1, 9)]
    addr, lens, _ = dpd._batch_pointers(xs, "u")
    assert [int(a) for a in addr] == [x.data_ptr() for x in xs]
    assert [int(n) for n in lens] == [3, 1, 9]


@pytest.mark.parametrize("bad", [torch.zeros(6, dtype=torch.complex64),            # 1-D tensor
                                 torch.zeros((0, 4), dtype=torch.complex64),       # no problems
                                 torch.zeros((3, 0), dtype=torch.complex64),       # empty rows
                                 torch.zeros((2, 2, 2), dtype=torch.complex64)])   # 3-D
def test_malformed_batches_are_refused(cpu_tensors_allowed, bad):
    with pytest.raises(ValueError):
        dpd._batch_pointers(bad, "u")


def test_empty_list_is_refused(cpu_tensors_allowed):
    with pytest.raises(ValueError):
        dpd._batch_pointers([], "u")


def test_checks_still_run_without_the_stand_in():
    """With the real checks a CPU tensor (not a CUDA one) is refused before any
    address is formed, in both forms."""
    X = torch.zeros((2, 4), dtype=torch.complex64)
    with pytest.raises(ValueError):
        dpd._batch_pointers(X, "u")
    with pytest.raises(ValueError):
        dpd._batch_pointers(list(X), "u")
    with pytest.raises(TypeError):
        dpd._batch_pointers([torch.zeros(4, dtype=torch.float32)], "u")
