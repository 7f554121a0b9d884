"""The binding's argument checks: a tensor the library cannot take (host
memory where device memory is needed and the reverse, a wrong dtype, shape
or layout) is refused in Python, before its pointer reaches the library."""

import numpy as np
import pytest
import torch

from paper_2602_21600_gb300.aqr import _check_len, _check_tensor


def test_host_tensor_refused_where_device_memory_is_needed():
    with pytest.raises(ValueError, match="CUDA tensor"):
        _check_tensor(torch.zeros((4, 8)), torch.float32, "q", True)


def test_device_flag_false_accepts_host_tensors():
    p = _check_tensor(torch.zeros((4, 8)), torch.float32, "q_host", False, ndim=2)
    assert p.value is not None


def test_dtype_ndim_shape_and_layout():
    t = torch.zeros((4, 8))
    with pytest.raises(TypeError, match="dtype"):
        _check_tensor(t.double(), torch.float32, "q", False)
    with pytest.raises(ValueError, match="dimensions"):
        _check_tensor(t[0], torch.float32, "q", False, ndim=2)
    with pytest.raises(ValueError, match="shape"):
        _check_tensor(t, torch.float32, "ids", False, shape=(4, 9))
    with pytest.raises(ValueError, match="contiguous"):
        _check_tensor(t.t(), torch.float32, "q", False)
    # rows: a row stride is allowed, a strided last dimension is not
    wide = torch.zeros((4, 12))
    _check_tensor(wide[:, :8], torch.float32, "x", False, rows=True)
    with pytest.raises(ValueError, match="dense"):
        _check_tensor(wide[:, ::2], torch.float32, "x", False, rows=True)
    with pytest.raises(TypeError, match="torch tensor"):
        _check_tensor(np.zeros((4, 8), np.float32), torch.float32, "q", False)


def test_list_lengths():
    _check_len(np.zeros(3), 3, "k_list")
    with pytest.raises(ValueError, match="2 entries, expected 3"):
        _check_len(np.zeros(2), 3, "k_list")
