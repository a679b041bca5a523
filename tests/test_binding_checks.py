"""The Python binding refuses, before any library call, what the C ABI cannot
check through bare pointers: a misspelt svn_params field, and buffers whose
element count, dtype or memory layout differs from the layout the call reads
or writes (no GPU)."""
import numpy as np
import pytest
import torch

from paper_2204_10822_gb300 import solver as S


def test_unknown_param_is_refused():
    with pytest.raises(TypeError, match="restrat"):
        S.default_params(restrat=100)
    p = S.default_params(restart=100, ew_tail=0.25, precision="mixed")
    assert p.restart == 100 and p.ew_tail == 0.25


def test_element_counts_are_checked():
    S._check_numel(np.zeros((5, 5, 2)), 50, "v")
    S._check_numel(torch.zeros(5, 5, 2), 50, "v")
    with pytest.raises(ValueError, match="v: expected 50"):
        S._check_numel(np.zeros((4, 5, 2)), 50, "v")
    with pytest.raises(ValueError, match="pi: expected 48"):
        S._check_numel(torch.zeros(2, 2, 4, 2), 48, "pi")
    S._check_numel(np.zeros(7), None, "any")            # no expected size: not checked


def test_host_inputs_are_converted_and_sized():
    ptr, keep = S._hptr(np.arange(9, dtype=np.float32).reshape(3, 3), 9, "h")
    assert keep.dtype == np.float64 and keep.flags.c_contiguous and ptr == keep.ctypes.data
    with pytest.raises(ValueError, match="h: expected 16"):
        S._hptr(np.zeros((3, 3)), 16, "h")


def test_host_output_buffer_is_checked():
    out = np.zeros((5, 5, 2))
    assert S._host_out(out, 50) == out.ctypes.data
    with pytest.raises(TypeError):
        S._host_out(np.zeros((5, 5, 2), dtype=np.float32), 50)
    with pytest.raises(TypeError):
        S._host_out(np.zeros((5, 10, 2))[:, ::2], 50)          # not contiguous
    ro = np.zeros((5, 5, 2))
    ro.flags.writeable = False
    with pytest.raises(TypeError):
        S._host_out(ro, 50)
    with pytest.raises(ValueError):
        S._host_out(np.zeros((5, 5, 3)), 50)


def test_device_pointer_requires_a_cuda_float64_tensor():
    with pytest.raises(TypeError, match="x: expected a contiguous CUDA float64 tensor"):
        S._ptr(torch.zeros(10, dtype=torch.float64), 10, "x")
    with pytest.raises(TypeError):
        S._ptr(np.zeros(10), 10, "x")
