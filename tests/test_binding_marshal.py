"""Argument marshalling of the ctypes binding (no GPU, no library call): which memory
kind each array type maps to, when inputs are copied, and which outputs are refused."""
import numpy as np
import pytest

from paper_2502_10640_gb300 import capi


def test_contiguous_float64_host_array_is_passed_in_place():
    a = np.zeros((7, 3))
    ptr, kind, keep = capi._arg(a, 7, writable=True)
    assert kind == capi.PP_MEM_HOST and ptr == a.ctypes.data and keep is a


def test_inputs_of_other_layouts_are_copied_to_c_float64():
    f = np.asfortranarray(np.arange(21.0).reshape(7, 3))
    ptr, kind, keep = capi._arg(f, 7, writable=False)
    assert kind == capi.PP_MEM_HOST and keep.flags.c_contiguous and np.array_equal(keep, f)
    ptr, kind, keep = capi._arg(np.ones((7, 3), dtype=np.float32), 7, writable=False)
    assert keep.dtype == np.float64
    ptr, kind, keep = capi._arg([[1, 2, 3]] * 7, 7, writable=False)
    assert keep.shape == (7, 3)


def test_outputs_must_be_writable_in_place():
    with pytest.raises(ValueError):
        capi._arg(np.zeros((7, 3), dtype=np.float32), 7, writable=True)
    with pytest.raises(ValueError):
        capi._arg(np.asfortranarray(np.zeros((7, 3))), 7, writable=True)


def test_shape_is_checked():
    with pytest.raises(ValueError):
        capi._arg(np.zeros((7, 2)), 7, writable=False)
    with pytest.raises(ValueError):
        capi._arg(np.zeros((6, 3)), 7, writable=True)


def test_cpu_tensor_that_is_not_pinned_goes_through_host_memory():
    torch = pytest.importorskip("torch")
    t = torch.zeros((5, 3), dtype=torch.float64)
    ptr, kind, keep = capi._arg(t, 5, writable=True)
    assert kind == capi.PP_MEM_HOST and ptr == t.data_ptr()   # a view, no copy


def test_mixed_kinds_in_one_call_are_refused():
    assert capi._same_kind(capi.PP_MEM_HOST, None, capi.PP_MEM_HOST) == capi.PP_MEM_HOST
    with pytest.raises(ValueError):
        capi._same_kind(capi.PP_MEM_HOST, capi.PP_MEM_DEVICE)
    with pytest.raises(ValueError):
        capi._same_kind(capi.PP_MEM_HOST_MAPPED, capi.PP_MEM_HOST)
