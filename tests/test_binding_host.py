"""Host logic of the Python binding, without a GPU: argument marshalling and
option handling (no library call computes anything here)."""
import numpy as np
import pytest

from paper_1812_10302_gb300 import dtws


def test_arg_makes_contiguous_arrays_of_the_wanted_type():
    a = np.arange(20, dtype=np.float64)[::2]  # strided FP64
    arg = dtws._Arg(a, np.float32)
    assert arg.obj.dtype == np.float32 and arg.obj.flags["C_CONTIGUOUS"]
    assert arg.size == 10 and arg.ptr == arg.obj.ctypes.data
    np.testing.assert_array_equal(arg.obj, a.astype(np.float32))
    lst = dtws._Arg([3, 1, 2], np.int64)
    assert lst.obj.dtype == np.int64 and lst.size == 3


def test_arg_converts_torch_tensors():
    torch = pytest.importorskip("torch")
    t = torch.arange(12, dtype=torch.float64).reshape(3, 4).t()  # not contiguous
    arg = dtws._Arg(t, np.float32)
    assert arg.obj.dtype == torch.float32 and arg.obj.is_contiguous()
    assert arg.size == 12 and arg.ptr == arg.obj.data_ptr()
    np.testing.assert_array_equal(arg.obj.numpy(), t.numpy().astype(np.float32))
    i = dtws._Arg(torch.tensor([1, 2], dtype=torch.int32), np.int64)
    assert i.obj.dtype == torch.int64


def test_stream_pointer():
    class S:
        cuda_stream = 1234

    assert dtws._stream_ptr(5) == 5
    assert dtws._stream_ptr(S()) == 1234
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert dtws._stream_ptr(None) == 0


def test_apply_options_sets_fields_and_rejects_unknown_names():
    o = dtws.dtws_options()
    dtws.apply_options(o, {"exclusion_zone": 7, "unnormalised": 1, "delta": 0.25})
    assert (o.exclusion_zone, o.unnormalised, o.delta) == (7, 1, 0.25)
    with pytest.raises(KeyError, match="exclusion_zon"):
        dtws.apply_options(o, {"exclusion_zon": 3})
    assert o.exclusion_zone == 7  # nothing was applied
