"""The Python binding checks what the C ABI cannot check on a bare pointer
(device or host memory, density, element width, length) before it calls the
library, so that a wrong buffer is an exception and never a stray access."""
import numpy as np
import pytest

from paper_2508_11443_b300 import fks as F


class FakeDeviceTensor:
    """Stands in for a CUDA tensor: the checks read only these attributes."""
    is_cuda = True
    dtype = "fake"

    def __init__(self, n, size, contiguous=True):
        self.n, self.size, self.contiguous = n, size, contiguous

    def is_contiguous(self):
        return self.contiguous

    def element_size(self):
        return self.size

    def numel(self):
        return self.n

    def data_ptr(self):
        return 0x7000


def test_device_pointer_checks():
    assert F._ptr(None) is None
    assert F._ptr(FakeDeviceTensor(4, 8), "keys", 8, 4).value == 0x7000
    with pytest.raises(TypeError, match="keys: elements of 8 bytes"):
        F._ptr(FakeDeviceTensor(4, 4), "keys", 8)
    with pytest.raises(ValueError, match="vals: at least 5 elements"):
        F._ptr(FakeDeviceTensor(4, 8), "vals", None, 5)
    with pytest.raises(ValueError, match="contiguous"):
        F._ptr(FakeDeviceTensor(4, 8, contiguous=False), "q", 8)
    with pytest.raises(TypeError, match="a CUDA tensor is expected"):
        F._ptr(np.zeros(4, np.int64), "q", 8)


def test_lookup_outputs_take_the_map_width():
    asked = []

    def width():
        asked.append(1)
        return 4

    ov, of = F._outs(FakeDeviceTensor(10, 4), FakeDeviceTensor(10, 1), 10, width)
    assert ov.value == 0x7000 and of.value == 0x7000 and asked == [1]
    with pytest.raises(TypeError, match="out_vals: elements of 4 bytes"):
        F._outs(FakeDeviceTensor(10, 8), None, 10, width)
    with pytest.raises(ValueError, match="out_found: at least 10"):
        F._outs(None, FakeDeviceTensor(9, 1), 10, width)
    asked.clear()
    F._outs(None, FakeDeviceTensor(10, 1), 10, width)  # membership only: the width is not asked for
    assert asked == []


def test_host_pointer_checks():
    a = np.zeros(6, np.int64)
    assert F._hptr(a, "q", 8, 6).value == a.ctypes.data
    with pytest.raises(TypeError, match="elements of 4 bytes"):
        F._hptr(a, "out_vals", 4)
    with pytest.raises(ValueError, match="at least 7"):
        F._hptr(a, "q", 8, 7)
    with pytest.raises(ValueError, match="contiguous"):
        F._hptr(np.zeros((4, 4), np.int64)[:, 1], "q", 8)
    with pytest.raises(TypeError, match="host buffer"):
        F._hptr(FakeDeviceTensor(4, 8), "q", 8)


def test_cpu_tensors_never_reach_the_library():
    torch = pytest.importorskip("torch")
    k = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(TypeError, match="keys: a CUDA tensor is expected"):
        F.fks_build_u64(k, k, 1)
    with pytest.raises(TypeError, match="ctx: a CUDA tensor is expected"):
        F.fks_build_bytes(torch.zeros(8, dtype=torch.uint8), k, k[:0], 1)
