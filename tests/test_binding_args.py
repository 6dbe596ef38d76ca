"""Argument checks of the Python binding (CPU).

The C ABI takes device pointers for almost every buffer; a host tensor's
address handed to a kernel would be dereferenced on the GPU.  The binding
refuses host tensors there, refuses device tensors where the host-buffer entry
point expects host memory, and checks the dtype and size of the solver's
output buffers before any library call.  CUDA tensors are stood in for by a
small fake (only its attributes are read), so these checks run without a GPU.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")


class FakeCuda:
    """The attributes of a CUDA tensor the binding's checks read."""

    def __init__(self, shape, dtype=torch.float64, strides=None, addr=1 << 20):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = True
        self._strides = strides or self._fortran(self.shape)
        self._addr = addr

    @staticmethod
    def _fortran(shape):
        if len(shape) == 1:
            return (1,)
        return (1, max(1, shape[0]))

    def numel(self):
        k = 1
        for d in self.shape:
            k *= d
        return k

    def dim(self):
        return len(self.shape)

    def stride(self, i=None):
        return self._strides if i is None else self._strides[i]

    def data_ptr(self):
        return self._addr


def test_device_pointer_refuses_host_tensors():
    import paper_1912_04062_gb300 as sk
    assert sk._ptr(None).value is None
    assert sk._ptr(FakeCuda((4,))).value == 1 << 20
    with pytest.raises(TypeError):
        sk._ptr(torch.zeros(4, dtype=torch.float64))


def test_host_pointer_refuses_device_tensors():
    import paper_1912_04062_gb300 as sk
    t = torch.zeros(4, dtype=torch.float64)
    assert sk._hptr(t).value == t.data_ptr()
    assert sk._hptr(None).value is None
    with pytest.raises(TypeError):
        sk._hptr(FakeCuda((4,)))


def test_output_buffers_checked_for_dtype_and_size():
    import paper_1912_04062_gb300 as sk
    assert isinstance(sk._out(FakeCuda((8,)), torch.float64, 8, "lam"), ctypes.c_void_p)
    assert sk._out(None, torch.float64, 8, "lam").value is None
    with pytest.raises(TypeError):
        sk._out(FakeCuda((7,)), torch.float64, 8, "lam")            # too short
    with pytest.raises(TypeError):
        sk._out(FakeCuda((8,), dtype=torch.float32), torch.float64, 8, "lam")
    with pytest.raises(TypeError):
        sk._out(FakeCuda((1,), dtype=torch.int64), torch.int32, 1, "d_info")
    with pytest.raises(TypeError):
        sk._out(torch.zeros(8, dtype=torch.float64), torch.float64, 8, "lam")  # host memory


def test_eigenvector_blocks_checked_for_shape_and_layout():
    import paper_1912_04062_gb300 as sk
    n, nev = 10, 5
    assert sk._zbuf(FakeCuda((n, nev)), n, nev, "Zr").value == 1 << 20
    assert sk._zbuf(FakeCuda((n, nev + 3)), n, nev, "Zr").value == 1 << 20   # more columns than asked
    assert sk._zbuf(FakeCuda((n, 1)), n, 1, "Zr").value == 1 << 20
    assert sk._zbuf(None, n, nev, "Zr").value is None
    with pytest.raises(TypeError):
        sk._zbuf(FakeCuda((n + 1, nev)), n, nev, "Zr")                       # wrong row count
    with pytest.raises(TypeError):
        sk._zbuf(FakeCuda((n, nev - 1)), n, nev, "Zr")                       # too few columns
    with pytest.raises(TypeError):
        sk._zbuf(FakeCuda((n, nev), strides=(nev, 1)), n, nev, "Zr")        # row-major
    with pytest.raises(TypeError):
        sk._zbuf(FakeCuda((n, nev), dtype=torch.float32), n, nev, "Zr")


def test_solver_entry_points_refuse_a_host_matrix():
    import paper_1912_04062_gb300 as sk
    A = torch.zeros((4, 4), dtype=torch.float64)
    with pytest.raises(TypeError):
        sk.skew_eig_ex(A, 2, None, None, None, FakeCuda((16,), dtype=torch.uint8), None)
    with pytest.raises(TypeError):
        sk.skew_eig(A, 2)
