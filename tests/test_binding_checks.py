"""The Python binding refuses device buffers of the wrong placement, layout,
dtype or size before any kernel sees them (checked here with stand-in tensor
objects, so no GPU is needed)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1707_01170_gb300 import lrvol as lv


class FakeCuda:
    """Just enough of a CUDA tensor for the binding's checks."""

    def __init__(self, numel, dtype=torch.float32, contiguous=True, shape=None):
        self._n, self.dtype, self._c = numel, dtype, contiguous
        self.is_cuda = True
        self.shape = shape if shape is not None else (numel,)

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return 0xdead0000


def test_dev_accepts_a_matching_buffer():
    assert lv._dev(FakeCuda(12), torch.float32, 12, exact=True) == 0xdead0000
    assert lv._dev(FakeCuda(40), torch.float32, 12) == 0xdead0000       # larger is fine unless exact


@pytest.mark.parametrize("bad,err", [
    (torch.zeros(12), ValueError),                                      # host tensor
    (FakeCuda(12, contiguous=False), ValueError),                       # strided view
    (FakeCuda(12, dtype=torch.float64), TypeError),                     # wrong dtype
    (FakeCuda(11), ValueError),                                         # too small
])
def test_dev_rejects(bad, err):
    with pytest.raises(err):
        lv._dev(bad, torch.float32, 12)


def test_dev_exact_size():
    with pytest.raises(ValueError):
        lv._dev(FakeCuda(13), torch.float32, 12, exact=True)


def test_points_shape():
    assert lv._points(FakeCuda(30, shape=(10, 3))) == 10
    with pytest.raises(ValueError):
        lv._points(FakeCuda(30, shape=(15, 2)))
    with pytest.raises(TypeError):
        lv._points(FakeCuda(30, dtype=torch.float16, shape=(10, 3)))
