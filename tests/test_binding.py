"""Host-side argument checks of the Python binding: a tensor that is not a
contiguous CUDA tensor of the right element size and length is refused with
HEGET_EINVAL before any call reaches the library, so a CPU tensor or a short
buffer never becomes a device address.  No GPU needed."""
import pytest


class FakeTensor:
    """Just the tensor attributes the binding inspects."""

    def __init__(self, numel, itemsize=8, floating=True, cuda=True, contiguous=True):
        import torch
        self._n, self._size, self.is_cuda, self._contig = numel, itemsize, cuda, contiguous
        self.dtype = {(8, True): torch.float64, (8, False): torch.int64, (4, True): torch.float32,
                      (4, False): torch.int32, (1, False): torch.uint8}[(itemsize, floating)]

    def is_contiguous(self):
        return self._contig

    def element_size(self):
        return self._size

    def numel(self):
        return self._n

    def data_ptr(self):
        return 0x7F0000001000


def _einval(H, fn, *args, what):
    with pytest.raises(H.HegetError) as e:
        fn(*args)
    assert e.value.status == H.HEGET_EINVAL and what in str(e.value)


def test_tensor_checks(heget_lib):
    H = heget_lib
    ok = FakeTensor(10)
    assert H._f64s(ok, "x", 10) == ok.data_ptr()
    assert H._f64s(None, "x", 10) is None and H._f64s(1234, "x", 10) == 1234
    _einval(H, H._f64s, FakeTensor(10, cuda=False), "x", 10, what="x must be a CUDA tensor")
    _einval(H, H._f64s, FakeTensor(10, contiguous=False), "x", 10, what="x must be contiguous")
    _einval(H, H._f64s, FakeTensor(10, itemsize=4), "x", 10, what="needs 8-byte floating-point elements")
    _einval(H, H._f64s, FakeTensor(10, floating=False), "x", 10, what="needs 8-byte floating-point elements")
    _einval(H, H._f64s, FakeTensor(9), "x", 10, what="holds 9 elements, needs 10")
    assert H._dev(FakeTensor(8, 4, False), "words", 8, 4, False) == ok.data_ptr()
    _einval(H, H._dev, FakeTensor(8, 4, True), "words", 8, 4, False, what="needs 4-byte integer elements")
    # result buffers: 80 bytes of any element type
    assert H._result(FakeTensor(80, 1, False)) and H._result(FakeTensor(10, 8, True))
    _einval(H, H._result, FakeTensor(79, 1, False), what="holds 79 elements, needs 80")
    _einval(H, H._result, FakeTensor(9, 8, True), what="holds 9 elements, needs 10")


def test_wrappers_refuse_cpu_tensors_before_the_call(heget_lib):
    """CPU tensors (real ones) are refused with the argument's name; the
    library is never handed a host address."""
    import torch
    H = heget_lib
    n, N = 4, 8
    mom = torch.zeros((N, n + 2, 4), dtype=torch.float64)
    out = torch.zeros(N, dtype=torch.float64)
    _einval(H, H.heget_amp2, None, n, N, mom, out, what="momenta must be a CUDA tensor")
    _einval(H, H.heget_phase_space_ex, None, 1, 0, N, n, H.sampler_toy_pdf(), mom, what="momenta must be a CUDA")
    _einval(H, H.heget_xsec_async, None, n, 1, 0, N, H.sampler_toy_pdf(), 32, torch.zeros(80, dtype=torch.uint8),
            what="result_dev must be a CUDA tensor")
    _einval(H, H.heget_f32_round, out, torch.zeros(N, dtype=torch.float32), N, what="x must be a CUDA tensor")
    _einval(H, H.heget_hist, None, n, 1, 0, N, H.sampler_toy_pdf(), out, [(0, 4, 0.0, 1.0)], out,
            what="w must be a CUDA tensor")
