"""The Python binding checks tensors before their raw addresses reach the C entry
points, which trust the sizes they are given (CPU tensors stand in for CUDA ones)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1406_0236_gb300.binding import check_device_vectors  # noqa: E402


def _c(*shape, dtype=torch.complex128):
    return torch.zeros(shape, dtype=dtype)


def test_accepts_matching_operands():
    check_device_vectors(10, 0, _c(10), _c(10), expect_cuda=False)
    check_device_vectors(10, 0, _c(10, 3), None, _c(10, 3), expect_cuda=False)


@pytest.mark.parametrize("bad,msg", [
    (lambda: _c(10, dtype=torch.complex64), "complex128"),
    (lambda: _c(9), "N = 10"),
    (lambda: _c(10, 4)[:, ::2], "contiguous"),
    (lambda: _c(10, 2, 2), "N = 10"),
    (lambda: torch.zeros(10, dtype=torch.float64), "complex128"),
    (lambda: [0.0] * 10, "torch tensor"),
])
def test_rejects_bad_first_operand(bad, msg):
    with pytest.raises(ValueError, match=msg):
        check_device_vectors(10, 0, bad(), expect_cuda=False)


def test_rejects_shape_mismatch_between_operands():
    with pytest.raises(ValueError, match="differ in shape"):
        check_device_vectors(10, 0, _c(10, 3), _c(10, 2), expect_cuda=False)
    with pytest.raises(ValueError, match="differ in shape"):
        check_device_vectors(10, 0, _c(10), _c(10, 1), expect_cuda=False)


def test_rejects_host_tensor_where_cuda_is_required():
    with pytest.raises(ValueError, match="CUDA tensor"):
        check_device_vectors(10, 0, _c(10))
