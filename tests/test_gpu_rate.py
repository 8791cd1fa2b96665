"""GPU: the measured dense tensor-core rate (dds_tensor_rate) that the roofline fractions of the
tensor-core kernels are also read against."""

import ctypes

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_tensor_rate_is_plausible_and_bf16_is_faster():
    from paper_2003_02585_gb300 import dds
    tf32 = dds.tensor_rate("tf32")
    bf16 = dds.tensor_rate("bf16")
    # nominal dense rates of a GB300: 1.1 PF/s TF32, 2.25 PF/s BF16; a measured rate far outside
    # [0.2, 1.2] of them means the loop did not run as written
    assert 0.2 * 1100 < tf32 < 1.2 * 1100, tf32
    assert 0.2 * 2250 < bf16 < 1.2 * 2250, bf16
    assert bf16 > 1.5 * tf32
    # another piece type is rejected without a launch
    v = ctypes.c_double(-1.0)
    assert dds.load().dds_tensor_rate(2, ctypes.byref(v)) == 1   # DDS_EINVAL
