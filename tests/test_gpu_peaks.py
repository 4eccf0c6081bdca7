"""The library's own roofline measurements on the GPU: CUDA-core FMA throughput and the rate of
bulk asynchronous global -> shared copies."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2605_01774_gb300 import elbm
    elbm.lib()
    return elbm


def test_fma_peak(E):
    f64, f32 = E.elbm_fma_peak("f64"), E.elbm_fma_peak("f32")
    assert 1e11 < f64 < f32 < 1e15


def test_bulk_copy_rate(E):
    """Large copies from several blocks per SM stream at DRAM speed; with small copies and one
    issuing warp per SM the issue rate of that warp bounds the bytes (far below DRAM speed)."""
    big, nbig = E.elbm_bulk_copy_rate(8192, 2)
    small, nsmall = E.elbm_bulk_copy_rate(512, 1)
    assert 1e12 < big < 2e13
    assert abs(nbig * 8192 - big) <= 1e-9 * big and abs(nsmall * 512 - small) <= 1e-9 * small
    assert small < 0.8 * big
