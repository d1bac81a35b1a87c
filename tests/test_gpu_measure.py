"""GPU: the measurement utilities behind the popcount and tensor-core kernels' rooflines."""
import pytest

pytestmark = pytest.mark.gpu


def test_popc_rate_is_a_plausible_pipe_rate():
    """md_popc_rate reports popc lane-operations per SM per clock: a power-of-two pipe width of
    at least 8 lanes and at most the 128 lanes an SM issues per clock; two calls agree."""
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding as B
    a = B.md_popc_rate()
    b = B.md_popc_rate()
    assert 8 <= a <= 128
    assert abs(a - b) / a < 0.05


def test_mma_rate_is_a_plausible_pipe_rate():
    """md_mma_rate reports dense e4m3 flops per SM per clock.  One M = 128, N = 256, K = 32 MMA
    is 2 * 128 * 256 * 32 flops, and the tensor pipe takes at least 64 and at most 1024 cycles
    for it, so the rate lies in [2048, 32768]; two calls agree."""
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding as B
    a = B.md_mma_rate()
    b = B.md_mma_rate()
    assert 2048 <= a <= 32768
    assert abs(a - b) / a < 0.05
