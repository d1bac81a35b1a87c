"""GPU: the measurement utility behind the popcount kernels' roofline."""
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
