"""The random-gather ceiling call (mcx_gather_rate): positive finite rates, an
L2-sized buffer served at least as fast as one far above L2 for independent
loads, and argument checks."""
import math

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_gather_rate():
    import paper_1904_12759_gb300 as P

    P.load()
    small = P.gather_rate(64 << 20, dependent=False, loads=1 << 28)
    big = P.gather_rate(4 << 30, dependent=False, loads=1 << 28)
    dep = P.gather_rate(64 << 20, dependent=True, loads=1 << 27)
    assert all(math.isfinite(r) and r > 1e9 for r in (small, big, dep))
    assert small >= 0.8 * big
    for nbytes, loads in (((1 << 20) - 32, 1000), (1 << 40, 1000), (64 << 20, 0)):
        with pytest.raises(P.MCXError):
            P.gather_rate(nbytes, loads=loads)
