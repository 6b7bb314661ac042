"""Host-side feature encoding of the cost model (no GPU: pure arithmetic in
the library)."""

import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def cm():
    from paper_1710_01839_gb300 import build
    build.build()
    from paper_1710_01839_gb300 import costmodel
    return costmodel


def test_feature_vector(cm):
    assert cm.num_features() == 16
    f = cm.features("dd", 1024, 512, 256, "block", 32)
    assert f[0] == 10 and f[1] == 9 and f[2] == 8 and f[3] == 27
    assert list(f[4:7]) == [1, 0, 0]                         # DD one-hot
    assert abs(f[7] - math.log2(106)) < 1e-5                 # 106-bit significand
    assert f[8] == 5                                         # log2 tile
    assert list(f[9:12]) == [0, 1, 0] and f[12] == 0         # block, depth 0
    ctas = (1024 // 32) * (256 // 32)
    assert abs(f[13] - math.log2(ctas)) < 1e-5
    assert abs(f[14] - math.log2(math.ceil(ctas / 152))) < 1e-5
    g = cm.features("mp", 64, 64, 64, "strassen", 16, depth=2, prec_bits=256)
    assert list(g[4:7]) == [0, 0, 1] and g[7] == 8 and g[12] == 2 and g[11] == 1
    # Strassen multiplies the CTA count by 7^depth of (m/2^d x n/2^d) tiles
    assert abs(g[13] - math.log2(49 * 1)) < 1e-5
    q = cm.features("qd", 100, 100, 100, "simple", 16)
    assert list(q[4:7]) == [0, 1, 0] and q[9] == 1
    assert np.all(np.isfinite(q))
