"""The oracle still reproduces its committed regression fixture."""
import os

import numpy as np

from paper_2309_04581_gb300 import scenes as S

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_c1_16x16_regression(orc):
    rows = np.loadtxt(os.path.join(HERE, "c1_16x16_oracle.txt"))
    res = orc.render(S.config1(16, 16), threads=1)
    assert np.allclose(res["rgba"], rows[:, 1:5], rtol=1e-13, atol=1e-15)
    assert np.array_equal(res["segments"][:, 0], rows[:, 5].astype(np.uint32))
    assert np.array_equal(res["tri"][:, 0, 0].astype(np.float64), rows[:, 6])
