"""Writes the oracle regression fixtures in this folder.

Calls only ``oracle/`` and the seeded scene generators; the CUDA library is
never involved.  The paper prints no worked numerical example of its
renderer, so these fixtures pin the oracle against its own earlier output
(regression), not against the paper: they catch an unintended change of the
oracle's arithmetic.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2309_04581_gb300 import scenes as S  # noqa: E402


def write_c1_16():
    sc = S.config1(16, 16)
    res = oracle.render(sc, threads=1)
    path = os.path.join(HERE, "c1_16x16_oracle.txt")
    with open(path, "w") as f:
        f.write("# Oracle output, config 1 scene (8 Gaussian blobs, mirror cube, 4 segments,\n")
        f.write("# 128 midpoint samples per segment) at 16x16, 1 spp.  Written by make_golden.py.\n")
        f.write("# pixel r g b alpha segments first_hit_triangle first_hit_t\n")
        for i in range(res["rgba"].shape[0]):
            r, g, b, a = res["rgba"][i]
            f.write(f"{i} {r:.17g} {g:.17g} {b:.17g} {a:.17g} {res['segments'][i, 0]} "
                    f"{int(res['tri'][i, 0, 0])} {res['t'][i, 0, 0]:.17g}\n")
    return path


if __name__ == "__main__":
    print(write_c1_16())
