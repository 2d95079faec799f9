"""Writes the stored expected values under tests/golden/.

It calls only the oracle (and the seeded input generators); nothing here
comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_0909_2000_gb300 import synth  # noqa: E402


def main():
    c = synth.dna_plot_512(0)
    p = oracle.plot(c.x, c.y, c.w)
    with open(os.path.join(HERE, "lcs_dna_512_w16.txt"), "w") as f:
        f.write("# LCS plot of uniform DNA, m = n = 512, w = 16, seed 0 (plot of Section 2,\n")
        f.write("# values by the oracle's window-pair dynamic programme).\n")
        f.write("shape=%dx%d\n" % p.shape)
        f.write("checksum=%d\n" % oracle.checksum(p))
        f.write("histogram=%s\n" % ",".join(str(v) for v in oracle.histogram(p, c.w + 1)))
        f.write("first_row=%s\n" % ",".join(str(v) for v in p[0, :32]))


if __name__ == "__main__":
    main()
