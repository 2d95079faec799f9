"""Writes the stored expected values under tests/golden/.

It calls only the oracle (and the seeded input generators); nothing here
comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

With no names it writes every file.  The small 512 x 512 plot is the
dynamic programme's full plot.  The large plots are digests (checksum and
value histogram, as defined in oracle/blcs.c) of the whole plot:
* where the dynamic programme finishes on the host in minutes (the two
  20k x 20k plots of windows 100 and 64), both the dynamic programme and the
  bit-parallel reference compute the digest, and the script stops unless
  they agree;
* the larger ones (the 100k x 100k plot, w = 256, the 80k Table 1 shape)
  come from the bit-parallel reference alone, which the CPU tests check
  against the dynamic programme and the brute-force pins.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_0909_2000_gb300 import synth  # noqa: E402


def small_512():
    c = synth.dna_plot_512(0)
    p = oracle.plot(c.x, c.y, c.w)
    with open(os.path.join(HERE, "lcs_dna_512_w16.txt"), "w") as f:
        f.write("# LCS plot of uniform DNA, m = n = 512, w = 16, seed 0 (plot of Section 2,\n")
        f.write("# values by the oracle's window-pair dynamic programme).\n")
        f.write("shape=%dx%d\n" % p.shape)
        f.write("checksum=%d\n" % oracle.checksum(p))
        f.write("histogram=%s\n" % ",".join(str(v) for v in oracle.histogram(p, c.w + 1)))
        f.write("first_row=%s\n" % ",".join(str(v) for v in p[0, :32]))


# name -> (generator, also by the dynamic programme)
LARGE = {
    "lcs_dna_20k_w100": (synth.dna_plot_20k, True),
    "score_protein_20k_w64": (synth.protein_score_20k, True),
    "lcs_dna_20k_w256": (synth.dna_plot_20k_w256, False),
    "lcs_dna_100k_w100": (synth.dna_plot_100k, False),
    "score_dna_80k_w100_step5": (synth.dna_score_80k_step5, False),
}


def large(name):
    gen, with_dp = LARGE[name]
    c = gen(0)
    match, mismatch = c.scores
    nbins = match * c.w + 1
    rows, cols = oracle.step_shape(len(c.x), len(c.y), c.w, c.step)
    t = time.time()
    cs, hist = oracle.blcs_digest(c.x, c.y, c.w, match, mismatch, c.step, nbins)
    methods = ["bit-parallel LCS (oracle.blcs_digest) %.0f s" % (time.time() - t)]
    if with_dp:
        t = time.time()
        cs2, hist2 = oracle.plot_digest(c.x, c.y, c.w, match, mismatch, c.step, nbins)
        if cs2 != cs or list(hist2) != list(hist):
            raise SystemExit("%s: the dynamic programme and the bit-parallel reference disagree" % name)
        methods.append("dynamic programme (oracle.plot_digest) %.0f s, equal" % (time.time() - t))
    assert int(sum(hist)) == rows * cols
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write("# Digest of the whole plot of the seeded workload %s (seed 0):\n" % name)
        f.write("# m = %d, n = %d, w = %d, scores {%d,%d,0}, vertical step %d.\n"
                % (len(c.x), len(c.y), c.w, match, mismatch, c.step))
        f.write("# checksum = sum of P[r][j] * (r*2654435761 + j*40503 + 1) mod 2^64;\n")
        f.write("# histogram[v] = cells with value v.  Written by tests/golden/make_golden.py\n")
        f.write("# from the oracle only: %s.\n" % "; ".join(methods))
        f.write("shape=%dx%d\n" % (rows, cols))
        f.write("checksum=%d\n" % cs)
        f.write("histogram=%s\n" % ",".join(str(int(v)) for v in hist))


def main(names):
    names = names or ["lcs_dna_512_w16"] + list(LARGE)
    for name in names:
        t = time.time()
        if name == "lcs_dna_512_w16":
            small_512()
        else:
            large(name)
        print("%s: %.0f s" % (name, time.time() - t), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
