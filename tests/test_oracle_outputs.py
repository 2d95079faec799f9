"""The oracle's plot-derived outputs, pinned to hand-worked values (CPU only).

``oracle.dots`` (Section 1: one dot per window pair whose score passes the
threshold, listed row-major here), ``oracle.checksum`` and
``oracle.histogram`` decide every dot-list and digest comparison of the GPU
tests.  Here they are fixed by literal values worked out by hand on small
plots, and planted mistakes in copies of them (the order of the dots, the
threshold, the checksum's weights and its 64-bit wrap, the histogram's
bins) must each fail one of those checks.  The digests that the C oracles
compute without storing the plot are then tied to these functions and to a
closed form.
"""
import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

# A 3 x 4 plot worked by hand.
P = np.array([[3, 0, 7, 5],
              [1, 9, 2, 8],
              [6, 4, 9, 0]], dtype=np.int64)

# Dots >= 5 in row-major order (i, then j).
DOTS_GE5 = [(0, 2, 7), (0, 3, 5), (1, 1, 9), (1, 3, 8), (2, 0, 6), (2, 2, 9)]

# Checksum sum v * (i*2654435761 + j*40503 + 1) mod 2^64, by hand:
#   row 0 (weights 1, 40504, 81007, 121510):
#       3*1 + 7*81007 + 5*121510                          = 1,174,602
#   row 1 (weights 2654435762, 2654476265, 2654516768, 2654557271):
#       2654435762 + 9*2654476265 + 2*2654516768 + 8*2654557271
#                                                         = 53,090,213,851
#   row 2 (weights 5308871523, 5308912026, 5308952529, 5308993032):
#       6*5308871523 + 4*5308912026 + 9*5308952529        = 100,869,450,003
CHECKSUM_P = 153_960_838_456
# With the rows numbered from 10^12 on, every cell's weight grows by
# 10^12 * 2654435761, i.e. the sum by 54 (the sum of P) times that, which is
# 1.43e23: reduced mod 2^64 = 18446744073709551616,
#   153960838456 + 54 * 2654435761 * 10^12 = 143339531094153960838456
#   143339531094153960838456 mod 2^64       = 8329641430744782136
CHECKSUM_P_ROW0_1E12 = 8_329_641_430_744_782_136
# 16-bit values (nothing truncated to a byte): [[300, 1], [65535, 256]]
#   300*1 + 1*40504 + 65535*2654435762 + 256*2654476265 = 174637993627314
P16 = np.array([[300, 1], [65535, 256]], dtype=np.int64)
CHECKSUM_P16 = 174_637_993_627_314

HIST_P_10 = [2, 1, 1, 1, 1, 1, 1, 1, 1, 2]      # values 0..9 of P
HIST_P_8 = [2, 1, 1, 1, 1, 1, 1, 1]             # values 8 and 9 are not counted


def _pins(dots_fn, checksum_fn, histogram_fn):
    """Names of the failed hand-worked checks."""
    fails = []
    d = np.asarray(dots_fn(P, 5)).reshape(-1, 3)
    if [tuple(int(v) for v in r) for r in d] != DOTS_GE5:
        fails.append("dots_row_major_inclusive")
    if np.asarray(dots_fn(P, 10)).size != 0:
        fails.append("dots_none")
    if [tuple(int(v) for v in r) for r in np.asarray(dots_fn(P16, 256)).reshape(-1, 3)] != [(0, 0, 300), (1, 0, 65535), (1, 1, 256)]:
        fails.append("dots_16bit")
    if checksum_fn(P, 0) != CHECKSUM_P:
        fails.append("checksum")
    if checksum_fn(P, 10 ** 12) != CHECKSUM_P_ROW0_1E12:
        fails.append("checksum_wrap")
    if checksum_fn(P16, 0) != CHECKSUM_P16:
        fails.append("checksum_16bit")
    if list(histogram_fn(P, 10)) != HIST_P_10:
        fails.append("histogram")
    if list(histogram_fn(P, 8)) != HIST_P_8:
        fails.append("histogram_short")
    return fails


def test_oracle_outputs_against_hand_worked_values():
    assert _pins(oracle.dots, oracle.checksum, oracle.histogram) == []


# ---- planted mistakes, each in a copy of one function ----

def dots_column_major(p, thr):
    jj, ii = np.nonzero(p.T >= thr)
    return np.stack([ii, jj, p[ii, jj]], axis=1)


def dots_exclusive(p, thr):
    ii, jj = np.nonzero(p > thr)
    return np.stack([ii, jj, p[ii, jj]], axis=1)


def dots_byte_values(p, thr):
    ii, jj = np.nonzero(p >= thr)
    return np.stack([ii, jj, p[ii, jj] & 0xFF], axis=1)


def _cs(p, row0, mi, mj, one, dtype=np.uint64):
    v = np.asarray(p, dtype=dtype)
    i = (np.arange(v.shape[0], dtype=dtype) + dtype(row0))[:, None]
    j = np.arange(v.shape[1], dtype=dtype)[None, :]
    with np.errstate(over="ignore"):
        return int(np.sum(v * (i * dtype(mi) + j * dtype(mj) + dtype(one)), dtype=dtype)) % (1 << 64)


def checksum_swapped(p, row0=0):
    return _cs(p, row0, oracle.CHECKSUM_MUL_J, oracle.CHECKSUM_MUL_I, 1)


def checksum_no_one(p, row0=0):
    return _cs(p, row0, oracle.CHECKSUM_MUL_I, oracle.CHECKSUM_MUL_J, 0)


def checksum_row0_ignored(p, row0=0):
    return _cs(p, 0, oracle.CHECKSUM_MUL_I, oracle.CHECKSUM_MUL_J, 1)


def checksum_float(p, row0=0):
    v = np.asarray(p, dtype=np.float64)
    i = (np.arange(v.shape[0]) + row0)[:, None].astype(np.float64)
    j = np.arange(v.shape[1])[None, :].astype(np.float64)
    return int(np.sum(v * (i * oracle.CHECKSUM_MUL_I + j * oracle.CHECKSUM_MUL_J + 1))) % (1 << 64)


def checksum_byte_values(p, row0=0):
    return oracle.checksum(np.asarray(p) & 0xFF, row0)


def histogram_shifted(p, nbins):
    return np.bincount(np.asarray(p).ravel() + 1, minlength=nbins)[:nbins]


def histogram_clamped(p, nbins):
    return np.bincount(np.minimum(np.asarray(p).ravel(), nbins - 1), minlength=nbins)[:nbins]


MUTANTS = {
    "dots column-major": (dots_column_major, oracle.checksum, oracle.histogram),
    "dots threshold exclusive": (dots_exclusive, oracle.checksum, oracle.histogram),
    "dots value truncated to a byte": (dots_byte_values, oracle.checksum, oracle.histogram),
    "checksum multipliers swapped": (oracle.dots, checksum_swapped, oracle.histogram),
    "checksum without the +1": (oracle.dots, checksum_no_one, oracle.histogram),
    "checksum ignores row0": (oracle.dots, checksum_row0_ignored, oracle.histogram),
    "checksum in floating point": (oracle.dots, checksum_float, oracle.histogram),
    "checksum of byte values": (oracle.dots, checksum_byte_values, oracle.histogram),
    "histogram off by one": (oracle.dots, oracle.checksum, histogram_shifted),
    "histogram clamps large values": (oracle.dots, oracle.checksum, histogram_clamped),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name):
    assert _pins(*MUTANTS[name]) != [], name


# ---- the streamed digests of the C oracles ----

@pytest.mark.parametrize("w,sc,step", [(9, (1, 0), 1), (12, (2, 1), 1), (7, (3, 1), 1), (10, (1, 0), 3),
                                       (70, (1, 0), 1), (33, (2, 1), 2)])
def test_streamed_digests_equal_the_digest_of_the_stored_plot(w, sc, step):
    x, y = synth.dna(w, 1, 160), synth.dna(w, 2, 140)
    full = oracle.plot(x, y, w, *sc)[::step]
    want = (oracle.checksum(full), list(oracle.histogram(full, sc[0] * w + 1)))
    for fn in (oracle.plot_digest, oracle.blcs_digest):
        cs, hist = fn(x, y, w, sc[0], sc[1], step, sc[0] * w + 1, nthreads=3)
        assert (cs, list(hist)) == want, fn.__name__


def test_streamed_digest_closed_form():
    """Disjoint alphabets under {2,1,0}: every value is w (all mismatches),
    so the checksum is w * sum_{i<R, j<C} (i*K1 + j*K2 + 1)
    = w * (K1*C*R(R-1)/2 + K2*R*C(C-1)/2 + R*C) mod 2^64."""
    w = 11
    x = synth.alphabet_string(3, 1, 300, list(b"AC"))
    y = synth.alphabet_string(3, 2, 250, list(b"GT"))
    R, C = 300 - w, 250 - w
    K1, K2 = 2654435761, 40503
    want = w * (K1 * C * R * (R - 1) // 2 + K2 * R * C * (C - 1) // 2 + R * C) % (1 << 64)
    for fn in (oracle.plot_digest, oracle.blcs_digest):
        cs, hist = fn(x, y, w, 2, 1, 1, 2 * w + 1, nthreads=4)
        assert cs == want
        assert hist[w] == R * C and hist.sum() == R * C
