"""The method as the kernels implement it, restated as a slow scalar model
and checked against the oracle on the CPU (no GPU).

The paper's Algorithm 1 figure is lost, so the CUDA comb rests on readings
of Sections 2 and 3.  This test pins those readings, not the kernels:
* the cell rule: seaweeds keyed by start column (larger = newer, the left
  boundary's seaweeds oldest), and the bottom output is h when the cell
  matches or h >= v, else v (Section 2);
* the window count: WLCS of the window ending at column J is w - d(J), with
  d(J) the seaweeds that started inside the window and have left at the
  bottom by J (Theorem 3.1).  d is kept incrementally: + a valid exit, - the
  exit of the start that leaves the window;
* fresh-start chunks: a comb started at column c0 with w - 1 warm-up
  columns is exact for every window starting at c0 or later;
* saturating renormalisation (Proposition 3.4): every P columns all keys
  drop by P and saturate at 0, which maps keys monotonically;
* score mode: {nu, mu, 0} as the LCS of strings where every character
  becomes mu '$' then nu - mu copies of itself, keys per character (unit),
  value nu * w - d (Section 2, Definition 3.2).
The model shares nothing with the CUDA path; the oracle is the plain DP.
"""
import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

DOLLAR = -1   # the '$' symbol: equal only to itself, never to a character


def blow_up(s, nu, mu):
    """Every character becomes mu '$' followed by nu - mu copies of itself."""
    out = []
    for c in s:
        out += [DOLLAR] * mu + [int(c)] * (nu - mu)
    return out


def model_strip(xs, ys, w, nu, mu, c0, c1, period=None, rule=None):
    """Values of plot row (x-window xs, len w) for plot columns [c0, c1):
    a fresh comb of the units c0 .. c1 + w - 2 of y (w - 1 warm-up units).
    One unit = nu physical columns (one y character); rows = the blown-up
    x-window.  Keys are per unit: the unit combed t-th gets key w + t, less
    the drops of the renormalisation every `period` units.  rule: the cell's
    swap decision (match, h, v) -> bool."""
    rule = rule or (lambda match, h, v: match or h >= v)
    rows = blow_up(xs, nu, mu)
    h = [0] * len(rows)               # left seaweeds: key 0, older than all
    kc, since = w, 0
    d = 0
    flags = {}                        # start unit -> exits that left validly
    vals = []
    for t, u in enumerate(range(c0, c1 + w - 1)):
        if t > 0:
            kc += 1
            since += 1
            if period is not None and since == period:
                h = [max(0, k - period) for k in h]
                kc -= period
                since = 0
        cols = blow_up([ys[u]], nu, mu)
        d -= flags.pop(t - w, 0)      # the start unit t - w leaves the window
        for c in cols:
            v = kc
            for k, r in enumerate(rows):
                match = (r == c)
                if rule(match, h[k], v):
                    h[k], v = v, h[k]
            age = kc - v              # units since the exiting seaweed started
            if age < w:
                d += 1
                flags[t - age] = flags.get(t - age, 0) + 1
        if t >= w - 1:
            vals.append(nu * w - d)
    assert len(vals) == c1 - c0
    return vals


def model_plot(x, y, w, nu=1, mu=0, chunk=None, period=None, rule=None):
    """The whole plot from the model, column chunks combed independently."""
    rows, cols = max(0, len(x) - w), max(0, len(y) - w)
    out = np.zeros((rows, cols), dtype=np.int64)
    chunk = chunk or max(cols, 1)
    for i in range(rows):
        for c0 in range(0, cols, chunk):
            c1 = min(cols, c0 + chunk)
            out[i, c0:c1] = model_strip(x[i:i + w], y, w, nu, mu, c0, c1, period, rule)
    return out


CASES = [
    # (seed, m, n, w, alphabet)
    (1, 30, 34, 1, b"AC"),
    (2, 33, 40, 3, b"ACGT"),
    (3, 40, 37, 5, b"AC"),
    (4, 36, 45, 8, b"ACGT"),
    (5, 28, 50, 12, b"AB"),
    (6, 45, 30, 9, bytes(range(256))),
]


@pytest.mark.parametrize("seed,m,n,w,alph", CASES)
def test_lcs_model_equals_the_oracle(seed, m, n, w, alph):
    """One comb per plot row, no renormalisation, one chunk."""
    a = np.frombuffer(alph, np.uint8)
    x = synth.alphabet_string(seed, 1, m, a)
    y = synth.alphabet_string(seed, 2, n, a)
    assert np.array_equal(model_plot(x, y, w), oracle.plot(x, y, w))


@pytest.mark.parametrize("chunk,period", [(1, None), (3, None), (7, 1), (5, 2), (None, 3)])
def test_chunks_and_renormalisation_are_exact(chunk, period):
    """Fresh-start chunks with w - 1 warm-up columns, and keys that drop and
    saturate every `period` columns, give the same plot."""
    x = synth.dna(7, 1, 34)
    y, _ = synth.plant(x, synth.dna(7, 2, 42), 1, 14, 7, 3, synth.DNA, 0.1, 0.05)
    for w in (4, 9):
        assert np.array_equal(model_plot(x, y, w, chunk=chunk, period=period),
                              oracle.plot(x, y, w)), (w, chunk, period)


@pytest.mark.parametrize("nu,mu", [(2, 1), (3, 1), (3, 2), (4, 3)])
def test_score_model_equals_the_oracle(nu, mu):
    """{nu, mu, 0} through the blown-up strings, keys per character,
    value nu * w - d; with chunks and renormalisation as well."""
    x = synth.alphabet_string(8, nu, 22, np.frombuffer(b"ACGT", np.uint8))
    y = synth.alphabet_string(8, 10 + mu, 26, np.frombuffer(b"ACGT", np.uint8))
    for w, chunk, period in ((3, None, None), (5, 4, 2)):
        assert np.array_equal(model_plot(x, y, w, nu, mu, chunk, period),
                              oracle.plot(x, y, w, nu, mu)), (nu, mu, w, chunk, period)


def test_plausible_misreadings_fail():
    """Each of these wrong readings of the rule differs from the oracle, so
    the model above pins the readings it states."""
    x = synth.dna(9, 1, 30)
    y, _ = synth.plant(x, synth.dna(9, 2, 36), 1, 12, 9, 3, synth.DNA, 0.1, 0.05)
    want = oracle.plot(x, y, 6)
    wrong_rules = {
        "match treated as mismatch": lambda match, h, v: h >= v,
        "mismatch swaps when h < v": lambda match, h, v: match or h < v,
        "match never swaps": lambda match, h, v: (not match) and h >= v,
    }
    for name, rule in wrong_rules.items():
        assert not np.array_equal(model_plot(x, y, 6, rule=rule), want), name
