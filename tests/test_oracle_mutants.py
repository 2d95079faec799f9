"""Plants plausible mistakes in copies of the oracle's recurrence (on the CPU)
and requires that the pin battery rejects every one of them."""
import numpy as np
import pytest

import oracle
from tests import pins


def dp(a, b, match, mismatch, mutation=None):
    """The Section 2 recurrence with an optional planted mistake."""
    a, b = list(a), list(b)
    D = [[0] * (len(b) + 1) for _ in range(len(a) + 1)]
    for k in range(1, len(a) + 1):
        if mutation == "boundary":
            D[k][0] = 1 if k == len(a) else 0
        for l in range(1, len(b) + 1):
            eq = a[k - 1] == b[l - 1]
            if mutation == "scores_swapped":
                s = mismatch if eq else match
            elif mutation == "mismatch_sign":
                s = match if eq else -mismatch
            elif mutation == "cross_index":
                eq = a[k - 1] == b[len(b) - l]
                s = match if eq else mismatch
            else:
                s = match if eq else mismatch
            diag = D[k - 1][l - 1] + (0 if mutation == "dropped_score" else s)
            if mutation == "dropped_left":
                D[k][l] = max(D[k - 1][l], diag)
            elif mutation == "gap_penalty":
                D[k][l] = max(D[k - 1][l] - 1, D[k][l - 1] - 1, diag)
            else:
                D[k][l] = max(D[k - 1][l], D[k][l - 1], diag)
    return D[len(a)][len(b)]


def mutant_plot(mutation):
    def fn(x, y, w, match, mismatch):
        x, y = np.asarray(x), np.asarray(y)
        m, n = len(x), len(y)
        rows, cols = max(0, m - w), max(0, n - w)
        if mutation == "extent":
            rows, cols = max(0, m - w + 1), max(0, n - w + 1)
        if mutation == "transposed":
            x, y = y, x
            rows, cols = cols, rows
        out = np.zeros((rows, cols), dtype=np.int64)
        for i in range(rows):
            for j in range(cols):
                a = x[i:i + w + (1 if mutation == "window_plus_one" else 0)]
                jj = j + 1 if (mutation == "y_shift" and j + 1 + w <= n) else j
                b = y[jj:jj + w]
                if mutation == "same_window":
                    b = y[i:i + w] if i + w <= n else y[j:j + w]
                out[i, j] = dp(a, b, match, mismatch,
                               mutation if mutation in ("boundary", "scores_swapped", "mismatch_sign",
                                                        "cross_index", "dropped_score", "dropped_left",
                                                        "gap_penalty") else None)
        if mutation == "transposed":
            out = out.T if out.shape != (rows, cols) else out
        return out
    return fn


MUTATIONS = ["extent", "transposed", "window_plus_one", "y_shift", "same_window", "boundary",
             "scores_swapped", "mismatch_sign", "cross_index", "dropped_score", "dropped_left",
             "gap_penalty"]


def test_unmutated_copy_passes():
    assert pins.pin_battery(mutant_plot(None)) == []


@pytest.mark.parametrize("mutation", MUTATIONS)
def test_mutant_is_caught(mutation):
    fails = pins.pin_battery(mutant_plot(mutation), quick=True)
    if not fails:
        fails = pins.pin_battery(mutant_plot(mutation))
    assert fails, "planted mistake %r passed every pin" % mutation
