"""Checks that pin a plot function to facts fixed by the paper and by the
mathematics, independent of any implementation of the plot.

``pin_battery(plot_fn)`` runs every check on small seeded inputs and returns
the names of the checks that failed.  The oracle must pass all of them.
``test_oracle_mutants`` plants plausible mistakes in copies of the oracle and
requires that each one fails at least one check.

``plot_fn(x, y, w, match, mismatch)`` must return the (m-w) x (n-w) plot of
window-pair alignment scores (Section 2 of the paper).
"""
from __future__ import annotations

import itertools

import numpy as np

from paper_0909_2000_gb300 import synth


# ---------------------------------------------------------------------------
# Brute force, independent of any dynamic programme
# ---------------------------------------------------------------------------

def is_subsequence(s, t) -> bool:
    it = iter(t)
    return all(c in it for c in s)


def lcs_bruteforce(a, b) -> int:
    """Longest common subsequence by enumerating every subsequence of a."""
    a, b = list(a), list(b)
    best = 0
    for mask in range(1 << len(a)):
        k = bin(mask).count("1")
        if k <= best:
            continue
        sub = [a[p] for p in range(len(a)) if mask >> p & 1]
        if is_subsequence(sub, b):
            best = k
    return best


def alignment_bruteforce(a, b, match, mismatch, gap=0.0):
    """Best alignment score by enumerating every alignment: k aligned pairs at
    increasing positions of both strings, every other character against a
    gap (Section 2's definition of an alignment)."""
    a, b = list(a), list(b)
    best = None
    for k in range(0, min(len(a), len(b)) + 1):
        for pa in itertools.combinations(range(len(a)), k):
            for pb in itertools.combinations(range(len(b)), k):
                s = sum(match if a[p] == b[q] else mismatch for p, q in zip(pa, pb))
                s += gap * (len(a) + len(b) - 2 * k)
                if best is None or s > best:
                    best = s
    return best


def dollar_interleave(s: bytes, dollar: int = 0x24) -> bytes:
    """Section 2's transformation: a new character '$' before every character."""
    out = bytearray()
    for c in s:
        out.append(dollar)
        out.append(c)
    return bytes(out)


# ---------------------------------------------------------------------------
# The battery
# ---------------------------------------------------------------------------

def _rand(seed, stream, n, alphabet):
    return synth.alphabet_string(seed, stream, n, np.frombuffer(alphabet, dtype=np.uint8))


def pin_battery(plot_fn, quick: bool = False) -> list[str]:
    fails: list[str] = []

    def check(name, ok):
        if not ok:
            fails.append(name)

    # 1. brute force, LCS, several shapes (m != n catches transposition)
    for seed, (m, n, w, alph) in enumerate([(11, 9, 4, b"AC"), (10, 13, 5, b"ACGT"),
                                            (9, 9, 3, b"AB"), (12, 8, 6, b"ABC")]):
        x, y = _rand(seed, 1, m, alph), _rand(seed, 2, n, alph)
        p = np.asarray(plot_fn(x, y, w, 1, 0))
        want = np.array([[lcs_bruteforce(x[i:i + w], y[j:j + w]) for j in range(n - w)]
                         for i in range(m - w)], dtype=np.int64).reshape(max(0, m - w), max(0, n - w))
        check("bruteforce_lcs_%d" % seed, p.shape == want.shape and np.array_equal(p, want))

    # 2. brute force, score scheme (2, 1, 0)
    for seed, (m, n, w, alph) in enumerate([(8, 7, 3, b"AC"), (7, 9, 4, b"ACG")]):
        x, y = _rand(seed, 3, m, alph), _rand(seed, 4, n, alph)
        p = np.asarray(plot_fn(x, y, w, 2, 1))
        want = np.array([[alignment_bruteforce(x[i:i + w], y[j:j + w], 2, 1) for j in range(n - w)]
                         for i in range(m - w)], dtype=np.int64)
        check("bruteforce_score_%d" % seed, p.shape == want.shape and np.array_equal(p, want))

    # 3. the paper's reduction: T = S + w and T = LLCS of the '$'-interleaved windows
    x, y = _rand(7, 5, 8, b"ACG"), _rand(7, 6, 8, b"ACG")
    w = 3
    p = np.asarray(plot_fn(x, y, w, 2, 1))
    ok = p.shape == (5, 5)
    for i in range(min(5, p.shape[0])):
        for j in range(min(5, p.shape[1])):
            a, b = bytes(x[i:i + w]), bytes(y[j:j + w])
            s_half = alignment_bruteforce(a, b, 1.0, 0.0, -0.5)
            llcs = lcs_bruteforce(dollar_interleave(a), dollar_interleave(b))
            ok &= (p[i, j] == llcs) and abs(s_half + w - p[i, j]) < 1e-9
    check("dollar_reduction", ok)

    # 4. closed forms
    w = 5
    y = _rand(3, 7, 17, b"ACGT")
    x = np.full(14, ord("A"), dtype=np.uint8)
    cnt = np.array([np.count_nonzero(y[j:j + w] == ord("A")) for j in range(len(y) - w)])
    p = np.asarray(plot_fn(x, y, w, 1, 0))
    check("closed_constant_x_lcs", p.shape == (9, 12) and np.all(p == cnt[None, :]))
    p = np.asarray(plot_fn(x, y, w, 2, 1))
    check("closed_constant_x_score", p.shape == (9, 12) and np.all(p == (w + cnt)[None, :]))
    x2 = _rand(4, 8, 13, b"AC")
    y2 = _rand(4, 9, 11, b"GT")
    check("closed_disjoint_lcs", np.all(np.asarray(plot_fn(x2, y2, 4, 1, 0)) == 0))
    check("closed_disjoint_score", np.all(np.asarray(plot_fn(x2, y2, 4, 2, 1)) == 4))
    per = np.frombuffer(b"AC" * 10, dtype=np.uint8)
    p = np.asarray(plot_fn(per[:16], per[:15], 6, 1, 0))
    ii, jj = np.meshgrid(np.arange(10), np.arange(9), indexing="ij")
    check("closed_periodic", p.shape == (10, 9) and np.array_equal(p, np.where((ii - jj) % 2 == 0, 6, 5)))

    if quick:
        return fails

    # 5. invariants on a larger random case
    for seed, alph, w in [(5, b"ACGT", 7), (6, b"AC", 6)]:
        x, y = _rand(seed, 10, 24, alph), _rand(seed, 11, 21, alph)
        p = np.asarray(plot_fn(x, y, w, 1, 0)).astype(np.int64)
        rows, cols = len(x) - w, len(y) - w
        ok = p.shape == (rows, cols)
        if ok:
            ok &= bool(np.all((p >= 0) & (p <= w)))
            ok &= bool(np.all(np.abs(np.diff(p, axis=0)) <= 1))
            ok &= bool(np.all(np.abs(np.diff(p, axis=1)) <= 1))
            ok &= bool(np.all(np.abs(p[1:, 1:] - p[:-1, :-1]) <= 1))
            for i in range(rows):
                for j in range(cols):
                    a, b = x[i:i + w], y[j:j + w]
                    ham = int(np.count_nonzero(a == b))
                    cap = sum(min(np.count_nonzero(a == c), np.count_nonzero(b == c)) for c in set(a.tolist()))
                    ok &= ham <= p[i, j] <= cap
                    ok &= (p[i, j] == w) == bool(np.array_equal(a, b))
        check("invariants_lcs_%d" % seed, ok)
        pt = np.asarray(plot_fn(y, x, w, 1, 0))
        check("swap_symmetry_%d" % seed, pt.shape == (cols, rows) and np.array_equal(pt, p.T))
        pr = np.asarray(plot_fn(x[::-1].copy(), y[::-1].copy(), w, 1, 0))
        ok = pr.shape == p.shape
        if ok:
            # reversed window i_r holds the reversed original window rows - i_r
            ok = np.array_equal(pr[1:, 1:], p[:0:-1, :0:-1])
        check("reversal_%d" % seed, ok)
        perm = np.arange(256, dtype=np.uint8)[::-1].copy()
        pb = np.asarray(plot_fn(perm[x], perm[y], w, 1, 0))
        check("relabel_%d" % seed, np.array_equal(pb, p))
        ps = np.asarray(plot_fn(x, y, w, 2, 1)).astype(np.int64)
        ok = ps.shape == p.shape and bool(np.all((ps >= w) & (ps <= 2 * w)))
        ok = ok and bool(np.all(np.abs(np.diff(ps, axis=0)) <= 2)) and bool(np.all(np.abs(np.diff(ps, axis=1)) <= 2))
        ok = ok and bool(np.all(np.abs(ps[1:, 1:] - ps[:-1, :-1]) <= 1))
        # T = 2M + X with M <= LCS and M + X <= w; the LCS alignment alone gives 2 LCS
        ok = ok and bool(np.all((ps >= np.maximum(w, 2 * p)) & (ps <= w + p)))
        check("invariants_score_%d" % seed, ok)

    # 6. empty plots
    x = _rand(9, 1, 5, b"ACGT")
    check("empty_m_le_w", np.asarray(plot_fn(x, _rand(9, 2, 9, b"ACGT"), 5, 1, 0)).size == 0)
    check("empty_n_le_w", np.asarray(plot_fn(_rand(9, 3, 9, b"ACGT"), x, 6, 1, 0)).size == 0)
    return fails
