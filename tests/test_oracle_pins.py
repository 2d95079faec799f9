"""The oracle against facts the paper and the mathematics fix (CPU only)."""
import os

import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth
from tests import pins

HERE = os.path.dirname(os.path.abspath(__file__))


def c_plot(x, y, w, match, mismatch):
    return oracle.plot(x, y, w, match, mismatch, nthreads=3)


def py_plot(x, y, w, match, mismatch):
    return oracle.plot_py(x, y, w, match, mismatch)


def test_battery_c_oracle():
    assert pins.pin_battery(c_plot) == []


def test_battery_python_oracle():
    assert pins.pin_battery(py_plot) == []


def test_c_and_python_oracles_agree():
    for seed, (m, n, w, sc) in enumerate([(30, 27, 7, (1, 0)), (25, 31, 9, (2, 1)), (40, 12, 11, (1, 0))]):
        x = synth.dna(seed, 1, m)
        y = synth.dna(seed, 2, n)
        assert np.array_equal(c_plot(x, y, w, *sc), py_plot(x, y, w, *sc))


def test_thread_count_does_not_matter():
    x, y = synth.protein(3, 1, 90), synth.protein(3, 2, 70)
    a = oracle.plot(x, y, 13, 2, 1, nthreads=1)
    b = oracle.plot(x, y, 13, 2, 1, nthreads=7)
    assert np.array_equal(a, b)


def test_samples_match_full_plot():
    x, y = synth.dna(4, 1, 120), synth.dna(4, 2, 101)
    full = oracle.plot(x, y, 17)
    ii = synth.below(4, 3, 500, full.shape[0])
    jj = synth.below(4, 4, 500, full.shape[1])
    assert np.array_equal(oracle.samples(x, y, 17, ii, jj), full[ii, jj])
    with pytest.raises(ValueError):
        oracle.samples(x, y, 17, [full.shape[0]], [0])


def test_all_byte_values_are_symbols():
    # equality is byte equality: 0x00 and 0xFF are ordinary characters
    x = np.arange(256, dtype=np.uint8)
    y = np.arange(256, dtype=np.uint8)[::-1].copy()
    p = oracle.plot(np.concatenate([x, x]), np.concatenate([x, y]), 8)
    assert p[0, 0] == 8 and p[3, 3] == 8          # identical windows
    assert p[0, 300] == 1 or p[0, 300] == 0


def test_dollar_golden():
    # Section 2 prints the example abab -> $a$b$a$b
    with open(os.path.join(HERE, "golden", "dollar_interleave.txt")) as f:
        lines = [l.split("#")[0].strip() for l in f if l.split("#")[0].strip()]
    src, dst = lines[0].split()
    assert pins.dollar_interleave(src.encode()).decode() == dst


def test_plot_512_golden():
    """The 496 x 496 LCS plot of uniform DNA (m = n = 512, w = 16, seed 0),
    against the checksum and histogram stored by tests/golden/make_golden.py."""
    c = synth.dna_plot_512(0)
    p = oracle.plot(c.x, c.y, c.w)
    gold = dict(l.split("=", 1) for l in open(os.path.join(HERE, "golden", "lcs_dna_512_w16.txt")).read().split()
                if "=" in l)
    assert p.shape == (496, 496)
    assert oracle.checksum(p) == int(gold["checksum"])
    assert oracle.histogram(p, c.w + 1).tolist() == [int(v) for v in gold["histogram"].split(",")]


def test_chvatal_sankoff_sanity():
    # not a pin: the mean LCS fraction of random DNA windows of length 64 sits
    # a little below the sigma = 4 Chvatal-Sankoff constant (about 0.654)
    x, y = synth.dna(11, 1, 400), synth.dna(11, 2, 400)
    p = oracle.plot(x, y, 64)
    assert 0.55 < p.mean() / 64 < 0.66


def test_checksum_bands_add_up():
    x, y = synth.dna(12, 1, 60), synth.dna(12, 2, 50)
    p = oracle.plot(x, y, 9)
    total = oracle.checksum(p)
    parts = (oracle.checksum(p[:20], 0) + oracle.checksum(p[20:], 20)) % (1 << 64)
    assert total == parts


@pytest.mark.parametrize("nu,mu", [(2, 1), (3, 1), (3, 2), (4, 1), (4, 2), (4, 3), (5, 2), (6, 1), (7, 3),
                                   (8, 5)])
def test_blow_up_reduction_small_rational_scores(nu, mu):
    """Section 2: small rational scores reduce to LCS by blowing the strings
    up.  Reading: every character becomes mu '$' then nu - mu copies of
    itself.  Checked here by brute force (subsequence enumeration on the
    blown-up windows against alignment enumeration with scores nu, mu, 0),
    then the oracle's weighted recurrence against both."""
    def blow(s):
        out = bytearray()
        for c in s:
            out += bytes([0x24]) * mu + bytes([c]) * (nu - mu)
        return bytes(out)
    for t in range(12):
        a = synth.alphabet_string(t, 1 + 10 * nu + mu, 1 + t % 3, np.frombuffer(b"ACG", np.uint8)).tobytes()
        b = synth.alphabet_string(t, 2 + 10 * nu + mu, 1 + (t * 5) % 3, np.frombuffer(b"ACG", np.uint8)).tobytes()
        brute_align = pins.alignment_bruteforce(a, b, nu, mu)
        if len(a) * nu <= 9:
            assert pins.lcs_bruteforce(blow(a), blow(b)) == brute_align
        assert oracle.pair_score(a, b, nu, mu) == brute_align
        assert oracle.pair_score(blow(a), blow(b), 1, 0) == brute_align


# ---- the bit-parallel second reference (large-plot digests) ----

def blcs_plot(x, y, w, match, mismatch):
    return oracle.blcs_plot(x, y, w, match, mismatch, nthreads=3)


def test_battery_bit_parallel_reference():
    assert pins.pin_battery(blcs_plot) == []


@pytest.mark.parametrize("seed", range(6))
def test_bit_parallel_reference_equals_the_dynamic_programme(seed):
    """Random shapes across the word boundaries of the bit-parallel method
    (blown-up windows of 63, 64, 65, 128, 129 ... characters), all byte
    values, LCS and {nu, mu, 0}, with and without a vertical step."""
    rng = synth.below(seed, 1, 8, 1 << 30)
    alph = [b"AC", b"ACGT", bytes(range(256)), b"ACDEFGHIKLMNPQRSTVWY"][seed % 4]
    cases = [(1, 0, 63), (1, 0, 64), (1, 0, 65), (1, 0, 128), (1, 0, 129), (2, 1, 32), (2, 1, 33),
             (2, 1, 64), (3, 2, 43), (4, 1, 16), (4, 3, 33), (1, 0, 300), (5, 2, 20), (8, 3, 17)]
    for k, (nu, mu, w) in enumerate(cases):
        m = w + 1 + int(rng[k % 8]) % 60
        n = w + 1 + int(rng[(k + 3) % 8]) % 70
        x = _rand_alpha(seed * 100 + k, 1, m, alph)
        y = _rand_alpha(seed * 100 + k, 2, n, alph)
        step = 1 + k % 3
        want = oracle.plot(x, y, w, nu, mu)[::step]
        got = oracle.blcs_plot(x, y, w, nu, mu, step)
        assert got.shape == want.shape and np.array_equal(got, want), (nu, mu, w, step)


def _rand_alpha(seed, stream, n, alph):
    return synth.alphabet_string(seed, stream, n, np.frombuffer(alph, dtype=np.uint8))
