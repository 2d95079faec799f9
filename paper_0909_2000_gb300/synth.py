"""Seeded synthetic inputs for alignment plots.

This module generates sequences only; it holds none of the plot arithmetic.
It is the one piece of code that both the oracle side (tests, CPU baseline)
and the CUDA side (tests, bench, smoke) use, so that both sides see the same
bytes for the same seed.

Randomness comes from a counter-based SplitMix64: value k of stream s under
seed S is ``mix64(S' + (k + 1) * 0x9E3779B97F4A7C15)`` with
``S' = mix64(S ^ (s * 0xD1B54A32D192ED03))`` (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  Everything is
vectorised with numpy uint64 wrap-around arithmetic.

The paper's data sets (Table 1: Mikey, Berti, Jimmy, Henry) are not
available, so these recipes stand in for them:

* DNA: bytes 'A','C','G','T' drawn uniformly (two bits of a draw).
* Protein: 20 letters drawn uniformly by multiply-shift on 32 random bits.
* Homologous segments: a segment of x is copied into y, with substitutions to
  a different letter and single-character insertions or deletions; y keeps its
  length (the copy is truncated at the end of y).
* Lengths: log-uniform, round(exp(U(ln a, ln b))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0xD1B54A32D192ED03)

DNA = np.frombuffer(b"ACGT", dtype=np.uint8)
PROTEIN = np.frombuffer(b"ACDEFGHIKLMNPQRSTVWY", dtype=np.uint8)


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _STREAM)
    return mix64(np.array([s], dtype=np.uint64))[0]


def draws(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` uint64 values of stream ``stream``, starting at ``offset``."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(stream_key(seed, stream) + k * GOLDEN)


def uniform01(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Floats in [0, 1) from the top 53 bits."""
    return (draws(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def below(seed: int, stream: int, count: int, bound: int, offset: int = 0) -> np.ndarray:
    """Integers in [0, bound) by multiply-shift on the top 32 bits."""
    hi = draws(seed, stream, count, offset) >> np.uint64(32)
    return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def dna(seed: int, stream: int, n: int) -> np.ndarray:
    return DNA[(draws(seed, stream, n) >> np.uint64(62)).astype(np.int64)]


def protein(seed: int, stream: int, n: int) -> np.ndarray:
    return PROTEIN[below(seed, stream, n, len(PROTEIN))]


def alphabet_string(seed: int, stream: int, n: int, alphabet) -> np.ndarray:
    alphabet = np.asarray(alphabet, dtype=np.uint8)
    return alphabet[below(seed, stream, n, len(alphabet))]


def log_uniform_int(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    u = uniform01(seed, stream, count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def mutate(src: np.ndarray, seed: int, stream: int, alphabet, sub: float,
           indel: float) -> np.ndarray:
    """Copy of ``src`` with substitutions (to a different letter, rate ``sub``)
    and single-character indels (rate ``indel``, half insertions, half
    deletions).  Position p draws u[p]: u < sub substitutes, the next indel/2
    inserts a random letter before the character, the next indel/2 deletes
    it, anything else copies it."""
    alphabet = np.asarray(alphabet, dtype=np.uint8)
    sigma = len(alphabet)
    code = np.full(256, -1, dtype=np.int64)
    code[alphabet] = np.arange(sigma)
    src = np.asarray(src, dtype=np.uint8)
    L = len(src)
    u = uniform01(seed, stream, L)
    r = below(seed, stream + 1, L, max(1, sigma - 1))
    ins = below(seed, stream + 2, L, sigma)
    k = np.maximum(code[src], 0)
    subst = alphabet[(k + 1 + r) % sigma]
    is_sub = u < sub
    is_ins = (~is_sub) & (u < sub + indel / 2)
    is_del = (~is_sub) & (~is_ins) & (u < sub + indel)
    body = np.where(is_sub, subst, src)              # the character each position keeps
    lens = np.where(is_del, 0, np.where(is_ins, 2, 1))
    out = np.empty(int(lens.sum()), dtype=np.uint8)
    start = np.cumsum(lens) - lens                   # first output slot of each position
    keep = ~is_del
    # the kept character is the last slot of its position
    out[(start + lens - 1)[keep]] = body[keep]
    out[start[is_ins]] = alphabet[ins[is_ins]]
    return out


def plant(x: np.ndarray, y: np.ndarray, count: int, length: int, seed: int,
          stream: int, alphabet, sub: float, indel: float):
    """Copy ``count`` mutated segments of x into y, in place on a copy of y.

    x and y are cut into ``count`` equal slots each.  Segment k is taken from
    a random place in x slot pi(k), for a seeded permutation pi.  It goes to a
    random place in y slot k.  Returns (y, list of (x_pos, y_pos, length))."""
    y = y.copy()
    m, n = len(x), len(y)
    slot_x, slot_y = m // count, n // count
    if slot_x < length or slot_y < length:
        raise ValueError("segments do not fit")
    perm = np.argsort(draws(seed, stream, count))
    offx = below(seed, stream + 1, count, slot_x - length + 1)
    offy = below(seed, stream + 2, count, slot_y - length + 1)
    placed = []
    for k in range(count):
        xs = int(perm[k]) * slot_x + int(offx[k])
        ys = k * slot_y + int(offy[k])
        seg = mutate(x[xs:xs + length], seed, stream + 10 + 3 * k, alphabet, sub, indel)
        seg = seg[: n - ys]
        y[ys:ys + len(seg)] = seg
        placed.append((xs, ys, len(seg)))
    return y, placed


# ---------------------------------------------------------------------------
# Workloads.  Each is described by what it is and its sizes.
# ---------------------------------------------------------------------------

@dataclass
class Pair:
    x: np.ndarray
    y: np.ndarray
    w: int
    scores: tuple = (1, 0)          # (match, mismatch), gap 0
    threshold: int | None = None
    name: str = ""
    planted: list = field(default_factory=list)
    step: int = 1                   # vertical step: plot row r is x-window r * step


def dna_plot_512(seed: int = 0) -> Pair:
    """LCS plot, uniform DNA, m = n = 512, w = 16 (full 496 x 496 plot)."""
    return Pair(dna(seed, 1, 512), dna(seed, 2, 512), 16, (1, 0), None,
                "lcs_dna_512_w16")


def dna_plot_100k(seed: int = 0, m: int = 100_000, n: int = 100_000, w: int = 100,
                  segments: int = 20, seg_len: int = 2000) -> Pair:
    """LCS plot, DNA m = n = 100,000, w = 100, with 20 planted homologous
    segments of length 2000 (10% substitutions, 5% indels); dots >= 80."""
    x = dna(seed, 1, m)
    y = dna(seed, 2, n)
    y, placed = plant(x, y, segments, seg_len, seed, 100, DNA, 0.10, 0.05)
    return Pair(x, y, w, (1, 0), 80, "lcs_dna_100k_w100", placed)


def dna_plot_20k(seed: int = 0) -> Pair:
    """The 100k DNA recipe at m = n = 20,000 (4 planted segments), w = 100:
    a smaller case of the same kernel for profiler captures."""
    c = dna_plot_100k(seed, 20_000, 20_000, 100, 4, 2000)
    c.name = "lcs_dna_20k_w100"
    return c


def dna_plot_20k_w128(seed: int = 0) -> Pair:
    """The 20k DNA recipe at w = 128, a serving-mix window in full 8-bit keys
    on two threads per strip group; dots >= ceil(0.8 w) = 103."""
    c = dna_plot_100k(seed, 20_000, 20_000, 128, 4, 2000)
    c.threshold = threshold_08(128)
    c.name = "lcs_dna_20k_w128"
    return c


def dna_plot_20k_w256(seed: int = 0) -> Pair:
    """The 20k DNA recipe at w = 256, the serving mix's largest window: 16-bit
    keys and a uint16 plot (values reach 256); dots >= ceil(0.8 w) = 205."""
    c = dna_plot_100k(seed, 20_000, 20_000, 256, 4, 2000)
    c.threshold = threshold_08(256)
    c.name = "lcs_dna_20k_w256"
    return c


def dna_score_80k_step5(seed: int = 0) -> Pair:
    """The shape of the paper's largest Table 1 runs: m = n = 80,000, w = 100,
    scores (1, 0, -1/2) as {2,1,0}, vertical step 5 (DNA with 16 planted
    homologous segments of length 2000 stands in for the absent sequences)."""
    c = dna_plot_100k(seed, 80_000, 80_000, 100, 16, 2000)
    c.scores = (2, 1)
    c.threshold = None
    c.step = 5
    c.name = "score_dna_80k_w100_step5"
    return c


def protein_score_20k(seed: int = 0, m: int = 20_000, n: int = 20_000, w: int = 64) -> Pair:
    """Score plot (match 2, mismatch 1, gap 0), uniform 20-letter protein,
    m = n = 20,000, w = 64, uint16 output."""
    return Pair(protein(seed, 1, m), protein(seed, 2, n), w, (2, 1), None,
                "score_protein_20k_w64")


def batch_jobs(seed: int = 0, count: int = 4096, lo: int = 200, hi: int = 20_000,
               windows=(16, 32, 64, 128), homolog_frac: float = 0.30) -> list:
    """Many DNA pairs: m and n log-uniform over [lo, hi] (independent), w
    uniform over ``windows``, a share of pairs with one planted segment of
    length min(m, n) // 4 carrying 10% substitutions."""
    ms = log_uniform_int(seed, 1, count, lo, hi)
    ns = log_uniform_int(seed, 2, count, lo, hi)
    ws = np.asarray(windows)[below(seed, 3, count, len(windows))]
    hom = uniform01(seed, 4, count) < homolog_frac
    jobs = []
    for k in range(count):
        m, n, w = int(ms[k]), int(ns[k]), int(ws[k])
        x = dna(seed, 1000 + 4 * k, m)
        y = dna(seed, 1001 + 4 * k, n)
        placed = []
        if hom[k]:
            L = min(m, n) // 4
            if L > 0:
                y, placed = plant(x, y, 1, L, seed, 1002 + 4 * k + 100000, DNA, 0.10, 0.0)
        jobs.append(Pair(x, y, w, (1, 0), None, "batch_%d" % k, placed))
    return jobs


def threshold_08(w: int) -> int:
    """ceil(0.8 w) in integer arithmetic (26, 52, 103, 205 for w = 32..256)."""
    return -(-4 * w // 5)


def serving_requests(seed: int = 0, rate: float = 200.0, duration: float = 60.0,
                     lo: int = 1000, hi: int = 200_000, windows=(32, 64, 128, 256),
                     max_requests: int | None = None) -> list:
    """Poisson arrivals at ``rate`` per second over ``duration`` seconds of DNA
    dot-plot jobs: m, n log-uniform over [lo, hi], w uniform over
    ``windows``, threshold ceil(0.8 w).  Returns (arrival_s, Pair) tuples."""
    expect = int(rate * duration * 1.5) + 16
    gaps = -np.log1p(-uniform01(seed, 1, expect)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration]
    if max_requests is not None:
        t = t[:max_requests]
    count = len(t)
    ms = log_uniform_int(seed, 2, count, lo, hi)
    ns = log_uniform_int(seed, 3, count, lo, hi)
    ws = np.asarray(windows)[below(seed, 4, count, len(windows))]
    reqs = []
    for k in range(count):
        w = int(ws[k])
        p = Pair(dna(seed, 1000 + 2 * k, int(ms[k])), dna(seed, 1001 + 2 * k, int(ns[k])),
                 w, (1, 0), threshold_08(w), "req_%d" % k)
        reqs.append((float(t[k]), p))
    return reqs
