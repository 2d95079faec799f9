"""CUDA path against the oracle, element by element (needs a GPU).

Every call goes through the C ABI (libalnplot.so) via the ctypes binding."""
import math

import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def gpu_plot(ap, x, y, w, scores=(1, 0, 0), out_dtype=None):
    p = ap.alignment_plot(dev(x), dev(y), w, scores, out_dtype=out_dtype)
    torch.cuda.synchronize()
    return p.cpu().numpy().astype(np.int64)


def test_plot_512_matches_oracle_and_golden(cuda_lib):
    ap = cuda_lib
    c = synth.dna_plot_512(0)
    g = gpu_plot(ap, c.x, c.y, c.w)
    o = oracle.plot(c.x, c.y, c.w)
    assert g.shape == (496, 496)
    assert np.array_equal(g, o)


CASES = [
    # (m, n, w, alphabet, scores)
    (40, 37, 1, b"AC", (1, 0, 0)),
    (70, 333, 5, b"ACGT", (1, 0, 0)),
    (300, 301, 16, b"ACGT", (1, 0, 0)),
    (257, 1000, 31, b"AB", (1, 0, 0)),
    (700, 650, 100, b"ACGT", (1, 0, 0)),
    (300, 999, 117, b"ACGT", (1, 0, 0)),
    (400, 420, 120, b"ACGTN", (1, 0, 0)),
    (200, 900, 121, b"ACGT", (1, 0, 0)),
    (300, 500, 128, b"ACGT", (1, 0, 0)),
    (400, 700, 200, b"AC", (1, 0, 0)),
    (600, 600, 256, b"ACGT", (1, 0, 0)),
    (500, 620, 254, b"AC", (1, 0, 0)),
    (430, 700, 129, b"ACGT", (1, 0, 0)),
    (380, 450, 173, bytes(range(256)), (1, 0, 0)),
    (40, 45, 3, b"AC", (2, 1, 0)),
    (190, 211, 16, b"ACDEFGHIKLMNPQRSTVWY", (2, 1, 0)),
    (300, 333, 64, b"ACDEFGHIKLMNPQRSTVWY", (2, 1, 0)),
    (250, 270, 63, b"ACGT", (2, 1, 0)),
    (300, 310, 65, b"ACGT", (2, 1, 0)),
    (300, 330, 99, b"ACGT", (2, 1, 0)),
    (400, 401, 120, b"ACGT", (2, 1, 0)),
    (420, 430, 121, b"ACGT", (2, 1, 0)),
    (600, 640, 200, b"AC", (2, 1, 0)),
    (600, 620, 254, b"ACGT", (2, 1, 0)),
    (620, 640, 255, b"ACGT", (2, 1, 0)),
    # 16-bit lanes (min/max cells) on 4 threads of up to 96 rows: 256 < w <= 384,
    # then 8 threads
    (600, 620, 257, b"ACGT", (1, 0, 0)),
    (700, 760, 300, b"ACGT", (1, 0, 0)),
    (640, 700, 384, b"AC", (1, 0, 0)),
    (600, 640, 480, b"ACGT", (1, 0, 0)),
    (620, 600, 481, b"ACGT", (1, 0, 0)),
    (560, 700, 299, bytes(range(256)), (1, 0, 0)),
    # the largest windows built: LCS w = 512 (16-bit lanes, 8 threads of 64
    # rows), {2,1,0} w = 256 (8 threads of 32 pairs)
    (700, 680, 512, b"ACGT", (1, 0, 0)),
    (690, 700, 511, b"AC", (1, 0, 0)),
    (560, 600, 256, b"ACGT", (2, 1, 0)),
]


@pytest.mark.parametrize("m,n,w,alph,scores", CASES)
def test_random_shapes(cuda_lib, m, n, w, alph, scores):
    ap = cuda_lib
    seed = m * 7 + n * 3 + w
    x = synth.alphabet_string(seed, 1, m, np.frombuffer(alph, np.uint8))
    y = synth.alphabet_string(seed, 2, n, np.frombuffer(alph, np.uint8))
    vmax = 2 * w if scores[0] == 2 else w
    g = gpu_plot(ap, x, y, w, scores, torch.uint8 if vmax <= 255 else torch.int16)
    o = oracle.plot(x, y, w, scores[0], scores[1])
    assert g.shape == o.shape
    bad = np.argwhere(g != o)
    assert len(bad) == 0, "first mismatches %s: gpu %s oracle %s" % (
        bad[:4].tolist(), g[tuple(bad[:4].T)].tolist(), o[tuple(bad[:4].T)].tolist())


BLOWUP_CASES = [
    (120, 130, 5, (3, 1, 0)), (200, 170, 17, (3, 2, 0)), (300, 260, 32, (4, 1, 0)),
    (150, 222, 24, (4, 2, 0)), (190, 140, 9, (4, 3, 0)), (260, 300, 33, (3, 1, 0)),
    (300, 330, 70, (4, 3, 0)), (420, 400, 128, (3, 2, 0)), (350, 300, 100, (4, 1, 0)),
    # nu = 5..8: one kernel per nu and row count, the '$' count read at run
    # time; windows up to the largest built (192, 160, 128, 128)
    (150, 140, 7, (5, 1, 0)), (260, 240, 40, (5, 2, 0)), (300, 320, 96, (5, 3, 0)),
    (380, 400, 192, (5, 4, 0)), (200, 230, 33, (6, 1, 0)), (330, 300, 160, (6, 5, 0)),
    (210, 190, 20, (7, 2, 0)), (260, 280, 64, (7, 4, 0)), (320, 300, 128, (7, 6, 0)),
    (180, 200, 12, (8, 1, 0)), (300, 280, 100, (8, 5, 0)), (330, 340, 128, (8, 7, 0)),
    (260, 250, 50, (10, 4, 0)),
]


@pytest.mark.parametrize("m,n,w,scores", BLOWUP_CASES)
def test_blown_up_score_schemes(cuda_lib, m, n, w, scores):
    ap = cuda_lib
    seed = m + 3 * n + w + 7 * scores[0] + scores[1]
    x = synth.protein(seed, 1, m)
    y, _ = synth.plant(x, synth.protein(seed, 2, n), 1, min(m, n) // 3, seed, 5, synth.PROTEIN, 0.1, 0.05)
    o = oracle.plot(x, y, w, scores[0], scores[1])
    g = gpu_plot(ap, x, y, w, scores, torch.int16)
    assert g.shape == o.shape and np.array_equal(g, o), np.argwhere(g != o)[:4].tolist()


# Schemes with a common factor g: the reduced scheme is combed and the plot
# scaled by g as it is written; and the reduced blow-ups {3,x,0}, {4,x,0} above
# w = 128 (16-bit lanes, up to 32 units per thread).
SCALED_CASES = [
    (300, 280, 40, (2, 0, 0)), (260, 300, 100, (3, 0, 0)), (300, 330, 50, (4, 2, 0)),
    (320, 300, 60, (6, 3, 0)), (400, 420, 40, (6, 2, 0)), (500, 520, 200, (3, 1, 0)),
    (560, 600, 256, (4, 3, 0)), (420, 440, 150, (8, 6, 0)), (200, 210, 20, (4, 2, 0)),
    (300, 310, 120, (2, 0, 0)), (450, 470, 300, (2, 0, 0)), (330, 300, 90, (9, 3, 0)),
]


@pytest.mark.parametrize("m,n,w,scores", SCALED_CASES)
def test_scaled_and_wide_score_schemes(cuda_lib, m, n, w, scores):
    ap = cuda_lib
    seed = m + 5 * n + w + 11 * scores[0] + scores[1]
    x = synth.dna(seed, 1, m)
    y, _ = synth.plant(x, synth.dna(seed, 2, n), 1, min(m, n) // 3, seed, 5, synth.DNA, 0.1, 0.05)
    o = oracle.plot(x, y, w, scores[0], scores[1])
    for dt in ((torch.uint8, torch.int16) if scores[0] * w <= 255 else (torch.int16,)):
        g = gpu_plot(ap, x, y, w, scores, dt) & 0xFFFF
        assert g.shape == o.shape and np.array_equal(g, o), (dt, np.argwhere(g != o)[:4].tolist())
    # dots of the scaled plot: thresholds apply to the scaled values
    thr = int(o.max()) - scores[0]
    dots, count = ap.alignment_dots(dev(x), dev(y), w, thr, scores)
    want = oracle.dots(o, thr)
    assert count == len(want) and np.array_equal(ap.dots_to_numpy(dots, count), want)


# Every lane format at windows it shares with the others (ap_set_lane_bits):
# 8-bit full keys, 10-bit lanes and 16-bit lanes on 2, 4 and 8 threads, DNA
# (table paths) and 20 letters (general paths).
LANE_CASES = [(bits, g, w, alph) for bits, g, w in
              [(10, 4, 121), (10, 4, 128), (10, 4, 129), (10, 4, 200), (10, 4, 256), (10, 8, 250),
               (16, 2, 126), (16, 4, 200), (16, 8, 254), (8, 2, 127), (8, 4, 201),
               (10, 4, 300), (10, 8, 480), (16, 8, 384)]
              for alph in (b"ACGT", b"ACDEFGHIKLMNPQRSTVWY")]


@pytest.mark.parametrize("bits,g,w,alph", LANE_CASES)
def test_lane_formats_at_shared_windows(cuda_lib, bits, g, w, alph):
    ap = cuda_lib
    seed = bits * 1000 + g * 100 + w
    x = synth.alphabet_string(seed, 1, w + 230, np.frombuffer(alph, np.uint8))
    y = synth.alphabet_string(seed, 2, w + 310, np.frombuffer(alph, np.uint8))
    if alph == b"ACGT":
        y, _ = synth.plant(x, y, 1, 150, seed, 3, synth.DNA, 0.1, 0.05)
    o = oracle.plot(x, y, w)
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        pl = ap.plot_plan(len(x), len(y), w)
        assert pl["lane_bits"] == bits and pl["lanes_per_strip"] == g, pl
        got = gpu_plot(ap, x, y, w, (1, 0, 0), torch.int16) & 0xFFFF
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    assert got.shape == o.shape and np.array_equal(got, o), np.argwhere(got != o)[:4].tolist()


# Match tables shared by the threads of a strip group, on DNA (four letters):
# windows whose row split must be rounded up (plan "tables" 3) in full 8-bit
# keys on 2 and 4 threads and 16-bit lanes on 2 and 8, and 7-bit keys on 2
# and 4 threads (requested layouts; one thread is their default).  In 8-bit
# lanes the padding fold spans 0 (w = 128), up to 4 (126, 133, 207, 254, 100,
# 63, 58, 21) or 8 rows (20 on 2 threads, 10 on 4), by the most padding rows
# one thread of the group holds.
SPLIT_CASES = [(0, 0, 126, 3), (0, 0, 133, 3), (0, 0, 207, 3), (8, 0, 254, 3), (0, 0, 505, 3),
               (8, 2, 100, 2), (8, 2, 63, 3), (8, 4, 58, 3), (8, 4, 21, 3), (16, 2, 127, 3),
               (0, 0, 128, 2), (8, 2, 20, 2), (8, 4, 10, 2)]


@pytest.mark.parametrize("bits,g,w,mode", SPLIT_CASES)
def test_shared_tables_row_splits(cuda_lib, bits, g, w, mode):
    ap = cuda_lib
    seed = 7000 + bits * 100 + g * 10 + w
    x = synth.alphabet_string(seed, 1, w + 260, synth.DNA)
    y = synth.alphabet_string(seed, 2, w + 333, synth.DNA)
    y, _ = synth.plant(x, y, 1, 150, seed, 3, synth.DNA, 0.1, 0.05)
    o = oracle.plot(x, y, w)
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        pl = ap.plot_plan(len(x), len(y), w)
        assert pl["tables"] == mode and pl["lanes_per_strip"] > 1, pl
        got = gpu_plot(ap, x, y, w, (1, 0, 0), torch.int16) & 0xFFFF
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    assert got.shape == o.shape and np.array_equal(got, o), np.argwhere(got != o)[:4].tolist()


@pytest.mark.parametrize("w", [241, 250, 255])
def test_16bit_lanes_into_byte_plots(cuda_lib, w):
    """From w = 241 the default plan takes 16-bit lanes while the plot still
    fits bytes: the uint8 plot equals the oracle's."""
    ap = cuda_lib
    x = synth.alphabet_string(w, 1, w + 300, synth.DNA)
    y, _ = synth.plant(x, synth.alphabet_string(w, 2, w + 280, synth.DNA), 1, 150, w, 3, synth.DNA, 0.1, 0.05)
    assert ap.plot_plan(len(x), len(y), w)["lane_bits"] == 16
    got = gpu_plot(ap, x, y, w, (1, 0, 0), torch.uint8)
    o = oracle.plot(x, y, w)
    assert got.shape == o.shape and np.array_equal(got, o), np.argwhere(got != o)[:4].tolist()


@pytest.mark.parametrize("w,scores", [(9, (1, 0, 0)), (100, (1, 0, 0)), (150, (1, 0, 0)),
                                      (300, (1, 0, 0)), (20, (2, 1, 0)), (90, (2, 1, 0)),
                                      (140, (2, 1, 0))])
def test_tiny_chunks_cross_many_tiles(cuda_lib, w, scores):
    ap = cuda_lib
    x = synth.dna(5, 1, w + 140)
    y = synth.dna(5, 2, w + 1000)
    o = oracle.plot(x, y, w, scores[0], scores[1])
    try:
        ap.set_chunk(32)
        g = gpu_plot(ap, x, y, w, scores, torch.int16)
    finally:
        ap.set_chunk(0)
    assert np.array_equal(g, o)


def test_all_byte_values_and_identical_windows(cuda_lib):
    ap = cuda_lib
    x = np.concatenate([np.arange(256), np.arange(256)[::-1], np.arange(0, 256, 3)]).astype(np.uint8)
    y = np.concatenate([np.arange(256)[::-1], np.arange(256), synth.dna(1, 1, 100)]).astype(np.uint8)
    for w in (8, 33, 130):
        for sc in ((1, 0, 0), (2, 1, 0)):
            o = oracle.plot(x, y, w, sc[0], sc[1])
            g = gpu_plot(ap, x, y, w, sc, torch.int16)
            assert np.array_equal(g, o), (w, sc)


@pytest.mark.parametrize("case", ["high", "split", "one_high_y"])
def test_top_bit_of_the_alphabet(cuda_lib, case):
    """Tiles whose characters all share the top bit take the short mismatch
    test; the others the general one.  Alphabets entirely at or above 128,
    and mixes across the tiles of one plot, against the oracle."""
    ap = cuda_lib
    hi = bytes([0xC1, 0xC3, 0xC7, 0xF0])
    if case == "high":                      # every tile: all characters >= 128
        x = synth.alphabet_string(5, 1, 700, list(hi))
        y = synth.alphabet_string(5, 2, 900, list(hi))
    elif case == "split":                   # x high, y low: tiles mix top bits
        x = synth.alphabet_string(5, 3, 700, list(hi))
        y = synth.alphabet_string(5, 4, 900, [0x41, 0x43, 0x47, 0x70])
    else:                                   # one character >= 128 in an ASCII y
        x = synth.dna(5, 5, 300)
        y = synth.dna(5, 6, 3000)
        y[1600] = 0xC1
    set_chunk = ap.set_chunk
    try:
        set_chunk(256)                      # several column chunks: some tiles see it
        for w, sc in ((40, (1, 0, 0)), (100, (1, 0, 0)), (150, (1, 0, 0)), (50, (2, 1, 0))):
            o = oracle.plot(x, y, w, sc[0], sc[1])
            g = gpu_plot(ap, x, y, w, sc, torch.int16)
            assert np.array_equal(g, o), (case, w, sc)
            if w <= 100:                    # the vertical-step layout too
                gs = ap.alignment_plot_step(dev(x), dev(y), w, 3, sc, out_dtype=torch.int16)
                torch.cuda.synchronize()
                assert np.array_equal(gs.cpu().numpy().astype(np.int64), o[::3]), (case, w, sc, 3)
    finally:
        set_chunk(0)


def test_empty_and_degenerate(cuda_lib):
    ap = cuda_lib
    x = dev(synth.dna(2, 1, 10))
    y = dev(synth.dna(2, 2, 30))
    assert ap.alignment_plot(x, y, 10).shape == (0, 20)
    assert ap.alignment_plot(y, x, 12).shape == (18, 0)
    assert ap.alignment_plot(x, x, 11).shape == (0, 0)
    p = ap.alignment_plot(y, y, 1)          # w = 1: exact character equality
    torch.cuda.synchronize()
    ya = synth.dna(2, 2, 30)
    assert np.array_equal(p.cpu().numpy(), (ya[:29, None] == ya[None, :29]).astype(np.uint8))


def test_strided_and_wide_outputs(cuda_lib):
    ap = cuda_lib
    x, y = synth.dna(3, 1, 230), synth.dna(3, 2, 310)
    o = oracle.plot(x, y, 30)
    for ld, dt in [(280, torch.uint8), (283, torch.uint8), (301, torch.int16), (288, torch.int16)]:
        buf = torch.full((200, ld), 255, dtype=dt, device="cuda")
        view = buf[:, :280]
        ap.alignment_plot(dev(x), dev(y), 30, out=view)
        torch.cuda.synchronize()
        b = buf.cpu().numpy().astype(np.int64)
        assert np.array_equal(b[:, :280], o), ld
        if ld > 280:
            assert np.all(b[:, 280:] == (255 if dt == torch.uint8 else 255))


def test_validation_errors(cuda_lib):
    ap = cuda_lib
    x, y = dev(synth.dna(4, 1, 300)), dev(synth.dna(4, 2, 300))
    with pytest.raises(ap.ApError) as e:
        ap.alignment_plot(x, y, 200, out_dtype=torch.uint8, scores=(2, 1, 0))   # 2w > 255
    assert e.value.status == ap.AP_E_INVAL
    small = torch.empty((100, 150), dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        ap.alignment_plot(x, y, 100, out=small)


def test_plot_checksum_kernel(cuda_lib):
    ap = cuda_lib
    c = synth.dna_plot_512(0)
    p = ap.alignment_plot(dev(c.x), dev(c.y), c.w)
    cs, hist = ap.plot_checksum(p, c.w + 1)
    o = oracle.plot(c.x, c.y, c.w)
    assert cs == oracle.checksum(o)
    assert hist.tolist() == oracle.histogram(o, c.w + 1).tolist()


@pytest.mark.parametrize("w,thr,scores", [(16, 11, (1, 0, 0)), (40, 29, (1, 0, 0)),
                                          (24, 40, (2, 1, 0)), (130, 90, (1, 0, 0)),
                                          (300, 200, (1, 0, 0))])
def test_dots_match_oracle(cuda_lib, w, thr, scores):
    ap = cuda_lib
    x = synth.dna(6, 1, 700)
    y, _ = synth.plant(x, synth.dna(6, 2, 800), 2, 200, 6, 50, synth.DNA, 0.1, 0.05)
    o = oracle.dots(oracle.plot(x, y, w, scores[0], scores[1]), thr)
    dots, count = ap.alignment_dots(dev(x), dev(y), w, thr, scores)
    torch.cuda.synchronize()
    assert count == len(o)
    assert np.array_equal(ap.dots_to_numpy(dots, count), o)
    # from a materialised plot as well
    p = ap.alignment_plot(dev(x), dev(y), w, scores, out_dtype=torch.int16)
    d2, c2 = ap.plot_dots(p, thr)
    assert c2 == len(o) and np.array_equal(ap.dots_to_numpy(d2, c2), o)


def test_dots_overflow_reports_full_count(cuda_lib):
    ap = cuda_lib
    x, y = synth.dna(7, 1, 300), synth.dna(7, 2, 300)
    o = oracle.dots(oracle.plot(x, y, 12), 8)
    assert len(o) > 10
    with pytest.raises(ap.ApError) as e:
        ap.alignment_dots(dev(x), dev(y), 12, 8, cap=10)
    assert e.value.status == ap.AP_E_OVERFLOW
    dots = torch.empty((10, 3), dtype=torch.int32, device="cuda")
    try:
        ap.alignment_dots(dev(x), dev(y), 12, 8, dots=dots, cap=10)
    except ap.ApError as err:
        assert err.status == ap.AP_E_OVERFLOW
    assert np.array_equal(ap.dots_to_numpy(dots, 10), o[:10])


STEP_CASES = [
    (300, 260, 16, 2, (1, 0, 0)), (333, 290, 30, 5, (1, 0, 0)), (500, 410, 64, 3, (1, 0, 0)),
    (600, 500, 100, 5, (1, 0, 0)), (420, 380, 120, 7, (1, 0, 0)), (250, 300, 20, 5, (2, 1, 0)),
    (500, 430, 100, 5, (2, 1, 0)), (37, 60, 9, 4, (1, 0, 0)),
    # wide windows: full 8-bit keys, 16-bit lanes ({2,1,0} above w = 120)
    (500, 450, 150, 3, (1, 0, 0)), (600, 520, 200, 5, (1, 0, 0)), (620, 600, 128, 7, (1, 0, 0)),
    (700, 640, 256, 4, (1, 0, 0)), (800, 700, 300, 5, (1, 0, 0)), (900, 760, 480, 5, (1, 0, 0)),
    (600, 640, 200, 2, (2, 1, 0)), (700, 600, 150, 3, (2, 1, 0)), (720, 700, 256, 6, (2, 1, 0)),
]


@pytest.mark.parametrize("m,n,w,step,scores", STEP_CASES)
def test_vertical_step(cuda_lib, m, n, w, step, scores):
    """Section 3's step h: only x-windows at multiples of h (rows [::h] of the plot)."""
    ap = cuda_lib
    seed = m + n + w + step
    x = synth.dna(seed, 1, m)
    y, _ = synth.plant(x, synth.dna(seed, 2, n), 1, min(m, n) // 3, seed, 3, synth.DNA, 0.1, 0.05)
    o = oracle.plot(x, y, w, scores[0], scores[1])[::step]
    g = ap.alignment_plot_step(dev(x), dev(y), w, step, scores, out_dtype=torch.int16)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.int64)
    assert g.shape == o.shape and np.array_equal(g, o), np.argwhere(g != o)[:4].tolist()
    if step == 5:
        # step 1 through the same entry point is the plain plot
        g1 = ap.alignment_plot_step(dev(x), dev(y), w, 1, scores, out_dtype=torch.int16)
        torch.cuda.synchronize()
        assert np.array_equal(g1.cpu().numpy().astype(np.int64), oracle.plot(x, y, w, scores[0], scores[1]))


@pytest.mark.parametrize("m,n,w,thr,scores", [(900, 700, 40, 28, (1, 0, 0)), (500, 650, 30, 45, (2, 1, 0)),
                                              (3000, 2500, 100, 75, (1, 0, 0))])
def test_plot_into_host_memory(cuda_lib, m, n, w, thr, scores):
    """ap_alignment_plot_host: host sequences in, host plot and dots out, with
    band copies overlapping the comb; equal to the device plot and dots."""
    ap = cuda_lib
    x = synth.dna(m, 1, m)
    y, _ = synth.plant(x, synth.dna(n, 2, n), 2, min(m, n) // 4, 9, 3, synth.DNA, 0.1, 0.05)
    out, dots, count = ap.alignment_plot_host(x, y, w, scores, threshold=thr)
    dev_plot = ap.alignment_plot(dev(x), dev(y), w, scores, out_dtype=out.dtype)
    torch.cuda.synchronize()
    assert torch.equal(out, dev_plot.cpu())
    want = oracle.dots(dev_plot.cpu().numpy().astype(np.int64), thr)
    assert count == len(want) and np.array_equal(dots, want)
    if m * n < 1_000_000:
        assert np.array_equal(out.numpy().astype(np.int64), oracle.plot(x, y, w, scores[0], scores[1]))
    plot_only, _, _ = ap.alignment_plot_host(x, y, w, scores)
    assert torch.equal(plot_only, out)


@pytest.mark.parametrize("bits,g,w", [(0, 2, 10), (0, 2, 15), (10, 8, 128), (16, 8, 40), (16, 2, 9)])
def test_requests_no_variant_serves_fall_back(cuda_lib, bits, g, w):
    """Requests whose variant would leave a thread more unmasked padding rows
    than it masks take the automatic plan, and plot correctly."""
    ap = cuda_lib
    x, y = synth.dna(w, 1, w + 260), synth.dna(w, 2, w + 300)
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        got = gpu_plot(ap, x, y, w, (1, 0, 0), torch.int16) & 0xFFFF
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    assert np.array_equal(got, oracle.plot(x, y, w))
