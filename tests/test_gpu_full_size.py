"""The large workloads at full size, in the launch configuration the
benchmark times (needs a GPU; device memory up to ~150 GB).

Every value of every plot is checked against the oracle through the whole
plot's digest (checksum and value histogram, the GPU's checksum kernel
against the digest that tests/golden/make_golden.py stored from the oracle:
the dynamic programme and the bit-parallel reference where both finish on
the host, the bit-parallel reference alone for the largest plots).  The
oracle also computes seeded plot values on its own (the O(w^2) dynamic
programme of Section 2 per window pair).  Properties that hold at any size
are checked on the whole plot:
* the value range;
* the neighbour bounds;
* the dot list against the plot.

Those whole-plot checks use torch reductions on the device; they verify the
output and are not part of the product path."""
import os

import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BAND = 4096   # plot rows per verification band


def _sampled(plot, pair, count, seed):
    rows, cols = plot.shape
    ii = synth.below(seed, 1, count, rows)
    jj = synth.below(seed, 2, count, cols)
    dev = plot.device
    got = plot[torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy().astype(np.int64)
    want = oracle.samples(pair.x, pair.y, pair.w, ii, jj, pair.scores[0], pair.scores[1])
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first mismatch at (%d, %d): gpu %d, oracle %d" % (
        ii[bad[0]], jj[bad[0]], got[bad[0]], want[bad[0]])


def _neighbour_bounds(plot, lo, hi, step):
    """lo <= P <= hi and |P[i,j] - P[i',j']| <= step for the right, lower and
    lower-right neighbours (Section 2: one character more or less changes the
    LCS by at most one, the {2,1,0} score by at most two)."""
    rows = plot.shape[0]
    for r0 in range(0, rows, BAND):
        r1 = min(rows, r0 + BAND + 1)
        b = plot[r0:r1].to(torch.int32)
        if plot.dtype == torch.int16:
            b = b & 0xFFFF
        assert int(b.min()) >= lo and int(b.max()) <= hi
        assert int((b[:, 1:] - b[:, :-1]).abs().max()) <= step
        if b.shape[0] > 1:
            assert int((b[1:] - b[:-1]).abs().max()) <= step
            assert int((b[1:, 1:] - b[:-1, :-1]).abs().max()) <= step


def _dots_match_plot(plot, dots, count, thr):
    """The dot list is exactly the row-major list of plot cells >= thr."""
    rows = plot.shape[0]
    off = 0
    for r0 in range(0, rows, BAND):
        r1 = min(rows, r0 + BAND)
        b = plot[r0:r1].to(torch.int32)
        nz = torch.nonzero(b >= thr)
        k = nz.shape[0]
        d = dots[off:off + k].to(torch.int64)
        assert d.shape[0] == k
        assert torch.equal(d[:, 0], nz[:, 0] + r0)
        assert torch.equal(d[:, 1], nz[:, 1])
        assert torch.equal(d[:, 2] & 0xFFFF, b[nz[:, 0], nz[:, 1]].to(torch.int64))
        off += k
    assert off == count


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _digest_matches_golden(ap, plot, name, nbins):
    """The GPU checksum kernel's digest of the whole plot equals the
    oracle's stored digest (written from the oracle only)."""
    kv = dict(l.split("=", 1) for l in open(os.path.join(GOLDEN, name + ".txt")).read().split() if "=" in l)
    assert tuple(plot.shape) == tuple(int(v) for v in kv["shape"].split("x"))
    cs, hist = ap.plot_checksum(plot, nbins)
    want_hist = [int(v) for v in kv["histogram"].split(",")]
    assert list(hist) == want_hist, "histogram differs from the oracle's"
    assert cs == int(kv["checksum"]), "checksum differs from the oracle's"


def test_lcs_dna_100k_w100(cuda_lib):
    """m = n = 100,000 DNA with 20 planted homologies, w = 100: the full
    99,900 x 99,900 uint8 plot and the dots >= 80."""
    ap = cuda_lib
    c = synth.dna_plot_100k(0)
    dev = torch.device("cuda")
    rows, cols = ap.plot_shape(len(c.x), len(c.y), c.w)
    x, y = torch.from_numpy(c.x).to(dev), torch.from_numpy(c.y).to(dev)
    plot = ap.empty_plot(rows, cols, torch.uint8, dev)
    ap.alignment_plot(x, y, c.w, ap.LCS, out=plot)
    torch.cuda.synchronize()
    _sampled(plot, c, 100_000, seed=21)
    _neighbour_bounds(plot, 0, c.w, 1)
    dots, count = ap.plot_dots(plot, c.threshold)
    assert count > 0
    _dots_match_plot(plot, dots, count, c.threshold)
    # the dots come from the planted homologies: almost all lie on a planted
    # segment's diagonal band (indels let the diagonal drift), and every
    # segment yields dots
    d = dots[:count].to(torch.int64)
    on_band = torch.zeros(count, dtype=torch.bool, device=dev)
    for xs, ys, ln in c.planted:
        band = ((d[:, 0] >= xs - c.w) & (d[:, 0] <= xs + ln)
                & ((d[:, 1] - d[:, 0]) - (ys - xs)).abs().le(150))
        assert int(band.sum()) >= 100
        on_band |= band
    assert int(on_band.sum()) >= 0.99 * count
    # the banded plot-free path gives the same dots
    dots2, count2 = ap.alignment_dots(x, y, c.w, c.threshold)
    assert count2 == count and torch.equal(dots2[:count2], dots[:count])
    _digest_matches_golden(ap, plot, c.name, c.w + 1)
    del plot, dots, dots2
    torch.cuda.empty_cache()


def test_score_protein_20k_w64(cuda_lib):
    """m = n = 20,000 over 20 letters, w = 64, scores {2,1,0}: the full
    uint16 plot (values w..2w)."""
    ap = cuda_lib
    c = synth.protein_score_20k(0)
    dev = torch.device("cuda")
    rows, cols = ap.plot_shape(len(c.x), len(c.y), c.w)
    x, y = torch.from_numpy(c.x).to(dev), torch.from_numpy(c.y).to(dev)
    plot = ap.empty_plot(rows, cols, torch.int16, dev)
    ap.alignment_plot(x, y, c.w, ap.SCORE, out=plot)
    torch.cuda.synchronize()
    _sampled(plot, c, 100_000, seed=22)
    # every window pair scores at least w (align position by position)
    _neighbour_bounds(plot, c.w, 2 * c.w, 2)
    _digest_matches_golden(ap, plot, c.name, 2 * c.w + 1)
    del plot
    torch.cuda.empty_cache()


@pytest.mark.parametrize("gen", [synth.dna_plot_20k, synth.dna_plot_20k_w256, synth.dna_score_80k_step5])
def test_more_whole_plots_against_stored_oracle_digests(cuda_lib, gen):
    """The 20k DNA plots at w = 100 (7-bit keys) and w = 256 (16-bit lanes,
    uint16 plot), and the shape of the paper's Table 1 runs (80k x 80k,
    {2,1,0}, w = 100, vertical step 5): whole-plot digests and samples."""
    ap = cuda_lib
    c = gen(0)
    dev = torch.device("cuda")
    x, y = torch.from_numpy(c.x).to(dev), torch.from_numpy(c.y).to(dev)
    rows, cols = oracle.step_shape(len(c.x), len(c.y), c.w, c.step)
    nb = c.scores[0] * c.w + 1
    plot = ap.empty_plot(rows, cols, torch.uint8 if nb <= 256 else torch.int16, dev)
    if c.step > 1:
        ap.alignment_plot_step(x, y, c.w, c.step, (c.scores[0], c.scores[1], 0), out=plot)
    else:
        ap.alignment_plot(x, y, c.w, (c.scores[0], c.scores[1], 0), out=plot)
    torch.cuda.synchronize()
    _digest_matches_golden(ap, plot, c.name, nb)
    ii = synth.below(24, 1, 20_000, rows)
    jj = synth.below(24, 2, 20_000, cols)
    got = plot[torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy().astype(np.int64)
    want = oracle.samples(c.x, c.y, c.w, ii * c.step, jj, c.scores[0], c.scores[1])
    assert np.array_equal(got & 0xFFFF, want)
    del plot
    torch.cuda.empty_cache()


def test_batch_4096_pairs(cuda_lib):
    """4096 DNA pairs (lengths log-uniform 200..20000, w in {16,32,64,128}):
    the autotuned graph launch against one plain launch per pair, and seeded
    oracle samples from every job."""
    ap = cuda_lib
    jobs = synth.batch_jobs(0)
    dev = torch.device("cuda")
    X = torch.from_numpy(np.concatenate([j.x for j in jobs])).to(dev)
    Y = torch.from_numpy(np.concatenate([j.y for j in jobs])).to(dev)
    xo = np.cumsum([0] + [len(j.x) for j in jobs])
    yo = np.cumsum([0] + [len(j.y) for j in jobs])
    shapes, oo = [], [0]
    for j in jobs:
        r, cl = max(0, len(j.x) - j.w), max(0, len(j.y) - j.w)
        ld = (cl + 31) // 32 * 32
        shapes.append((r, cl, ld))
        oo.append(oo[-1] + r * ld)
    out_p = torch.zeros(oo[-1], dtype=torch.uint8, device=dev)
    out_b = torch.zeros(oo[-1], dtype=torch.uint8, device=dev)

    def views(buf):
        return [buf[oo[k]:oo[k] + r * ld].view(r, ld)[:, :cl] if r else buf[:0].view(0, cl)
                for k, (r, cl, ld) in enumerate(shapes)]
    vp, vb = views(out_p), views(out_b)
    xs = [X[xo[k]:xo[k + 1]] for k in range(len(jobs))]
    ys = [Y[yo[k]:yo[k + 1]] for k in range(len(jobs))]
    batch = ap.Batch([(xs[k], ys[k], jobs[k].w, ap.LCS, vb[k]) for k in range(len(jobs))],
                     autotune=True)
    batch.run()
    for k, j in enumerate(jobs):
        if shapes[k][0] and shapes[k][1]:
            ap.alignment_plot(xs[k], ys[k], j.w, ap.LCS, out=vp[k])
    torch.cuda.synchronize()
    assert torch.equal(out_p, out_b)
    checked = 0
    for k, j in enumerate(jobs):
        r, cl, _ = shapes[k]
        if r == 0 or cl == 0:
            continue
        ii = synth.below(23, 2 * k, 8, r)
        jj = synth.below(23, 2 * k + 1, 8, cl)
        got = vb[k][torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy()
        want = oracle.samples(j.x, j.y, j.w, ii, jj)
        assert np.array_equal(got.astype(np.int64), want), "job %d" % k
        checked += 1
    assert checked > 4000
    batch.close()
    del out_p, out_b
    torch.cuda.empty_cache()
