"""The banded paths, many bands on small plots, against the oracle (needs a GPU).

ap_alignment_dots, ap_alignment_plot_host and the server's jobs comb a plot
band by band (about 1 GB of plot per band, or a share of the server's
budget), so at the sizes the oracle can finish they would run a single band.
ap_set_band_rows forces small bands here: every band boundary, the dot
lists appended band after band, the host plot's band copies (with the
halving bands at the end) and the server's band loop are then compared with
the oracle's full plot, cell by cell and dot by dot."""
import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def _pair(seed, m, n, alph=None):
    x = synth.dna(seed, 1, m) if alph is None else synth.alphabet_string(seed, 1, m, alph)
    y = synth.dna(seed, 2, n) if alph is None else synth.alphabet_string(seed, 2, n, alph)
    y, _ = synth.plant(x, y, 2, min(m, n) // 4, seed, 3, synth.DNA, 0.1, 0.05)
    return x, y


# (m, n, w, scores, threshold, band rows): band rows are rounded up to whole
# strip groups (128 strips for one-thread 8-bit lanes, 64 for two threads,
# 32 for the 16-bit lanes on four threads), so every case runs 3..10 bands
BANDED = [(900, 700, 40, (1, 0, 0), 28, 128), (1000, 800, 100, (1, 0, 0), 72, 100),
          (700, 900, 24, (2, 1, 0), 36, 128), (620, 700, 150, (1, 0, 0), 110, 64),
          (600, 650, 256, (1, 0, 0), 190, 32), (800, 600, 70, (2, 1, 0), 110, 100)]


@pytest.fixture
def band_rows(cuda_lib):
    def set_(r):
        cuda_lib.set_band_rows(r)
    yield set_
    cuda_lib.set_band_rows(0)


@pytest.mark.parametrize("m,n,w,scores,thr,br", BANDED)
def test_banded_dots_match_the_oracle(cuda_lib, band_rows, m, n, w, scores, thr, br):
    ap = cuda_lib
    x, y = _pair(m + w, m, n)
    want = oracle.dots(oracle.plot(x, y, w, scores[0], scores[1]), thr)
    assert len(want) > 0
    band_rows(br)
    dots, count = ap.alignment_dots(dev(x), dev(y), w, thr, scores)
    torch.cuda.synchronize()
    assert count == len(want) and np.array_equal(ap.dots_to_numpy(dots, count), want)


@pytest.mark.parametrize("m,n,w,scores,thr,br", BANDED)
def test_banded_host_plot_matches_the_oracle(cuda_lib, band_rows, m, n, w, scores, thr, br):
    ap = cuda_lib
    x, y = _pair(m + 2 * w, m, n)
    full = oracle.plot(x, y, w, scores[0], scores[1])
    band_rows(br)
    out, dots, count = ap.alignment_plot_host(x, y, w, scores, threshold=thr)
    assert np.array_equal(out.numpy().astype(np.int64) & 0xFFFF, full)
    want = oracle.dots(full, thr)
    assert count == len(want) and np.array_equal(dots, want)
    # a host plot with a row stride other than the device band's: 2-D copies
    rows, cols = full.shape
    wide = torch.full((rows, cols + 5), 7, dtype=out.dtype)
    ap.alignment_plot_host(x, y, w, scores, out=wide[:, :cols])
    assert np.array_equal(wide[:, :cols].numpy().astype(np.int64) & 0xFFFF, full)
    assert bool((wide[:, cols:] == 7).all())


def test_banded_server_jobs_match_the_oracle(cuda_lib, band_rows):
    ap = cuda_lib
    band_rows(64)                 # set before submission: jobs are planned at submit
    srv = ap.Server(mem_budget=2 << 30, max_slots=4)
    cases = [(m, n, w, sc, thr) for (m, n, w, sc, thr, _) in BANDED]
    tickets, wants = [], []
    for k, (m, n, w, sc, thr) in enumerate(cases):
        x, y = _pair(100 + k, m, n)
        wants.append(oracle.dots(oracle.plot(x, y, w, sc[0], sc[1]), thr))
        tickets.append(srv.submit(x, y, w, thr, sc))
    for t, want in zip(tickets, wants):
        assert srv.wait(t, 60000) == ap.AP_OK
        st, cnt, dots = srv.fetch(t)
        assert cnt == len(want) and np.array_equal(dots, want)
    srv.close()
