"""ap_plot_dots_noalloc against ap_plot_dots (needs a GPU).

ap_plot_dots_noalloc serves callers that cannot allocate device memory (a
plug-in inside a program that owns the GPU's memory, a service that must not
allocate after start-up).  It keeps its scratch in a fixed array inside the
library instead of a caller workspace.  This file runs last, so a failure
here comes after every other test has run."""
import numpy as np
import pytest

from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def test_noalloc_dots_equal_workspace_dots_on_two_calls_in_a_row(cuda_lib):
    ap = cuda_lib
    # Two different plots, one call each: the second call runs on the array the
    # first one left behind, and must still agree exactly with ap_plot_dots.
    cases = [(1, 900, 800, 20, 13, (1, 0, 0)), (2, 700, 1100, 33, 50, (2, 1, 0))]
    for seed, m, n, w, thr, scores in cases:
        x = synth.dna(seed, 1, m)
        y, _ = synth.plant(x, synth.dna(seed, 2, n), 2, 150, seed, 40, synth.DNA, 0.1, 0.05)
        plot = ap.alignment_plot(dev(x), dev(y), w, scores, out_dtype=torch.int16)
        want, want_count = ap.plot_dots(plot, thr)
        assert want_count > 0
        buf = torch.full((want_count + 5, 3), -1, dtype=torch.int32, device="cuda")
        got, got_count = ap.plot_dots_noalloc(plot, thr, buf)
        torch.cuda.synchronize()
        assert got_count == want_count
        assert np.array_equal(ap.dots_to_numpy(got, got_count), ap.dots_to_numpy(want, want_count))


def test_noalloc_rejects_plots_taller_than_its_scratch(cuda_lib):
    ap = cuda_lib
    rows = ap.PLOT_DOTS_NOALLOC_MAX_ROWS + 1
    plot = torch.zeros((rows, 1), dtype=torch.uint8, device="cuda")
    buf = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ap.ApError) as e:
        ap.plot_dots_noalloc(plot, 1, buf)
    assert e.value.status == ap.AP_E_NOMEM
