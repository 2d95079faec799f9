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


def _plot(ap, seed, m, n, w, scores, dtype):
    x = synth.dna(seed, 1, m)
    y, _ = synth.plant(x, synth.dna(seed, 2, n), 2, 150, seed, 40, synth.DNA, 0.1, 0.05)
    return ap.alignment_plot(dev(x), dev(y), w, scores, out_dtype=dtype)


def test_zero_size_call_loads_the_scratch(cuda_lib):
    # the start-up call a caller makes once per device: nothing to scan
    ap = cuda_lib
    plot = torch.zeros((0, 5), dtype=torch.uint8, device="cuda")
    buf = torch.empty((1, 3), dtype=torch.int32, device="cuda")
    _, count = ap.plot_dots_noalloc(plot, 1, buf)
    assert count == 0


def test_noalloc_dots_equal_workspace_dots_on_two_calls_in_a_row(cuda_lib):
    ap = cuda_lib
    # Plots of both element widths, one call each: every call after the first
    # runs on the array the previous one left behind, and must still agree
    # exactly with ap_plot_dots.
    cases = [(1, 900, 800, 20, 13, (1, 0, 0), torch.int16), (2, 700, 1100, 33, 50, (2, 1, 0), torch.int16),
             (3, 1200, 1000, 24, 16, (1, 0, 0), torch.uint8), (4, 800, 900, 40, 27, (1, 0, 0), torch.uint8)]
    for seed, m, n, w, thr, scores, dtype in cases:
        plot = _plot(ap, seed, m, n, w, scores, dtype)
        want, want_count = ap.plot_dots(plot, thr)
        assert want_count > 0
        buf = torch.full((want_count + 5, 3), -1, dtype=torch.int32, device="cuda")
        got, got_count = ap.plot_dots_noalloc(plot, thr, buf)
        torch.cuda.synchronize()
        assert got_count == want_count
        assert np.array_equal(ap.dots_to_numpy(got, got_count), ap.dots_to_numpy(want, want_count))


def test_noalloc_overflow_keeps_the_first_dots_and_the_full_count(cuda_lib):
    ap = cuda_lib
    plot = _plot(ap, 5, 1000, 1000, 20, (1, 0, 0), torch.uint8)
    want, want_count = ap.plot_dots(plot, 12)
    cap = want_count // 3
    assert cap > 0
    for _ in range(2):
        buf = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
        with pytest.raises(ap.ApError) as e:
            ap.plot_dots_noalloc(plot, 12, buf)
        assert e.value.status == ap.AP_E_OVERFLOW
        assert e.value.count == want_count
        assert np.array_equal(ap.dots_to_numpy(buf, cap), ap.dots_to_numpy(want, want_count)[:cap])


def test_noalloc_rejects_plots_taller_than_its_scratch(cuda_lib):
    ap = cuda_lib
    rows = ap.PLOT_DOTS_NOALLOC_MAX_ROWS + 1
    plot = torch.zeros((rows, 1), dtype=torch.uint8, device="cuda")
    buf = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ap.ApError) as e:
        ap.plot_dots_noalloc(plot, 1, buf)
    assert e.value.status == ap.AP_E_NOMEM
    with pytest.raises(ValueError):
        ap.plot_dots_noalloc(torch.zeros((4, 4), dtype=torch.uint8, device="cuda"), 1, buf, cap=5)
