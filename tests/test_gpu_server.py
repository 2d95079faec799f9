"""Dot-plot server (continuous batching, admission by device memory) against
the plain dots call and the oracle (needs a GPU)."""
import time

import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def requests(seed=0):
    specs = [(16, 12, (1, 0, 0)), (32, 24, (1, 0, 0)), (64, 46, (1, 0, 0)), (100, 72, (1, 0, 0)),
             (128, 92, (1, 0, 0)), (256, 178, (1, 0, 0)), (20, 35, (2, 1, 0)), (60, 100, (2, 1, 0))]
    out = []
    for k, (w, thr, sc) in enumerate(specs * 2):
        m = int(synth.below(seed, 50 + k, 1, 3000)[0]) + w + 50
        n = int(synth.below(seed, 80 + k, 1, 3000)[0]) + w + 50
        x = synth.dna(seed, 100 + k, m)
        y, _ = synth.plant(x, synth.dna(seed, 200 + k, n), 1, min(m, n) // 3, seed, 300 + 7 * k,
                           synth.DNA, 0.08, 0.04)
        out.append((x, y, w, thr, sc))
    return out


def reference(ap, x, y, w, thr, sc):
    d, c = ap.alignment_dots(dev(x), dev(y), w, thr, sc)
    return ap.dots_to_numpy(d, c)


def test_results_are_the_same_alone_and_in_the_mix(cuda_lib):
    ap = cuda_lib
    reqs = requests(0)
    refs = [reference(ap, *r) for r in reqs]
    assert sum(len(r) for r in refs) > 0
    srv = ap.Server(mem_budget=8 << 30, max_slots=6)
    # alone: one request at a time
    for r, ref in zip(reqs, refs):
        x, y, w, thr, sc = r
        t = srv.submit(x, y, w, thr, sc)
        assert srv.wait(t, 60000) == ap.AP_OK
        st, cnt, dots = srv.fetch(t)
        assert st == ap.AP_OK and cnt == len(ref) and np.array_equal(dots, ref)
    # in the mix: everything submitted at once, overlapping on the device
    tickets = [srv.submit(x, y, w, thr, sc) for x, y, w, thr, sc in reqs]
    for t, ref in zip(tickets, refs):
        assert srv.wait(t, 120000) == ap.AP_OK
        st, cnt, dots = srv.fetch(t)
        assert cnt == len(ref) and np.array_equal(dots, ref)
    s = srv.stats()
    assert s["completed"] == 2 * len(reqs) and s["failed"] == 0 and s["queued"] == 0
    assert s["latency_p99_ms"] >= s["latency_p50_ms"] > 0
    srv.close()


def test_small_results_match_the_oracle(cuda_lib):
    ap = cuda_lib
    srv = ap.Server(mem_budget=1 << 30, max_slots=3)
    for seed, (m, n, w, thr, sc) in enumerate([(300, 280, 12, 9, (1, 0, 0)), (250, 310, 30, 22, (1, 0, 0)),
                                               (200, 260, 10, 16, (2, 1, 0))]):
        x = synth.dna(seed, 1, m)
        y, _ = synth.plant(x, synth.dna(seed, 2, n), 1, 120, seed, 9, synth.DNA, 0.1, 0.0)
        t = srv.submit(x, y, w, thr, sc)
        assert srv.wait(t, 30000) == ap.AP_OK
        _, cnt, dots = srv.fetch(t)
        want = oracle.dots(oracle.plot(x, y, w, sc[0], sc[1]), thr)
        assert cnt == len(want) and np.array_equal(dots, want)
    srv.close()


def test_admission_by_memory_budget(cuda_lib):
    ap = cuda_lib
    reqs = requests(1)[:6]
    refs = [reference(ap, *r) for r in reqs]
    # a budget that holds only one or two jobs at a time: the rest wait in the queue
    srv = ap.Server(mem_budget=48 << 20, max_slots=8)
    tickets = [srv.submit(x, y, w, thr, sc, max_dots=100000) for x, y, w, thr, sc in reqs]
    for t, ref in zip(tickets, refs):
        assert srv.wait(t, 120000) == ap.AP_OK
        _, cnt, dots = srv.fetch(t)
        assert np.array_equal(dots, ref)
    assert 0 < srv.stats()["peak_device_bytes"] <= 48 << 20
    with pytest.raises(ap.ApError) as e:
        srv.submit(synth.dna(1, 1, 60000), synth.dna(1, 2, 60000), 50, 40)
    assert e.value.status == ap.AP_E_NOMEM
    srv.close()


def test_wait_timeout_cancel_and_overflow(cuda_lib):
    ap = cuda_lib
    srv = ap.Server(mem_budget=4 << 30, max_slots=1)
    big_x = synth.dna(3, 1, 60000)
    big_y, _ = synth.plant(big_x, synth.dna(3, 2, 60000), 6, 2000, 3, 11, synth.DNA, 0.1, 0.05)
    t_big = srv.submit(big_x, big_y, 100, 80)
    t_queued = srv.submit(big_x[:5000], big_y[:5000], 100, 80)
    assert srv.wait(t_big, 0) == ap.AP_E_TIMEOUT          # a bounded wait returns
    assert srv.poll(t_queued) == ap.AP_E_BUSY
    srv.cancel(t_queued)
    assert srv.wait(t_queued, 10000) == ap.AP_E_CANCELLED
    assert srv.wait(t_big, 120000) == ap.AP_OK
    # the big job runs several plot bands (its band is a share of the
    # budget): its dots equal the plain call's, and seeded oracle samples
    # confirm dot values and non-dots below the threshold
    _, cnt, dots = srv.fetch(t_big)
    plain = reference(ap, big_x, big_y, 100, 80, (1, 0, 0))
    assert cnt == len(plain) > 1000 and np.array_equal(dots, plain)
    pick = dots[synth.below(3, 40, 300, len(dots))]
    assert np.array_equal(oracle.samples(big_x, big_y, 100, pick[:, 0], pick[:, 1]), pick[:, 2])
    ii, jj = synth.below(3, 41, 300, 59900), synth.below(3, 42, 300, 59900)
    dotset = set(map(tuple, dots[:, :2].tolist()))
    off = [(i, j) for i, j in zip(ii.tolist(), jj.tolist()) if (i, j) not in dotset]
    vals = oracle.samples(big_x, big_y, 100, [i for i, _ in off], [j for _, j in off])
    assert bool((vals < 80).all())
    # overflow: the full count and the first max_dots dots
    x = synth.dna(4, 1, 800)
    y, _ = synth.plant(x, synth.dna(4, 2, 900), 1, 400, 4, 5, synth.DNA, 0.05, 0.0)
    ref = reference(ap, x, y, 20, 15, (1, 0, 0))
    assert len(ref) > 10
    t = srv.submit(x, y, 20, 15, max_dots=10)
    assert srv.wait(t, 30000) == ap.AP_E_OVERFLOW
    st, cnt, dots = srv.fetch(t)
    assert st == ap.AP_E_OVERFLOW and cnt == len(ref) and np.array_equal(dots, ref[:10])
    with pytest.raises(ap.ApError):
        srv.poll(t)                                        # fetched tickets are forgotten
    srv.close()
