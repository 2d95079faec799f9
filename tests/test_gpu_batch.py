"""Batched plots (one CUDA graph of persistent comb kernels) against plain
calls and the oracle (needs a GPU)."""
import numpy as np
import pytest

import oracle
from paper_0909_2000_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def make_jobs(seed=0):
    specs = [(1, (1, 0, 0)), (7, (1, 0, 0)), (16, (1, 0, 0)), (31, (1, 0, 0)), (64, (1, 0, 0)),
             (100, (1, 0, 0)), (120, (1, 0, 0)), (128, (1, 0, 0)), (200, (1, 0, 0)),
             (300, (1, 0, 0)),
             (5, (2, 1, 0)), (64, (2, 1, 0)), (90, (2, 1, 0)), (130, (2, 1, 0))]
    jobs = []
    k = 0
    for rep in range(3):
        for w, sc in specs:
            m = int(synth.below(seed, 100 + k, 1, 600)[0]) + w // 2 + 20
            n = int(synth.below(seed, 200 + k, 1, 900)[0]) + w // 2 + 20
            x = synth.dna(seed, 300 + k, m)
            y = synth.dna(seed, 400 + k, n)
            jobs.append((x, y, w, sc))
            k += 1
    jobs.append((synth.dna(seed, 1, 10), synth.dna(seed, 2, 50), 12, (1, 0, 0)))   # empty plot
    return jobs


def run_both(ap, jobs, **kw):
    plain, batched, keep = [], [], []
    for x, y, w, sc in jobs:
        dx, dy = dev(x), dev(y)
        rows, cols = max(0, len(x) - w), max(0, len(y) - w)
        dt = torch.int16
        out_b = ap.empty_plot(rows, cols, dt, "cuda").fill_(-1)
        p = ap.alignment_plot(dx, dy, w, sc, out_dtype=dt)
        plain.append(p)
        batched.append(out_b)
        keep.append((dx, dy, w, sc, out_b))
    b = ap.Batch(keep, **kw)
    b.run()
    torch.cuda.synchronize()
    return plain, batched, b


def test_batch_matches_plain_and_oracle(cuda_lib):
    ap = cuda_lib
    jobs = make_jobs(0)
    plain, batched, b = run_both(ap, jobs)
    info = b.info()
    nonempty = sum(1 for x, y, w, _ in jobs if len(x) > w and len(y) > w)
    assert info["jobs"] == nonempty and info["groups"] >= 8
    for (x, y, w, sc), p, q in zip(jobs, plain, batched):
        assert torch.equal(p, q), (w, sc, len(x), len(y))
    # small ones against the oracle, cell by cell
    for (x, y, w, sc), q in list(zip(jobs, batched))[:13]:
        if q.numel() and q.numel() < 200_000:
            assert np.array_equal(q.cpu().numpy().astype(np.int64), oracle.plot(x, y, w, sc[0], sc[1])), (w, sc)
    # replaying the graph gives the same plots
    for q in batched:
        q.fill_(-1)
    b.run()
    torch.cuda.synchronize()
    for p, q in zip(plain, batched):
        assert torch.equal(p, q)
    b.close()


def test_batch_autotuned_schedule_gives_identical_plots(cuda_lib):
    ap = cuda_lib
    jobs = make_jobs(1)[:20]
    plain, batched, b = run_both(ap, jobs, autotune=True)
    for p, q in zip(plain, batched):
        assert torch.equal(p, q)
    assert b.info()["tune_ms"] >= 0
    b.close()


def test_batch_validation_names_the_bad_job(cuda_lib):
    ap = cuda_lib
    x, y = dev(synth.dna(2, 1, 200)), dev(synth.dna(2, 2, 200))
    good = torch.empty((180, 180), dtype=torch.uint8, device="cuda")
    small = torch.empty((180, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(ap.ApError) as e:
        ap.Batch([(x, y, 20, (1, 0, 0), good), (x, y, 20, (1, 0, 0), small[:, :100])])
    assert e.value.status == ap.AP_E_INVAL and "job 1" in str(e.value)


TUNE_SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_0909_2000_gb300 as ap
from paper_0909_2000_gb300 import synth
keep, outs = [], []
for k, (w, sc) in enumerate([(16, (1, 0, 0)), (64, (1, 0, 0)), (128, (1, 0, 0)), (40, (2, 1, 0))] * 3):
    x = torch.from_numpy(synth.dna(k, 1, 2500 + 97 * k)).cuda()
    y = torch.from_numpy(synth.dna(k, 2, 3000 + 53 * k)).cuda()
    out = ap.empty_plot(x.numel() - w, y.numel() - w, torch.int16, "cuda")
    keep.append((x, y, w, sc, out))
    outs.append(out)
b = ap.Batch(keep, autotune=True)
b.run()
torch.cuda.synchronize()
print(json.dumps({"tune_ms": b.info()["tune_ms"], "sums": [int(o.to(torch.int64).sum()) for o in outs]}))
"""


def test_autotune_cache_persists_across_processes(cuda_lib, tmp_path):
    """The tuner's choices are kept in the cache file (AP_TUNE_CACHE): a second
    process on the same GPU kind tunes nothing and writes the same plots."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, AP_TUNE_CACHE=str(tmp_path / "tune.txt"))
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", TUNE_SCRIPT, root], env=env, capture_output=True,
                           text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert runs[0]["tune_ms"] > 0 and runs[1]["tune_ms"] == 0
    assert runs[0]["sums"] == runs[1]["sums"]
    lines = (tmp_path / "tune.txt").read_text().splitlines()
    assert len(lines) == 4 and all("|" in l for l in lines)      # one per window class
