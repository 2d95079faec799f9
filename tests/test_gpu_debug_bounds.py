"""The bounds-checked debug build against the oracle (needs a GPU).

The library compiled with AP_DEBUG_BOUNDS checks every plot store, sequence
read, exit-ring slot and match-table read of the comb kernels against its
buffer; a failed check records a bit and skips the access (no trap).  Here
the debug library (a few variants: one per kind of kernel) runs small plots
of every kind in a child process, each compared cell by cell with the
oracle, and no check may have failed."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import oracle, paper_0909_2000_gb300 as ap
from paper_0909_2000_gb300 import synth
ap.load(build_if_missing=False)
# (m, n, w, scores, step, threads per strip, alphabet, lane bits): one per
# debug variant (0: the automatic choice)
cases = [(300, 280, 16, (1, 0, 0), 1, 0, "dna", 0), (400, 420, 100, (1, 0, 0), 1, 0, "dna", 0),
         (350, 330, 100, (1, 0, 0), 1, 0, "protein", 0), (330, 300, 80, (1, 0, 0), 1, 2, "dna", 0),
         (400, 380, 128, (1, 0, 0), 1, 0, "dna", 0), (500, 520, 256, (1, 0, 0), 1, 0, "dna", 0),
         (600, 620, 300, (1, 0, 0), 1, 0, "dna", 0), (600, 620, 300, (1, 0, 0), 1, 4, "dna", 10),
         (200, 210, 24, (2, 1, 0), 1, 0, "protein", 0), (500, 480, 250, (2, 1, 0), 1, 0, "dna", 0),
         (150, 160, 8, (3, 1, 0), 1, 0, "dna", 0), (260, 240, 40, (5, 2, 0), 1, 0, "protein", 0),
         (300, 280, 16, (1, 0, 0), 3, 0, "dna", 0)]
out = []
for k, (m, n, w, sc, step, g, alph, lb) in enumerate(cases):
    gen = synth.dna if alph == "dna" else synth.protein
    x = gen(k, 1, m)
    y, _ = synth.plant(x, gen(k, 2, n), 1, min(m, n) // 3, k, 3,
                       synth.DNA if alph == "dna" else synth.PROTEIN, 0.1, 0.05)
    ap.set_lanes_per_strip(g)
    ap.set_lane_bits(lb)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    if step == 1:
        p = ap.alignment_plot(dx, dy, w, sc, out_dtype=torch.int16)
    else:
        p = ap.alignment_plot_step(dx, dy, w, step, sc, out_dtype=torch.int16)
    torch.cuda.synchronize()
    ap.set_lanes_per_strip(0)
    ap.set_lane_bits(0)
    got = p.cpu().numpy().astype(np.int64) & 0xFFFF
    want = oracle.plot(x, y, w, sc[0], sc[1])[::step]
    out.append([k, bool(got.shape == want.shape and np.array_equal(got, want))])
print(json.dumps({"equal": out, "flags": ap.debug_bounds()}))
"""


def test_debug_build_checks_every_access(cuda_lib):
    from paper_0909_2000_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, AP_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert all(ok for _, ok in d["equal"]), d
    assert d["flags"] == 0, "bounds checks failed: bits %#x" % d["flags"]
