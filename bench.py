#!/usr/bin/env python
"""Benchmark: window-pair cells per second of the GB300 alignment-plot path.

Default workload (one step = the whole hot path over one input):
    LCS alignment plot of DNA, m = n = 100,000, w = 100, with 20 planted
    homologous segments (2000 long, 10% substitutions, 5% indels): the full
    99,900 x 99,900 uint8 plot in HBM, then the dots with WLCS >= 80 from it.

metric  = m * n * w / step time (window-pair cells/s), whole job.
roofline: the strip-comb kernel is bound by the integer ALU.  Its algorithmic
    work is 6 lane-operations per comb cell (Section 3's vector step: match
    mask, compare/exchange as min and max, two blends, the per-column
    increment), i.e. 1.5 32-bit operations per cell with 4 lanes per
    register.  Comb cells per plot = (m - w)(n - 1)w.  The peak is
    SMs x 32-bit integer lanes per SM per clock x the SM clock.

After the headline, the default run (one GPU) adds a record for each other
workload, under "workloads", each with its own clock record and parity flag:
    lcs_dna_512_w16        LCS, DNA m = n = 512, w = 16: time per call, full
                           plot against the oracle;
    score_protein_20k_w64  {2,1,0}, 20-letter protein m = n = 20,000, w = 64,
                           uint16 plot: cells/s, roofline, whole-plot digest
                           against the stored oracle digest, oracle samples;
    batch_dna_4096         4096 DNA pairs as one graph launch against a loop of
                           plain calls: both times, identical outputs, samples;
    serve_dna_poisson      Poisson arrivals into the server: capacity under the
                           offered 200 req/s, p50/p99 at 70% of capacity,
                           served dots against plain calls and the oracle.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank combs its own copy of the workload (independent
problems, no collective on the data path; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

INT32_LANES_PER_SM_CLK = 128      # 32-bit integer lanes per SM per clock (GB300)
SM_MAX_MHZ = 2070.0               # maximum SM clock of a GB300
LANE_OPS_PER_CELL = 6.0           # the paper's vector step: 6 lane-ops per comb cell


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lcs_dna_100k_w100",
                    choices=["lcs_dna_100k_w100", "lcs_dna_512_w16", "score_protein_20k_w64",
                             "lcs_dna_20k_w100", "lcs_dna_20k_w128", "lcs_dna_20k_w256", "batch_dna_4096",
                             "serve_dna_poisson",
                             "score_dna_80k_w100_step5"])
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--batch-jobs", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the records of the other workloads in the default run")
    ap.add_argument("--workloads-steps", type=int, default=3,
                    help="timed steps of each other workload's record (default 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="seconds of oracle work per reference-arm step (default: "
                         "150 s over all steps, 2..10 s each)")
    return ap.parse_args()


def workload(name):
    from paper_0909_2000_gb300 import synth
    if name == "lcs_dna_100k_w100":
        return synth.dna_plot_100k(0)
    if name == "lcs_dna_512_w16":
        return synth.dna_plot_512(0)
    if name == "lcs_dna_20k_w100":
        return synth.dna_plot_20k(0)
    if name == "lcs_dna_20k_w128":
        return synth.dna_plot_20k_w128(0)
    if name == "lcs_dna_20k_w256":
        return synth.dna_plot_20k_w256(0)
    return synth.protein_score_20k(0)


def wide(c):
    """True for a uint16 plot: score plots (as the 20k protein workload
    specifies) and plots whose values reach match * w > 255."""
    return tuple(c.scores[:2]) != (1, 0) or c.scores[0] * c.w > 255


def describe(c):
    rows, cols = len(c.x) - c.w, len(c.y) - c.w
    score = tuple(c.scores[:2]) == (2, 1)
    return {
        "workload": c.name, "m": len(c.x), "n": len(c.y), "w": c.w,
        "scores": "match 2, mismatch 1, gap 0" if score else "LCS (match 1, mismatch 0, gap 0)",
        "output": "full %dx%d %s plot in HBM%s" % (rows, cols, "uint16" if wide(c) else "uint8",
                                                  "" if c.threshold is None else
                                                  " + row-major dots >= %d" % c.threshold),
        "inputs": "seeded synthetic (SplitMix64), resident in HBM",
        "l2": "output %.2f GB per step >> 129 MB L2; L2 flushed (256 MB write) before every timed step"
              % (rows * cols * (2 if wide(c) else 1) / 1e9),
    }


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


ARM_PARTS = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
             "0xd49": "Arm Neoverse-N2", "0xd8e": "Arm Neoverse-N3", "0xd84": "Arm Neoverse-V3"}


def cpu_model():
    """The host CPU's model name (x86 'model name', or the Arm part number
    mapped to its core name)."""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":", 1)[0].strip().lower()
            if key in ("model name", "cpu part", "hardware"):
                v = line.split(":", 1)[1].strip()
                return "%s (%s)" % (ARM_PARTS[v], v) if v in ARM_PARTS else v
    except OSError:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
# Multi-rank timing: every rank combs its own copy of the workload (the plot
# shards by strips with no exchange step); the job's time is the slowest
# rank's, and the value counts the units of all ranks.
# ---------------------------------------------------------------------------

def max_over_ranks(local_ms, dist=None, device=None):
    """The largest of the ranks' times (all-reduce MAX); local_ms on one rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank, world, steps, job_ms):
    """Units per second of the whole job: all ranks' units over the job time."""
    return float(units_per_rank) * world * steps / (job_ms / 1e3)


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_rate(c, seconds, seed=7):
    """Times the oracle on seeded window pairs of the workload, scaled so the
    run takes about ``seconds``; returns (cells/s, pairs, elapsed, threads)."""
    import oracle
    from paper_0909_2000_gb300 import synth
    rows, cols = len(c.x) - c.w, len(c.y) - c.w
    nth = cores()
    match, mismatch = c.scores[0], c.scores[1]

    def run(k, off):
        ii = synth.below(seed, 1, k, rows, off)
        jj = synth.below(seed, 2, k, cols, off)
        t = time.perf_counter()
        oracle.samples(c.x, c.y, c.w, ii, jj, match, mismatch, nthreads=nth)
        return time.perf_counter() - t

    k = 256 * nth
    dt = run(k, 0)
    while dt < 0.5:
        k *= 4
        dt = run(k, 0)
    k2 = max(k, int(k * seconds / max(dt, 1e-6) * 0.9))
    dt2 = run(k2, k)
    return k2 * c.w / dt2, k2, dt2, nth


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.file.read().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                  "sw_power_cap"], f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return None
        busy = sorted(sm)[len(sm) // 4:] or sm     # drop idle samples at the edges
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def issue_probe(ap, index, sms):
    """The integer issue rate behind the roofline's peak, measured by the
    library's probe (ap_int_issue_probe): 32-bit lane operations per clock
    and SM of three-input logic alone (ALU pipe), multiply-adds alone (FMA
    pipe) and the two alternately, at the SM clock sampled meanwhile."""
    kinds = {"alu_lop3": 0, "fma_imad": 1, "alu_and_fma": 2}
    clocks = Clocks(index)
    clocks.start()
    rates = {k: ap.int_issue_probe(v, 1000000) for k, v in kinds.items()}
    clk = clocks.stop()
    mhz = clk["sm_mhz"] if clk else SM_MAX_MHZ
    out = {k: r / (sms * mhz * 1e6) for k, r in rates.items()}
    out.update({"unit": "int32 lane-ops/clk/SM", "sm_mhz": mhz,
                "measured_peak_tops_at_max_clock": rates["alu_and_fma"] / mhz * SM_MAX_MHZ / 1e12,
                "assumed_lanes_per_clk_per_sm": INT32_LANES_PER_SM_CLK})
    return out


def profile_traffic(kernel_tag):
    """dram bytes per launch from the committed ncu summary (profiles/traffic.md),
    if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    from paper_0909_2000_gb300 import build as b
    for line in lines:
        f = line.split()
        if len(f) == 4 and f[0] == "traffic:" and f[1] == kernel_tag:
            kv = dict(t.split("=", 1) for t in f[2:])
            if kv.get("sources") == b.kernel_digest():
                return int(kv["dram_bytes_per_launch"])
    return None


def read_golden(name):
    """Stored digest of a workload's whole plot (tests/golden/<name>.txt,
    written from the oracle by tests/golden/make_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", name + ".txt")
    try:
        kv = dict(line.split("=", 1) for line in open(path).read().split() if "=" in line)
    except OSError:
        return None
    return {"checksum": int(kv["checksum"]), "histogram": [int(v) for v in kv["histogram"].split(",")],
            "shape": tuple(int(v) for v in kv["shape"].split("x"))}


def golden_check(ap, plot, name, nbins):
    """The GPU checksum kernel's digest of `plot` against the stored oracle
    digest: True / False, or None when no digest is stored."""
    g = read_golden(name)
    if g is None:
        return None
    cs, hist = ap.plot_checksum(plot, nbins)
    return bool(tuple(plot.shape) == g["shape"] and cs == g["checksum"] and list(hist) == g["histogram"])


def event_times(fn, steps, stream, flush=None):
    """CUDA-event milliseconds of `steps` calls of fn on `stream`, each
    bracketed by synchronisations, with an optional L2 flush before each."""
    import torch
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def comb_roofline(plan, rows, n, w, score, comb_ms, sms, clk):
    """Integer-issue roofline of one comb launch: algorithmic 32-bit ops =
    comb cells x 6 lane-ops / lanes per register, over the launch time."""
    comb_cells = float(rows) * (n - 1) * (2 * w if score else w) * (2 if score else 1)
    alg_ops = comb_cells * LANE_OPS_PER_CELL / plan["strips_per_reg"]
    achieved = alg_ops / (comb_ms / 1e3) / 1e12
    peak = sms * INT32_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "ops_per_cell": LANE_OPS_PER_CELL / plan["strips_per_reg"], "comb_ms": comb_ms,
            "peak_basis": "%d SMs x %d int32 lanes/clk x %.0f MHz (max SM clock)"
                          % (sms, INT32_LANES_PER_SM_CLK, SM_MAX_MHZ),
            "frac_at_measured_clock": (achieved / (sms * INT32_LANES_PER_SM_CLK * clk["sm_mhz"] * 1e6 / 1e12)
                                       if clk else None)}


def percentiles(ms):
    v = sorted(ms)

    def pct(p):
        return v[min(len(v) - 1, max(0, int(math.ceil(p * len(v))) - 1))]
    return {"p10": pct(0.10), "p50": pct(0.50), "p90": pct(0.90), "min": v[0], "max": v[-1]}


# ---------------------------------------------------------------------------
# Records of the other workloads, run after the headline in the default run
# (one GPU), each with its own clock record and parity flag
# ---------------------------------------------------------------------------

def plot_record(ap, c, steps, warmup, dev, host_calls=0):
    """One plot workload: comb time per call (CUDA events, L2 flushed before
    each), cells/s, the integer roofline, and parity: the whole plot against
    the oracle where it is small, else the stored whole-plot digest plus
    seeded oracle samples."""
    import numpy as np
    import torch

    import oracle
    from paper_0909_2000_gb300 import synth
    m, n, w = len(c.x), len(c.y), c.w
    score = tuple(c.scores[:2]) == (2, 1)
    scores = ap.SCORE if score else ap.LCS
    rows, cols = ap.plot_shape(m, n, w)
    plan = ap.plot_plan(m, n, w, scores)
    x, y = torch.from_numpy(c.x).to(dev), torch.from_numpy(c.y).to(dev)
    out = ap.empty_plot(rows, cols, torch.int16 if wide(c) else torch.uint8, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        ap.alignment_plot(x, y, w, scores, out=out)
    for _ in range(warmup):
        call()
    clocks = Clocks(dev.index or 0)
    clocks.start()
    ms = event_times(call, steps, stream, flush)
    host_ms = None
    if host_calls:
        # back-to-back calls with no synchronisation between them: what one
        # call costs a caller when the plot is too small to hide the launch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(host_calls):
            call()
        torch.cuda.synchronize()
        host_ms = (time.perf_counter() - t0) * 1e3 / host_calls
    clk = clocks.stop()
    props = torch.cuda.get_device_properties(dev)
    comb_ms = statistics.mean(ms)
    rec = {"workload": c.name, "m": m, "n": n, "w": w, "scores": "{%d,%d,0}" % tuple(c.scores[:2]),
           "output": "%dx%d %s" % (rows, cols, "uint16" if wide(c) else "uint8"), "steps": steps,
           "ms_per_call": statistics.median(ms), "ms_spread": percentiles(ms),
           "value": float(m) * n * w / (statistics.median(ms) / 1e3), "unit": "cells/s",
           "roofline": comb_roofline(plan, rows, n, w, score, comb_ms, props.multi_processor_count, clk),
           "plan": plan, "clocks": clk}
    if host_ms is not None:
        rec["host_ms_per_call_back_to_back"] = host_ms
        rec["host_calls"] = host_calls
    if rows * cols <= 1 << 20:
        got = out.cpu().numpy().astype(np.int64) & 0xFFFF
        rec["parity"] = {"oracle_full_plot_equal": bool(np.array_equal(got, oracle.plot(c.x, c.y, w, *c.scores[:2])))}
    else:
        ii, jj = synth.below(13, 1, 2000, rows), synth.below(13, 2, 2000, cols)
        got = out[torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy().astype(np.int64) & 0xFFFF
        rec["parity"] = {"oracle_samples_ok": bool(np.array_equal(got, oracle.samples(c.x, c.y, w, ii, jj, *c.scores[:2]))),
                         "oracle_samples": 2000,
                         "golden_digest_ok": golden_check(ap, out, c.name, c.scores[0] * w + 1)}
    del out, flush
    torch.cuda.empty_cache()
    return rec


# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    c = workload(args.workload)
    per = args.ref_seconds or max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    for s in range(args.warmup + args.steps):
        r, k, dt, nth = oracle_rate(c, per, seed=100 + s)
        if s >= args.warmup:
            rates.append((r, k, dt))
    v = statistics.median([r for r, _, _ in rates])
    line = {
        "impl": "reference", "metric": "window-pair cells/sec (m*n*w/s)", "value": v,
        "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # one step is a bounded sample of the workload; the full plot would take
        # m * n * w / value seconds
        "ms_per_step": statistics.median([dt for _, _, dt in rates]) * 1e3,
        "ms_per_full_workload": float(len(c.x)) * len(c.y) * c.w / v * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": describe(c),
        "cpu_baseline": {"value": v, "unit": "cells/s", "cores": cores(), "kind": "oracle",
                         "cpu": cpu_model(),
                         "sample": "%d seeded window pairs per step (O(w^2) DP each), all host cores"
                                   % rates[0][1]},
        "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_record(args, steps, warmup):
    """Many DNA pairs (lengths log-uniform 200..20000, w in {16,32,64,128},
    30% with a planted homology): one batched graph launch per step, against a
    loop of plain calls (one launch per pair) on the same GPU, same outputs."""
    import ctypes
    import numpy as np
    import torch

    import oracle
    import paper_0909_2000_gb300 as ap
    from paper_0909_2000_gb300 import synth

    ap.load(build_if_missing=True)
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    jobs = synth.batch_jobs(0, count=args.batch_jobs)
    gen_s = time.perf_counter() - t0
    # inputs: two concatenated device buffers; outputs: one buffer, rows padded to 32
    xo = np.cumsum([0] + [len(j.x) for j in jobs])
    yo = np.cumsum([0] + [len(j.y) for j in jobs])
    X = torch.from_numpy(np.concatenate([j.x for j in jobs])).to(dev)
    Y = torch.from_numpy(np.concatenate([j.y for j in jobs])).to(dev)
    shapes, oo = [], [0]
    for j in jobs:
        r, c = max(0, len(j.x) - j.w), max(0, len(j.y) - j.w)
        ld = (c + 31) // 32 * 32
        shapes.append((r, c, ld))
        oo.append(oo[-1] + r * ld)
    OUT_P = torch.empty(oo[-1], dtype=torch.uint8, device=dev)
    OUT_B = torch.empty(oo[-1], dtype=torch.uint8, device=dev)

    def views(buf):
        return [buf[oo[k]:oo[k] + r * ld].view(r, ld)[:, :c] if r else buf[:0].view(0, c)
                for k, (r, c, ld) in enumerate(shapes)]
    outs_p, outs_b = views(OUT_P), views(OUT_B)
    xs = [X[xo[k]:xo[k + 1]] for k in range(len(jobs))]
    ys = [Y[yo[k]:yo[k + 1]] for k in range(len(jobs))]
    logical = float(sum(len(j.x) * len(j.y) * j.w for j in jobs))

    # plain form: one ap_alignment_plot call (one launch) per pair
    lib = ap.load()
    sc = ap._scores(ap.LCS)
    st = ap._stream_handle(None)
    calls = [(ctypes.c_void_p(xs[k].data_ptr()), len(jobs[k].x), ctypes.c_void_p(ys[k].data_ptr()),
              len(jobs[k].y), jobs[k].w, ctypes.byref(sc), ctypes.c_void_p(outs_p[k].data_ptr()), 1,
              shapes[k][2]) for k in range(len(jobs))]

    def plain():
        for a in calls:
            rc = lib.ap_alignment_plot(*a, st)
            if rc:
                raise RuntimeError(lib.ap_last_error().decode())

    t0 = time.perf_counter()
    batch = ap.Batch([(xs[k], ys[k], jobs[k].w, ap.LCS, outs_b[k]) for k in range(len(jobs))],
                     autotune=True)
    create_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plain()
        batch.run()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    # the outputs (73.5 GB) are far larger than L2: no flush is needed
    ms_p = event_times(plain, steps, stream)
    ms_b = event_times(batch.run, steps, stream)
    clk = clocks.stop()
    same = bool(torch.equal(OUT_P, OUT_B))
    # oracle spot checks on seeded (job, i, j) samples
    rng = synth.below(5, 1, 300, len(jobs))
    ok, nsamp = True, 0
    for t, k in enumerate(rng):
        r, c, _ = shapes[k]
        if r == 0 or c == 0:
            continue
        ii = synth.below(5, 10 + t, 4, r)
        jj = synth.below(5, 20000 + t, 4, c)
        got = outs_b[k][torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy()
        ok &= bool(np.array_equal(got.astype(np.int64), oracle.samples(jobs[k].x, jobs[k].y, jobs[k].w, ii, jj)))
        nsamp += 4
    info = batch.info()
    batch.close()
    tb, tp = statistics.median(ms_b) / 1e3, statistics.median(ms_p) / 1e3
    rec = {
        "workload": "batch_dna_%d" % len(jobs),
        "jobs": "%d DNA pairs, m and n log-uniform 200..20000, w uniform in {16,32,64,128}, "
                "30%% with one planted homology (length min(m,n)/4, 10%% substitutions)" % len(jobs),
        "output": "every pair's full uint8 plot (%.1f GB)" % (oo[-1] / 1e9), "steps": steps,
        "value": logical / tb, "unit": "cells/s",
        "batched": {"ms": tb * 1e3, "ms_spread": percentiles(ms_b), "cells_per_s": logical / tb, "info": info,
                    "create_s": create_s, "gpu_launches_per_step": 1},
        "plain_loop": {"ms": tp * 1e3, "ms_spread": percentiles(ms_p), "cells_per_s": logical / tp,
                       "note": "one ap_alignment_plot call per pair, same stream",
                       "gpu_launches_per_step": sum(1 for r, c, _ in shapes if r and c)},
        "speedup_batched_vs_plain": tp / tb,
        "parity": {"outputs_identical_to_plain": same, "oracle_samples_ok": ok, "oracle_samples": nsamp},
        "clocks": clk, "gen_s": gen_s,
    }
    del OUT_P, OUT_B, X, Y, outs_p, outs_b, xs, ys
    torch.cuda.empty_cache()
    return rec


def bench_batch(args):
    rec = batch_record(args, args.steps, args.warmup)
    line = {"metric": "window-pair cells/sec (m*n*w/s)", "value": rec["value"], "unit": "cells/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["batched"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": rec["workload"], "jobs": rec["jobs"],
                                            "output": rec["output"]},
            "gpu_launches": args.steps}
    line.update({k: rec[k] for k in ("batched", "plain_loop", "speedup_batched_vs_plain", "parity", "clocks")})
    print(json.dumps(line), flush=True)
    p = rec["parity"]
    return 0 if (p["outputs_identical_to_plain"] and p["oracle_samples_ok"]) else 1


def bench_table1_shape(args):
    """The shape of the paper's Table 1 runs on its largest data set: 80k x 80k,
    w = 100, scores (1, 0, -1/2) as {2,1,0}, vertical step 5 (synthetic DNA
    with planted homologies stands in for the absent sequences).  The paper's
    times for that set are context, not a target: Sea-8 on one 1.83 GHz
    Core2 core 1614 s, MPI on 64 Xeon cores 23 s (Table 1)."""
    import numpy as np
    import torch

    import oracle
    import paper_0909_2000_gb300 as ap
    from paper_0909_2000_gb300 import synth

    ap.load(build_if_missing=True)
    dev = torch.device("cuda", 0)
    c = synth.dna_score_80k_step5(0)
    step = c.step
    x = torch.from_numpy(c.x).to(dev)
    y = torch.from_numpy(c.y).to(dev)
    rows = -(-(len(c.x) - c.w) // step)
    cols = len(c.y) - c.w
    out = ap.empty_plot(rows, cols, torch.uint8, dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ap.alignment_plot_step(x, y, c.w, step, ap.SCORE, out=out)
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ap.alignment_plot_step(x, y, c.w, step, ap.SCORE, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) / 1e3
    ii = synth.below(3, 1, 500, rows)
    jj = synth.below(3, 2, 500, cols)
    got = out[torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy().astype(np.int64)
    want = oracle.samples(c.x, c.y, c.w, ii * step, jj, 2, 1)
    logical = float(len(c.x)) * len(c.y) * c.w / step
    line = {"metric": "window-pair cells/sec (m*n*w/h/s)", "value": logical / t, "unit": "cells/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "score_dna_80k_w100_step5", "m": len(c.x), "n": len(c.y), "w": c.w,
                       "step": step, "scores": "match 2, mismatch 1, gap 0 (the paper's 1, 0, -1/2)",
                       "output": "%d x %d uint8 plot" % (rows, cols)},
            "paper_table1_same_shape_s": {"sea8_1core_core2_1.83GHz": 1614, "mpi_64cores_xeon_3GHz": 23},
            "seconds": t, "oracle_samples_ok": bool(np.array_equal(got, want)),
            "golden_digest_ok": golden_check(ap, out, c.name, 2 * c.w + 1)}
    print(json.dumps(line), flush=True)
    return 0


def serve_record(args, overload_seconds, sustained_seconds, check_requests=12, plain_requests=60):
    """Open-loop Poisson arrivals of DNA dot-plot requests (m, n log-uniform
    1000..200000, w uniform in {32,64,128,256}, dots >= ceil(0.8 w)) into the
    server: first at the offered rate (args.serve_rate) for overload_seconds,
    whose throughput under the backlog is the capacity; then at 70% of that
    capacity for sustained_seconds, with p50/p99 latency; served dots of
    seeded requests against plain calls and the oracle; at 50% of capacity
    for the same time; and a sequential loop of plain dots calls on the same
    kind of requests for comparison."""
    import threading as th

    import numpy as np
    import torch

    import oracle
    import paper_0909_2000_gb300 as ap
    from paper_0909_2000_gb300 import synth

    ap.load(build_if_missing=True)
    torch.cuda.set_device(0)

    def cells(p):
        return float(max(0, len(p.x) - p.w)) * max(0, len(p.y) - p.w) * p.w

    def run(rate, seconds, seed, check=None):
        reqs = synth.serving_requests(seed, rate=rate, duration=seconds)
        srv = ap.Server(mem_budget=64 << 30, max_slots=args.serve_slots)
        tickets = [None] * len(reqs)
        # a seeded set of moderate requests whose dots are kept for checking
        small = [k for k, (_, p) in enumerate(reqs) if cells(p) < 5e11]
        keep = (set(small[int(i)] for i in synth.below(seed, 77, check_requests, len(small)))
                if (check is not None and small) else set())
        t0 = time.perf_counter()

        def submitter():
            for k, (at, p) in enumerate(reqs):
                dt = at - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                tickets[k] = srv.submit(p.x, p.y, p.w, p.threshold, max_dots=1 << 24)

        thr = th.Thread(target=submitter)
        thr.start()
        thr.join()
        statuses = [srv.wait(t, -1) for t in tickets]
        wall = time.perf_counter() - t0
        ndots = 0
        for k, t in enumerate(tickets):
            st, cnt, dots = srv.fetch(t, cap=None if k in keep else 0)
            ndots += cnt
            if k in keep:
                check.append((reqs[k][1], dots))
        stats = srv.stats()
        srv.close()
        total = sum(cells(p) for _, p in reqs)
        return {"rate_req_s": rate, "arrival_seconds": seconds, "requests": len(reqs),
                "offered_cells_per_s": total / seconds, "completed": stats["completed"],
                "ok": sum(1 for s_ in statuses if s_ == ap.AP_OK), "dots": ndots,
                "wall_s": wall, "throughput_cells_per_s": total / wall,
                "latency_p50_ms": stats["latency_p50_ms"], "latency_p99_ms": stats["latency_p99_ms"],
                "latency_max_ms": stats["latency_max_ms"], "peak_device_bytes": stats["peak_device_bytes"],
                "mean_cells_per_request": total / max(1, len(reqs))}

    clocks = Clocks(0)
    clocks.start()
    overload = run(args.serve_rate, overload_seconds, 0)
    capacity = overload["throughput_cells_per_s"]
    sust_rate = max(1.0, 0.7 * capacity / overload["mean_cells_per_request"])
    checked = []
    sustained = run(sust_rate, sustained_seconds, 1, checked)
    # a lighter load: with sharing, a job's latency grows like its solo time
    # / (1 - load), so p99 (the largest jobs) falls steeply with the load
    half = run(max(1.0, 0.5 * capacity / overload["mean_cells_per_request"]), sustained_seconds, 3)
    clk = clocks.stop()
    # served dots against the plain call and the oracle (outside the timing):
    # identical dot lists, every sampled dot's value, and sampled non-dots
    # below the threshold
    dev = torch.device("cuda", 0)
    same, oracle_ok, nsamp = True, True, 0
    for k, (p, dots) in enumerate(checked):
        pd, pc = ap.alignment_dots(torch.from_numpy(p.x).to(dev), torch.from_numpy(p.y).to(dev), p.w,
                                   p.threshold)
        plain = ap.dots_to_numpy(pd, pc)
        same &= bool(np.array_equal(plain, dots))
        rows, cols = max(0, len(p.x) - p.w), max(0, len(p.y) - p.w)
        if rows == 0 or cols == 0:
            continue
        pick = dots[synth.below(9, 2 * k, min(200, len(dots)), len(dots))] if len(dots) else dots[:0]
        ii = synth.below(9, 2 * k + 1, 200, rows)
        jj = synth.below(9, 2 * k + 1000, 200, cols)
        dotset = set(map(tuple, dots[:, :2].tolist()))
        off = np.array([(i, j) for i, j in zip(ii, jj) if (int(i), int(j)) not in dotset], dtype=np.int64)
        if len(pick):
            want = oracle.samples(p.x, p.y, p.w, pick[:, 0], pick[:, 1])
            oracle_ok &= bool(np.array_equal(want, pick[:, 2])) and bool((pick[:, 2] >= p.threshold).all())
            nsamp += len(pick)
        if len(off):
            v = oracle.samples(p.x, p.y, p.w, off[:, 0], off[:, 1])
            oracle_ok &= bool((v < p.threshold).all())
            nsamp += len(off)
    # plain form: the same kind of requests, one ap_alignment_dots call after another
    reqs = synth.serving_requests(2, rate=args.serve_rate, duration=1.0)[:plain_requests]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, p in reqs:
        x = torch.from_numpy(p.x).to(dev)
        y = torch.from_numpy(p.y).to(dev)
        ap.alignment_dots(x, y, p.w, p.threshold)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_rate = sum(cells(p) for _, p in reqs) / plain_s
    return {
        "workload": "serve_dna_poisson",
        "requests": "Poisson arrivals; m, n log-uniform 1000..200000; w uniform in {32,64,128,256}; "
                    "dots >= ceil(0.8 w); device budget 64 GiB, %d slots" % args.serve_slots,
        "value": sustained["throughput_cells_per_s"], "unit": "cells/s",
        "capacity_cells_per_s": capacity,
        "open_loop_at_offered_rate": overload,
        "open_loop_at_sustainable_rate": sustained,
        "sustainable_rate_is": "70% of capacity",
        "open_loop_at_half_capacity": half,
        "offered_over_capacity": overload["offered_cells_per_s"] / capacity,
        "plain_sequential_dots": {"requests": len(reqs), "cells_per_s": plain_rate},
        "served_capacity_over_plain": capacity / plain_rate,
        "parity": {"requests_checked": len(checked), "identical_to_plain_calls": same,
                   "oracle_samples_ok": oracle_ok, "oracle_samples": nsamp},
        "clocks": clk,
    }


def bench_serve(args):
    rec = serve_record(args, args.serve_seconds, max(10.0, args.serve_seconds))
    line = {"metric": "window-pair cells/sec (m*n*w/s)", "value": rec["value"], "unit": "cells/s",
            "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/u16 keys", "data": "synthetic",
            "config": {"workload": rec["workload"], "requests": rec["requests"]}}
    line.update({k: v for k, v in rec.items() if k not in ("workload", "requests", "value", "unit")})
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_dna_4096":
        return bench_batch(args)
    if args.workload == "serve_dna_poisson":
        return bench_serve(args)
    if args.workload == "score_dna_80k_w100_step5":
        return bench_table1_shape(args)

    import numpy as np
    import torch

    import paper_0909_2000_gb300 as ap

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    ap.load(build_if_missing=True)
    c = workload(args.workload)
    dev = torch.device("cuda", local)
    m, n, w = len(c.x), len(c.y), c.w
    score = tuple(c.scores[:2]) == (2, 1)
    scores = ap.SCORE if score else ap.LCS
    rows, cols = ap.plot_shape(m, n, w)
    plan = ap.plot_plan(m, n, w, scores)
    x = torch.from_numpy(c.x).to(dev)
    y = torch.from_numpy(c.y).to(dev)
    out = ap.empty_plot(rows, cols, torch.int16 if wide(c) else torch.uint8, dev)
    thr = c.threshold
    ws = torch.empty(max(ap.plot_dots_workspace_size(rows), 1), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # size the dot buffer once (counting pass), outside the timed region
    ap.alignment_plot(x, y, w, scores, out=out)
    dots = None
    ndots = 0
    if thr is not None:
        _, ndots = ap.plot_dots(out, thr, workspace=ws)
        dots = torch.empty((max(ndots, 1), 3), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    launches_per_step = 1 + (3 if thr is not None else 0)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        ap.alignment_plot(x, y, w, scores, out=out)
        if ev:
            ev[1].record(stream)
        if thr is not None:
            ap.plot_dots(out, thr, dots=dots, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    step_ms, comb_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1)                      # evict L2 (outside the events)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        step((e[0], e[1]))
        e[2].record(stream)
        torch.cuda.synchronize()
        comb_ms.append(e[0].elapsed_time(e[1]))
        step_ms.append(e[0].elapsed_time(e[2]))
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if rank == 0 else None

    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    logical = float(m) * n * w
    value = weak_scaling_value(logical, world, args.steps, total_ms)

    # parity spot-check of this run's output against the oracle (outside timing)
    import oracle
    from paper_0909_2000_gb300 import synth
    ii = synth.below(11, 1, 2000, rows)
    jj = synth.below(11, 2, 2000, cols)
    got = out.cpu().numpy()[ii, jj].astype(np.int64) if rows * cols < (1 << 28) else \
        out[torch.from_numpy(ii).to(dev), torch.from_numpy(jj).to(dev)].cpu().numpy().astype(np.int64)
    want = oracle.samples(c.x, c.y, w, ii, jj, c.scores[0], c.scores[1])
    parity_ok = bool(np.array_equal(got, want))
    # the whole plot's digest against the oracle's stored digest
    golden_ok = golden_check(ap, out, c.name, c.scores[0] * w + 1)
    dev_dots = ap.dots_to_numpy(dots, ndots) if thr is not None else None

    # roofline of the comb kernel (integer ALU)
    comb_cells = float(rows) * (n - 1) * (2 * w if score else w) * (2 if score else 1)
    # 32-bit ops per cell: 6 lane-ops over the lanes of one register (4 or 2)
    alg_ops = comb_cells * LANE_OPS_PER_CELL / plan["strips_per_reg"]
    comb_s = statistics.mean(comb_ms) / 1e3
    achieved = alg_ops / comb_s / 1e12
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak = sms * INT32_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    traffic = profile_traffic("comb/" + c.name)

    del out, ws, flush
    torch.cuda.empty_cache()
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(ap, c, scores, thr, dev, max(10, min(args.steps, 20)), dist, world, dev_dots)

    line = {
        "metric": "window-pair cells/sec (m*n*w/s)",
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("u%d" % plan["lane_bits"]) + (", u16 out" if wide(c) and plan["lane_bits"] == 8 else ""),
        "data": "synthetic", "config": describe(c),
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "comb_kernel (strip comb), %d launch per step" % 1,
                     "peak_basis": "%d SMs x %d int32 lanes/clk x %.0f MHz (max SM clock)"
                                   % (sms, INT32_LANES_PER_SM_CLK, SM_MAX_MHZ),
                     "comb_ms": statistics.mean(comb_ms),
                     "frac_at_measured_clock": (achieved / (sms * INT32_LANES_PER_SM_CLK *
                                                            clk["sm_mhz"] * 1e6 / 1e12)
                                                if clk else None)},
        "plan": plan,
        "physical_cells_per_s": plan["physical_cells"] / comb_s,
        "dots": ndots,
        "parity_samples_ok": parity_ok,
        "parity": {"oracle_samples_ok": parity_ok, "oracle_samples": 2000, "golden_digest_ok": golden_ok},
        "clocks": clk,
        "wall_s": wall,
    }
    if e2e:
        line["e2e"] = e2e
    if world == 1:
        line["roofline"]["peak_probe"] = issue_probe(ap, local, sms)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, k, dt, nth = oracle_rate(c, args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": "cells/s", "cores": nth, "kind": "oracle",
                                "cpu": cpu_model(),
                                "sample": "%d seeded window pairs of this workload, O(w^2) DP each, "
                                          "%.1f s on %d host threads" % (k, dt, nth)}
    if world == 1 and not args.no_workloads and args.workload == "lcs_dna_100k_w100":
        # the other workloads, each on its own after the headline's timing
        from paper_0909_2000_gb300 import synth
        k = max(1, args.workloads_steps)
        others = {}
        t0 = time.perf_counter()
        others["lcs_dna_512_w16"] = plot_record(ap, synth.dna_plot_512(0), max(k, 20), 3, dev, host_calls=2000)
        others["score_protein_20k_w64"] = plot_record(ap, synth.protein_score_20k(0), max(k, 10), 3, dev)
        others["batch_dna_4096"] = batch_record(args, k, 1)
        others["serve_dna_poisson"] = serve_record(args, 4.0, 20.0)
        line["workloads"] = others
        line["workloads_wall_s"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_e2e(ap, c, scores, thr, dev, steps, dist=None, world=1, dev_dots=None):
    """Same metric through the public API from and to host memory:
    ap_alignment_plot_host copies x, y in from pinned host memory, combs the
    plot band by band and copies every band (and the dots) back while the
    next band is combed.  Timed per call, every byte moved inside.  Under
    torchrun every rank runs its own calls between barriers; the step time
    is the slowest rank's and the value counts all ranks' cells.  After the
    timing, the host plot of the last call is checked against the oracle on
    seeded samples, and its dots against the device path's dots."""
    import numpy as np
    import torch

    import oracle
    from paper_0909_2000_gb300 import synth
    m, n, w = len(c.x), len(c.y), c.w
    rows, cols = ap.plot_shape(m, n, w)
    dt = torch.int16 if wide(c) else torch.uint8
    ld = (cols + 31) // 32 * 32          # the device bands' row stride: contiguous copies
    try:
        hx = torch.from_numpy(c.x).pin_memory()
        hy = torch.from_numpy(c.y).pin_memory()
        hout = torch.empty((rows, ld), dtype=dt, pin_memory=True)[:, :cols]
        ok = 1.0
    except RuntimeError:                 # no room to pin the host plot on this rank
        ok = 0.0
    # every rank goes on only if all could pin their buffers (no rank waits alone)
    if -max_over_ranks(-ok, dist, dev) < 1.0:
        return None
    cap = 1 << 22
    dbuf = torch.empty((cap, 3), dtype=torch.int32, pin_memory=True)
    ws = torch.empty(ap.plot_host_workspace_size(m, n, w, scores, hout.element_size(), cap),
                     dtype=torch.uint8, device=dev)

    def call():
        return ap.alignment_plot_host(hx, hy, w, scores, out=hout, threshold=thr, dots_cap=cap,
                                      workspace=ws, dots_buf=dbuf)
    out, dots, count = call()   # warm-up
    ts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        out, dots, count = call()
        ts.append(max_over_ranks((time.perf_counter() - t0) * 1e3, dist, dev) / 1e3)
    t = statistics.median(ts)
    ii, jj = synth.below(17, 1, 2000, rows), synth.below(17, 2, 2000, cols)
    got = hout.numpy()[ii, jj].astype(np.int64) & 0xFFFF
    parity = {"host_plot_oracle_samples_ok": bool(np.array_equal(got, oracle.samples(c.x, c.y, w, ii, jj,
                                                                                      *c.scores[:2]))),
              "oracle_samples": 2000}
    if thr is not None and dev_dots is not None:
        parity["host_dots_equal_device_dots"] = bool(count == len(dev_dots) and np.array_equal(dots, dev_dots))
    return {"value": float(m) * n * w * world / t, "unit": "cells/s", "h2d_bytes_per_step": (m + n) * world,
            "d2h_bytes_per_step": (rows * ld * hout.element_size() + (count or 0) * 12 + 8) * world,
            "ms_per_step": t * 1e3, "steps": steps, "ms_spread": percentiles([v * 1e3 for v in ts]),
            "parity": parity, "api": "ap_alignment_plot_host (band copies overlap the comb)"}


if __name__ == "__main__":
    sys.exit(main())
