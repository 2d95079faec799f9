"""Builds libalnplot.so in-tree for sm_103a with nvcc.

The strip-comb kernel is a template over (lane format, rows per thread,
threads per strip group, score mode).  The compiled variants are listed in
VARIANTS.  Their instantiations are generated into a few translation units
under ``_build/``, and all units compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libalnplot.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _variants():
    """(lane type, key bits, lane bits, rows per thread, threads per strip
    group, nu, mu, padding units, vertical-step layout) of every compiled comb
    kernel.  (nu, mu) is the score blow-up {nu, mu, 0}; (1, 0) is LCS."""
    v = []
    # LCS, 7-bit keys in 8-bit lanes, one thread per strip group: w <= 120
    # (rows in steps of 4, one x word, so that R - w <= 3 padding rows)
    for r in range(8, 121, 4):
        v.append(("U8Lanes", 7, 8, r, 1, 1, 0, 8))
    # LCS, 7-bit keys, a strip group's rows split over 2 or 4 threads
    for g, rs in ((2, range(16, 61, 4)), (4, range(8, 33, 4))):
        for r in rs:
            v.append(("U8Lanes", 7, 8, r, g, 1, 0, 8))
    # {2,1,0}, 7-bit pair keys: w <= 64 on one thread, w <= 120 on two
    for rp in range(4, 65, 4):
        v.append(("U8Lanes", 7, 8, 2 * rp, 1, 2, 1, 4))
    for rp in range(36, 61, 4):
        v.append(("U8Lanes", 7, 8, 2 * rp, 2, 2, 1, 4))
    # LCS, full 8-bit keys in 8-bit lanes: 120 < w <= 254 on 2 or 4 threads
    # (blown-up scores keep 16-bit lanes above w = 120: their values reach nu w)
    v.append(("U8FLanes", 8, 8, 64, 2, 1, 0, 8))
    for r in range(32, 65, 4):
        v.append(("U8FLanes", 8, 8, r, 4, 1, 0, 8))
    # LCS, 9-bit keys in 10-bit lanes (three strips per register), rows split
    # over 4 or 8 threads: 256 < w <= 480 by default, 120 < w on request
    # (measured slower than full 8-bit keys and 16-bit lanes up to w = 256)
    for r in range(33, 97, 3):
        v.append(("U10Lanes", 9, 10, r, 4, 1, 0, 8))
    for r in range(33, 61, 3):
        v.append(("U10Lanes", 9, 10, r, 8, 1, 0, 8))

    # LCS, 15-bit keys in 16-bit lanes, rows split over 2, 4 or 8 threads: w <= 512
    # (4 threads up to 96 rows: w <= 384)
    for g in (2, 4, 8):
        for r in range(16, (97 if g == 4 else 65), 8):
            v.append(("U16Lanes", 15, 16, r, g, 1, 0, 8))
    # {2,1,0}, 15-bit pair keys, 8 threads: w <= 256
    for rp in range(16, 33, 4):
        v.append(("U16Lanes", 15, 16, 2 * rp, 8, 2, 1, 4))
    # other blow-ups {nu, mu, 0} in lowest terms (schemes with a common factor
    # g comb their reduced form and scale the plot by g), nu = 3, 4: w <= 32 on
    # one thread (8-bit lanes), w <= 256 on 8 threads (16-bit lanes)
    for nu, mu in ((3, 1), (3, 2), (4, 1), (4, 3)):
        for rp in (8, 16, 24, 32):
            v.append(("U8Lanes", 7, 8, nu * rp, 1, nu, mu, 8))
        for rp in range(4, 33, 4):
            v.append(("U16Lanes", 15, 16, nu * rp, 8, nu, mu, 4))
    # nu = 5..8: one kernel per nu and row count for every mu (read at run
    # time, mu = -1 here), 16-bit lanes on 8 threads, at most 128 rows a thread
    for nu in (5, 6, 7, 8):
        for rp in range(4, 128 // nu // 4 * 4 + 1, 4):
            v.append(("U16Lanes", 15, 16, nu * rp, 8, nu, -1, 4))
    v = [t + (False,) for t in v]
    # vertical step h > 1 (one x word per unit): LCS w <= 120 and {2,1,0} w <= 120
    # in 8-bit lanes with 7-bit keys
    for r in range(8, 65, 8):
        v.append(("U8Lanes", 7, 8, r, 1, 1, 0, 8, True))
    for r in range(36, 61, 4):
        v.append(("U8Lanes", 7, 8, r, 2, 1, 0, 8, True))
    for rp in range(2, 33, 2):
        v.append(("U8Lanes", 7, 8, 2 * rp, 4, 2, 1, min(4, rp), True))
    # ... LCS 120 < w <= 254 in full 8-bit keys, LCS w <= 512 and {2,1,0}
    # w <= 256 in 16-bit lanes
    v.append(("U8FLanes", 8, 8, 64, 2, 1, 0, 8, True))
    for r in range(32, 65, 4):
        v.append(("U8FLanes", 8, 8, r, 4, 1, 0, 8, True))
    for g in (4, 8):
        for r in range(16, 65, 8):
            v.append(("U16Lanes", 15, 16, r, g, 1, 0, 8, True))
    for rp in range(16, 33, 4):
        v.append(("U16Lanes", 15, 16, 2 * rp, 8, 2, 1, 4, True))
    return v


VARIANTS = _variants()
NUNITS = 12   # translation units for the instantiations

# The bounds-checked debug build (AP_DEBUG_BOUNDS) compiles a few variants
# only, one of each kind of kernel the tests exercise: LCS in 7-bit keys on
# one thread (w 13..16 and 97..100) and two threads, full 8-bit keys on two
# threads, 16-bit lanes on four (64 and 80 rows), 10-bit lanes on four; {2,1,0} on one thread
# and in 16-bit lanes; {3,1,0}; {5,x,0} (the '$' count read at run time); the
# vertical-step layout.
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(HERE, "libalnplot_debug.so")
DEBUG_KINDS = {("U8Lanes", 16, 1, 1, 0, False), ("U8Lanes", 100, 1, 1, 0, False),
               ("U8Lanes", 40, 2, 1, 0, False), ("U8FLanes", 64, 2, 1, 0, False),
               ("U16Lanes", 64, 4, 1, 0, False), ("U16Lanes", 80, 4, 1, 0, False),
               ("U10Lanes", 75, 4, 1, 0, False),
               ("U8Lanes", 48, 1, 2, 1, False), ("U16Lanes", 64, 8, 2, 1, False),
               ("U8Lanes", 24, 1, 3, 1, False), ("U16Lanes", 40, 8, 5, -1, False),
               ("U8Lanes", 16, 1, 1, 0, True)}


def _debug_variants():
    return [v for v in VARIANTS if (v[0], v[3], v[4], v[5], v[6], v[8]) in DEBUG_KINDS]


def _generate(build_dir: str = BUILD, variants=None) -> list[str]:
    variants = VARIANTS if variants is None else variants
    gen = os.path.join(build_dir, "gen")
    os.makedirs(gen, exist_ok=True)
    paths = []
    parts = [variants[k::NUNITS] for k in range(NUNITS)]
    for k, part in enumerate(parts):
        lines = ['#include "variants.h"', "namespace ap {",
                 "extern const Variant kVariants%d[];" % k,
                 "extern const int kNumVariants%d;" % k,
                 "const Variant kVariants%d[] = {" % k]
        for (lanes, kbits, bits, r, g, nu, mu, padu, xr) in part:
            lines.append("    AP_VARIANT(%s, %d, %d, %d, %d, %d, %d, %d, %s)," % (
                lanes, kbits, bits, r, g, nu, mu, padu, "true" if xr else "false"))
        if not part:
            lines.append("    {0, 0, 0, 0, 0, 0, 0, 0, nullptr, nullptr},")
        lines += ["};", "const int kNumVariants%d = %d;" % (k, len(part)), "}  // namespace ap", ""]
        paths.append(_write_if_changed(os.path.join(gen, "variants_%02d.cu" % k), "\n".join(lines)))
    table = ['#include <vector>', '#include <mutex>', '#include "variants.h"', "namespace ap {"]
    for k in range(NUNITS):
        table.append("extern const Variant kVariants%d[]; extern const int kNumVariants%d;" % (k, k))
    table += ["const Variant *variant_table(int *count) {",
              "    static std::vector<Variant> all;",
              "    static std::once_flag once;",
              "    std::call_once(once, [] {"]
    for k in range(NUNITS):
        table.append("        for (int i = 0; i < kNumVariants%d; ++i) all.push_back(kVariants%d[i]);" % (k, k))
    table += ["    });", "    *count = (int)all.size();", "    return all.data();", "}",
              "}  // namespace ap", ""]
    paths.append(_write_if_changed(os.path.join(gen, "variant_table.cu"), "\n".join(table)))
    return paths


def _write_if_changed(path: str, text: str) -> str:
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def _flags(debug: bool = False):
    # AP_KERNEL_DIGEST keys the batch autotuner's persistent cache to these
    # comb kernels
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE,
                   "-DAP_KERNEL_DIGEST=\"comb-%s%s\"" % (kernel_digest(), "-debug" if debug else "")] + \
        (["-DAP_DEBUG_BOUNDS"] if debug else [])


def _deps_digest(debug: bool = False) -> str:
    h = hashlib.sha1()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                h.update(open(p, "rb").read())
    h.update(repr(_debug_variants() if debug else VARIANTS).encode())
    h.update(repr(_flags(debug)).encode())
    return h.hexdigest()


def _code_only(text: str) -> str:
    """C++ source without comments and blank lines: what the compiler sees
    (string literals in comb.cuh hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_digest() -> str:
    """Digest of the strip-comb kernel code (comments left out) and variant
    list, used to tell whether stored profiler counters still describe the
    current kernel."""
    h = hashlib.sha1()
    h.update(_code_only(open(os.path.join(CSRC, "comb.cuh")).read()).encode())
    h.update(repr(VARIANTS).encode())
    return h.hexdigest()[:16]


def _compile(src: str, obj: str, verbose: bool, debug: bool = False) -> None:
    cmd = [NVCC] + _flags(debug) + ["-c", src, "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, r.stdout, r.stderr))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          debug: bool = False) -> str:
    """Compile (if sources changed) and return the path of libalnplot.so, or
    with debug=True of libalnplot_debug.so (bounds checks, a few variants)."""
    bdir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    os.makedirs(bdir, exist_ok=True)
    stamp = os.path.join(bdir, "stamp")
    digest = _deps_digest(debug)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read() == digest:
        return lib
    if shutil.which(NVCC) is None and not os.path.exists(NVCC):
        raise RuntimeError("nvcc not found; the CUDA library cannot be built")
    srcs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    srcs += _generate(bdir, _debug_variants() if debug else None)
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    jobs = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        list(ex.map(lambda so: _compile(so[0], so[1], verbose, debug), zip(srcs, objs)))
    LIB_ = lib
    tmp = LIB_ + ".%d.tmp" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB_)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB_


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
    print("built in %.1f s" % (time.time() - t))
