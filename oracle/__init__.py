"""Plain CPU reference ("oracle") for window-pair alignment plots.

TEST INFRASTRUCTURE ONLY.  The product library never imports, links or runs
anything here.  The users are the tests, ``__graft_entry__.smoke()``, and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The oracle
shares no code with the CUDA path.

The definitions follow Krusche & Tiskin, "Computing alignment plots
efficiently", Section 2.

* ``WLCS(i, j)`` is the LCS length of the w-windows ``x[i:i+w]`` and
  ``y[j:j+w]``.  Equivalently, it is the best alignment score with match 1,
  mismatch 0 and gap 0.
* The plot covers ``0 <= i < m-w`` and ``0 <= j < n-w``.  This is the paper's
  ``{1..m-w} x {1..n-w}``, written 0-based.
* The paper also scores alignments with (match 1, mismatch 0, gap -1/2).  Here
  that scheme is evaluated in integer form as (2, 1, 0).  The optimum is
  ``T = S + w``, where ``S`` is the (1, 0, -1/2) score.
* Each value comes from the textbook dynamic programme (Section 2, the
  alignment dag with score-0 horizontal and vertical edges).  Repeated for
  every window pair, it is the O(m n w^2) method.

``oracle.c`` holds the same recurrence as compiled C, threaded over plot rows
or samples.  The pure-Python functions below restate it for small cases.

``blcs.c`` is a second reference for plots too large for the dynamic
programme: the bit-parallel LCS of Crochemore et al. (2001), the comparison
method of the paper's Section 4, run once per window pair, with scores
{nu, mu, 0} through the blow-up of Section 2.  It is trusted only through
the tests that check it against the dynamic programme and the brute-force
pins.  Both report plot digests (checksum and value histogram) for whole
plots without storing them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "blcs.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LCS = (1, 0)     # (match, mismatch), gap 0
SCORE = (2, 1)   # Section 2's (1, 0, -1/2) scheme, shifted and doubled


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it with gcc."""
    with _lock:
        fresh = (os.path.exists(_LIB_PATH)
                 and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS))
        if force or not fresh:
            tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                                   "-pthread"] + _SRCS + ["-o", tmp])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.oracle_pair_score.restype = i64
        lib.oracle_pair_score.argtypes = [p, i64, p, i64, i32, i32, p]
        lib.oracle_plot.restype = ctypes.c_int
        lib.oracle_plot.argtypes = [p, i64, p, i64, i64, i32, i32, p, i64,
                                    ctypes.c_int]
        lib.oracle_samples.restype = ctypes.c_int
        lib.oracle_samples.argtypes = [p, i64, p, i64, i64, i32, i32, p, p,
                                       i64, p, ctypes.c_int]
        lib.oracle_plot_digest.restype = ctypes.c_int
        lib.oracle_plot_digest.argtypes = [p, i64, p, i64, i64, i32, i32, i64, i32, p,
                                           ctypes.c_int]
        lib.oracle_blcs_plot.restype = ctypes.c_int
        lib.oracle_blcs_plot.argtypes = [p, i64, p, i64, i64, i32, i32, i64, p, i64,
                                         ctypes.c_int]
        lib.oracle_blcs_digest.restype = ctypes.c_int
        lib.oracle_blcs_digest.argtypes = [p, i64, p, i64, i64, i32, i32, i64, i32, p,
                                           ctypes.c_int]
        _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    if isinstance(a, str):
        return np.frombuffer(a.encode("latin-1"), dtype=np.uint8)
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def plot_shape(m: int, n: int, w: int) -> tuple[int, int]:
    """Rows and columns of the plot (Section 2): (m-w) x (n-w), or empty."""
    return max(0, m - w), max(0, n - w)


def pair_score(a, b, match: int = 1, mismatch: int = 0) -> int:
    """Best alignment score of whole strings a, b under (match, mismatch, 0)."""
    a, b = _u8(a), _u8(b)
    row = np.zeros(len(b) + 1, dtype=np.int32)
    return int(_load().oracle_pair_score(a.ctypes.data, len(a), b.ctypes.data,
                                         len(b), match, mismatch,
                                         row.ctypes.data))


def plot(x, y, w: int, match: int = 1, mismatch: int = 0,
         nthreads: int | None = None) -> np.ndarray:
    """Full alignment plot as an int32 array of shape (m-w, n-w)."""
    x, y = _u8(x), _u8(y)
    rows, cols = plot_shape(len(x), len(y), w)
    out = np.zeros((rows, cols), dtype=np.int32)
    if rows and cols:
        rc = _load().oracle_plot(x.ctypes.data, len(x), y.ctypes.data, len(y),
                                 w, match, mismatch, out.ctypes.data, cols,
                                 nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_plot rejected its arguments")
    return out


def samples(x, y, w: int, ii, jj, match: int = 1, mismatch: int = 0,
            nthreads: int | None = None) -> np.ndarray:
    """Plot values at the index pairs (ii[s], jj[s])."""
    x, y = _u8(x), _u8(y)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.zeros(len(ii), dtype=np.int32)
    if len(ii):
        rc = _load().oracle_samples(x.ctypes.data, len(x), y.ctypes.data,
                                    len(y), w, match, mismatch, ii.ctypes.data,
                                    jj.ctypes.data, len(ii), out.ctypes.data,
                                    nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_samples: index outside the plot")
    return out


def step_shape(m: int, n: int, w: int, step: int) -> tuple[int, int]:
    """Shape of the plot of every step-th x-window (Section 3's step h)."""
    return (-(-(m - w) // step) if m > w else 0), max(0, n - w)


def plot_digest(x, y, w: int, match: int = 1, mismatch: int = 0, step: int = 1,
                nbins: int | None = None, nthreads: int | None = None):
    """(checksum, histogram) of the whole plot by the dynamic programme, row r
    being the x-window at r * step, without storing the plot.  nbins defaults
    to match * w + 1 (every possible value)."""
    x, y = _u8(x), _u8(y)
    nbins = match * w + 1 if nbins is None else nbins
    res = np.zeros(1 + nbins, dtype=np.uint64)
    rc = _load().oracle_plot_digest(x.ctypes.data, len(x), y.ctypes.data, len(y), w, match,
                                    mismatch, step, nbins, res.ctypes.data,
                                    nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle_plot_digest rejected its arguments")
    return int(res[0]), res[1:].astype(np.int64)


def _blow(match: int, mismatch: int) -> tuple[int, int]:
    if (match, mismatch) == (1, 0) or (match >= 2 and 1 <= mismatch < match):
        return match, mismatch
    raise ValueError("the bit-parallel reference takes LCS or {nu, mu, 0} with 0 < mu < nu")


def blcs_plot(x, y, w: int, match: int = 1, mismatch: int = 0, step: int = 1,
              nthreads: int | None = None) -> np.ndarray:
    """The plot by bit-parallel LCS of the (blown-up) window pairs."""
    x, y = _u8(x), _u8(y)
    nu, mu = _blow(match, mismatch)
    rows, cols = step_shape(len(x), len(y), w, step)
    out = np.zeros((rows, cols), dtype=np.int32)
    if rows and cols:
        rc = _load().oracle_blcs_plot(x.ctypes.data, len(x), y.ctypes.data, len(y), w, nu, mu,
                                      step, out.ctypes.data, cols, nthreads or default_threads())
        if rc != 0:
            raise ValueError("oracle_blcs_plot rejected its arguments")
    return out


def blcs_digest(x, y, w: int, match: int = 1, mismatch: int = 0, step: int = 1,
                nbins: int | None = None, nthreads: int | None = None):
    """(checksum, histogram) of the whole plot by bit-parallel LCS."""
    x, y = _u8(x), _u8(y)
    nu, mu = _blow(match, mismatch)
    nbins = match * w + 1 if nbins is None else nbins
    res = np.zeros(1 + nbins, dtype=np.uint64)
    rc = _load().oracle_blcs_digest(x.ctypes.data, len(x), y.ctypes.data, len(y), w, nu, mu,
                                    step, nbins, res.ctypes.data, nthreads or default_threads())
    if rc != 0:
        raise ValueError("oracle_blcs_digest rejected its arguments")
    return int(res[0]), res[1:].astype(np.int64)


# ---------------------------------------------------------------------------
# Pure-Python restatements (small inputs only)
# ---------------------------------------------------------------------------

def pair_score_py(a, b, match: int = 1, mismatch: int = 0) -> int:
    """The Section 2 recurrence over the full grid, as plain Python loops."""
    a, b = list(_u8(a)), list(_u8(b))
    D = [[0] * (len(b) + 1) for _ in range(len(a) + 1)]
    for k in range(1, len(a) + 1):
        for l in range(1, len(b) + 1):
            s = match if a[k - 1] == b[l - 1] else mismatch
            D[k][l] = max(D[k - 1][l], D[k][l - 1], D[k - 1][l - 1] + s)
    return D[len(a)][len(b)]


def plot_py(x, y, w: int, match: int = 1, mismatch: int = 0) -> np.ndarray:
    """Full plot with the pure-Python recurrence (tiny inputs only)."""
    x, y = _u8(x), _u8(y)
    rows, cols = plot_shape(len(x), len(y), w)
    out = np.zeros((rows, cols), dtype=np.int32)
    for i in range(rows):
        for j in range(cols):
            out[i, j] = pair_score_py(x[i:i + w], y[j:j + w], match, mismatch)
    return out


# ---------------------------------------------------------------------------
# Outputs derived from a plot (Section 1: dots above a threshold)
# ---------------------------------------------------------------------------

def dots(plot_values: np.ndarray, threshold: int) -> np.ndarray:
    """Window pairs with value >= threshold, in row-major order.

    Returns an (k, 3) int64 array of (i, j, value) rows."""
    ii, jj = np.nonzero(plot_values >= threshold)   # row-major by definition
    return np.stack([ii, jj, plot_values[ii, jj]], axis=1).astype(np.int64)


CHECKSUM_MUL_I = 2654435761
CHECKSUM_MUL_J = 40503


def checksum(plot_values: np.ndarray, row0: int = 0) -> int:
    """sum over cells of value * (i*2654435761 + j*40503 + 1) mod 2^64.

    ``row0`` offsets the row index, so that sums over row bands add up."""
    v = np.asarray(plot_values, dtype=np.uint64)
    if v.size == 0:
        return 0
    rows, cols = v.shape
    i = (np.arange(rows, dtype=np.uint64) + np.uint64(row0))[:, None]
    j = np.arange(cols, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        wgt = i * np.uint64(CHECKSUM_MUL_I) + j * np.uint64(CHECKSUM_MUL_J) + np.uint64(1)
        return int(np.sum(v * wgt, dtype=np.uint64))


def histogram(plot_values: np.ndarray, nbins: int) -> np.ndarray:
    """Count of each plot value 0..nbins-1."""
    return np.bincount(np.asarray(plot_values).ravel(), minlength=nbins)[:nbins]
