"""GB300-native alignment plots (Krusche & Tiskin, arXiv 0909.2000).

A thin ctypes binding over ``libalnplot.so``, whose C ABI is declared in
``include/alnplot.h``.  The functions here only marshal arguments; all
computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  Nothing here falls back to the CPU: if the library
cannot be loaded, every call raises.

    import torch, paper_0909_2000_gb300 as ap
    x = torch.tensor(list(b"ACGT..."), dtype=torch.uint8, device="cuda")
    plot = ap.alignment_plot(x, y, w=100)              # (m-w, n-w) uint8
    dots, count = ap.alignment_dots(x, y, w=100, threshold=80)
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "load", "ApError", "LCS", "SCORE", "plot_shape", "plot_plan", "alignment_plot",
    "alignment_dots", "plot_dots", "plot_checksum", "empty_plot", "version", "alignment_plot_step", "alignment_plot_host", "set_chunk", "set_band_rows", "set_lane_bits", "set_lanes_per_strip", "Batch", "Server", "DOT_DTYPE_FIELDS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

LCS = (1, 0, 0)
SCORE = (2, 1, 0)

AP_OK, AP_E_INVAL, AP_E_UNSUPPORTED, AP_E_NOMEM, AP_E_OVERFLOW = 0, 1, 2, 3, 4
AP_E_CUDA, AP_E_TIMEOUT, AP_E_BUSY, AP_E_CANCELLED = 5, 6, 7, 8
STATUS_NAMES = {0: "AP_OK", 1: "AP_E_INVAL", 2: "AP_E_UNSUPPORTED", 3: "AP_E_NOMEM",
                4: "AP_E_OVERFLOW", 5: "AP_E_CUDA", 6: "AP_E_TIMEOUT", 7: "AP_E_BUSY",
                8: "AP_E_CANCELLED"}
DOT_DTYPE_FIELDS = [("i", "<u4"), ("j", "<u4"), ("value", "<u2"), ("pad", "<u2")]


class ApError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class ap_scores(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32), ("gap", ctypes.c_int32)]


class ap_plan(ctypes.Structure):
    _fields_ = [("lane_bits", ctypes.c_int32), ("strips_per_reg", ctypes.c_int32),
                ("rows_per_lane", ctypes.c_int32), ("lanes_per_strip", ctypes.c_int32),
                ("comb_rows", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("tiles", ctypes.c_int64), ("physical_cells", ctypes.c_int64),
                ("logical_cells", ctypes.c_int64), ("tables", ctypes.c_int32),
                ("smem_per_block", ctypes.c_int32)]


class ap_job(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("m", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("w", ctypes.c_int32), ("scores", ap_scores),
                ("out", ctypes.c_void_p), ("out_elem_bytes", ctypes.c_int32), ("ld", ctypes.c_int64)]


class ap_batch_options(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("lanes_per_strip", ctypes.c_int32)]


class ap_batch_info(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int32), ("jobs", ctypes.c_int32), ("tiles", ctypes.c_int64),
                ("logical_cells", ctypes.c_int64), ("physical_cells", ctypes.c_int64),
                ("tune_ms", ctypes.c_double)]


class ap_request(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("m", ctypes.c_int64), ("y", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("w", ctypes.c_int32), ("scores", ap_scores),
                ("threshold", ctypes.c_int32), ("max_dots", ctypes.c_int64)]


class ap_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("logical_cells", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_max_ms", ctypes.c_double)]


def _declare(lib):
    i32, i64, p, u64p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    sc = ctypes.POINTER(ap_scores)
    lib.ap_version.restype = ctypes.c_char_p
    lib.ap_last_error.restype = ctypes.c_char_p
    lib.ap_status_string.restype = ctypes.c_char_p
    lib.ap_status_string.argtypes = [ctypes.c_int]
    sigs = {
        "ap_set_chunk": [i64],
        "ap_set_lanes_per_strip": [i32],
        "ap_set_band_rows": [i64],
        "ap_set_lane_bits": [i32],
        "ap_plot_shape": [i64, i64, i32, i64p, i64p],
        "ap_plot_plan": [i64, i64, i32, sc, ctypes.POINTER(ap_plan)],
        "ap_alignment_plot": [p, i64, p, i64, i32, sc, p, i32, i64, p],
        "ap_alignment_plot_step": [p, i64, p, i64, i32, sc, i64, p, i32, i64, p],
        "ap_plot_host_workspace_size": [i64, i64, i32, sc, i32, i64, i64p],
        "ap_alignment_plot_host": [p, i64, p, i64, i32, sc, p, i32, i64, i32, p, i64, i64p, p, i64,
                                   p],
        "ap_dots_workspace_size": [i64, i64, i32, sc, i64p],
        "ap_alignment_dots": [p, i64, p, i64, i32, sc, i32, p, i64, i64p, p, i64, p],
        "ap_plot_dots_workspace_size": [i64, i64p],
        "ap_plot_dots": [p, i32, i64, i64, i64, i32, p, i64, i64p, p, i64, p],
        "ap_plot_checksum": [p, i32, i64, i64, i64, i32, u64p, p],
        "ap_plot_dots_noalloc": [p, i32, i64, i64, i64, i32, p, i64, i64p, p],
        "ap_debug_bounds": [ctypes.POINTER(ctypes.c_uint32)],
        "ap_int_issue_probe": [i32, i64, ctypes.POINTER(ctypes.c_double)],
        "ap_batch_create": [ctypes.POINTER(ap_job), i32, ctypes.POINTER(ap_batch_options),
                            ctypes.POINTER(ctypes.c_void_p)],
        "ap_batch_run": [p, p],
        "ap_batch_get_info": [p, ctypes.POINTER(ap_batch_info)],
        "ap_batch_destroy": [p],
        "ap_server_create": [i64, i32, ctypes.POINTER(ctypes.c_void_p)],
        "ap_server_submit": [p, ctypes.POINTER(ap_request), ctypes.POINTER(ctypes.c_uint64)],
        "ap_server_poll": [p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)],
        "ap_server_wait": [p, ctypes.c_uint64, i32],
        "ap_server_fetch": [p, ctypes.c_uint64, p, i64, i64p],
        "ap_server_cancel": [p, ctypes.c_uint64],
        "ap_server_get_stats": [p, ctypes.POINTER(ap_server_stats)],
        "ap_server_destroy": [p],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    return lib


def library_path() -> str:
    """The library to load: $AP_LIB if set (e.g. the bounds-checked debug
    build), else the in-tree libalnplot.so."""
    return os.environ.get("AP_LIB") or os.path.join(_HERE, "libalnplot.so")


def load(build_if_missing: bool = True):
    """Load libalnplot.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and not os.environ.get("AP_LIB"):
                from . import build as _build
                path = _build.build()
            if not os.path.exists(path):
                raise ApError(AP_E_CUDA, "libalnplot.so is missing; run the build")
            _lib = _declare(ctypes.CDLL(path))
    return _lib


def version() -> str:
    return load().ap_version().decode()


def _check(status: int, allow=()):
    if status != AP_OK and status not in allow:
        raise ApError(status, load().ap_last_error().decode())
    return status


def _scores(scores) -> ap_scores:
    s = tuple(scores) if scores is not None else LCS
    if len(s) == 2:
        s = (s[0], s[1], 0)
    return ap_scores(int(s[0]), int(s[1]), int(s[2]))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _dev_u8(t, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.dtype != torch.uint8 or not t.is_cuda or t.dim() != 1 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous 1-D uint8 CUDA tensor" % name)
    return t


def set_chunk(chunk: int) -> None:
    """Force plot columns per tile (0 = automatic); results do not change."""
    _check(load().ap_set_chunk(int(chunk)))


def set_band_rows(rows: int) -> None:
    """Force the band height (plot rows) of the banded calls -- dots, plots
    into host memory, server jobs (0 = automatic); results do not change."""
    _check(load().ap_set_band_rows(int(rows)))


def set_lane_bits(bits: int) -> None:
    """Ask for a lane format of the LCS comb (0 = automatic, 8, 10 or 16
    bits); results do not change."""
    _check(load().ap_set_lane_bits(int(bits)))


def set_lanes_per_strip(groups: int) -> None:
    """Force threads per strip group (0 = automatic); results do not change."""
    _check(load().ap_set_lanes_per_strip(int(groups)))


def plot_shape(m: int, n: int, w: int) -> tuple[int, int]:
    r, c = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ap_plot_shape(m, n, w, ctypes.byref(r), ctypes.byref(c)))
    return r.value, c.value


def plot_plan(m: int, n: int, w: int, scores=LCS) -> dict:
    pl = ap_plan()
    sc = _scores(scores)
    _check(load().ap_plot_plan(m, n, w, ctypes.byref(sc), ctypes.byref(pl)))
    return {f: getattr(pl, f) for f, _ in ap_plan._fields_}


def empty_plot(rows: int, cols: int, dtype, device):
    """Uninitialised (rows, cols) plot whose rows start on 32-element
    boundaries (a view of a (rows, ld) tensor, ld = cols rounded up to 32), so
    that the kernels' row stores fill whole 32-byte sectors."""
    import torch
    ld = (cols + 31) // 32 * 32 if cols else 0
    return torch.empty((rows, ld), dtype=dtype, device=device)[:, :cols]


def alignment_plot(x, y, w: int, scores=LCS, out=None, out_dtype=None, stream=None):
    """Full plot P[i, j] for 0 <= i < m-w, 0 <= j < n-w (uint8 or uint16).

    ``out`` may be a preallocated 2-D CUDA tensor (rows x ld, ld >= cols, or a
    wider view); otherwise one is allocated.  Stream-ordered on ``stream``."""
    import torch
    x, y = _dev_u8(x, "x"), _dev_u8(y, "y")
    rows, cols = plot_shape(x.numel(), y.numel(), w)
    sc = _scores(scores)
    if out is None:
        if out_dtype is None:
            vmax = max(1, sc.match) * w
            out_dtype = torch.uint8 if vmax <= 255 else torch.int16
        out = empty_plot(rows, cols, out_dtype, x.device)
    if out.element_size() not in (1, 2) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor of 8- or 16-bit elements")
    if out.dim() != 2 or out.stride(1) != 1 or out.shape[0] < rows or out.shape[1] < cols:
        raise ValueError("out must be a row-major 2-D tensor of at least %d x %d" % (rows, cols))
    ld = out.stride(0) if rows > 1 else max(cols, out.shape[1])
    _check(load().ap_alignment_plot(ctypes.c_void_p(x.data_ptr()), x.numel(),
                                    ctypes.c_void_p(y.data_ptr()), y.numel(), w,
                                    ctypes.byref(sc), ctypes.c_void_p(out.data_ptr()),
                                    out.element_size(), ld, _stream_handle(stream)))
    return out


def alignment_plot_step(x, y, w: int, step: int, scores=LCS, out=None, out_dtype=None,
                        stream=None):
    """Plot of every ``step``-th x-window: row r is x-window r * step against
    every y-window (Section 3's vertical step h)."""
    import torch
    x, y = _dev_u8(x, "x"), _dev_u8(y, "y")
    m, n = x.numel(), y.numel()
    rows = -(-(m - w) // step) if m > w else 0
    cols = max(0, n - w)
    sc = _scores(scores)
    if out is None:
        if out_dtype is None:
            out_dtype = torch.uint8 if max(1, sc.match) * w <= 255 else torch.int16
        out = empty_plot(rows, cols, out_dtype, x.device)
    if out.dim() != 2 or out.stride(1) != 1 or out.shape[0] < rows or out.shape[1] < cols:
        raise ValueError("out must be a row-major 2-D tensor of at least %d x %d" % (rows, cols))
    ld = out.stride(0) if rows > 1 else max(cols, out.shape[1])
    _check(load().ap_alignment_plot_step(ctypes.c_void_p(x.data_ptr()), m, ctypes.c_void_p(y.data_ptr()),
                                         n, w, ctypes.byref(sc), int(step),
                                         ctypes.c_void_p(out.data_ptr()), out.element_size(), ld,
                                         _stream_handle(stream)))
    return out


def alignment_plot_host(x, y, w: int, scores=LCS, out=None, threshold=None,
                        dots_cap: int = 1 << 22, workspace=None, stream=None, dots_buf=None):
    """Plot into host memory end to end (ap_alignment_plot_host).

    x, y: host uint8 arrays or CPU tensors (pinned copies fastest); ``out``: a
    CPU uint8/16-bit tensor of at least (m-w, n-w), row-major, ideally pinned.
    With a threshold, also returns the dots ((k, 3) int64 numpy array) and
    their count.  ``dots_buf``: an optional reusable host buffer for the raw
    dot records, a contiguous CPU int32 tensor of shape (dots_cap, 3)
    (pinned copies fastest); otherwise one is allocated per call.  Returns
    (out, dots, count)."""
    import numpy as np
    import torch
    xt = torch.as_tensor(np.ascontiguousarray(x, dtype=np.uint8) if not isinstance(x, torch.Tensor) else x)
    yt = torch.as_tensor(np.ascontiguousarray(y, dtype=np.uint8) if not isinstance(y, torch.Tensor) else y)
    m, n = xt.numel(), yt.numel()
    rows, cols = plot_shape(m, n, w)
    sc = _scores(scores)
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.uint8 if max(1, sc.match) * w <= 255 else torch.int16,
                          pin_memory=torch.cuda.is_available())
    lib = load()
    cap = int(dots_cap) if threshold is not None else 0
    need = ctypes.c_int64()
    _check(lib.ap_plot_host_workspace_size(m, n, w, ctypes.byref(sc), out.element_size(), cap,
                                           ctypes.byref(need)))
    if workspace is None:
        workspace = torch.empty(max(need.value, 1), dtype=torch.uint8, device="cuda")
    if dots_buf is not None:
        if (dots_buf.dtype != torch.int32 or dots_buf.dim() != 2 or dots_buf.shape[1] != 3
                or dots_buf.is_cuda or not dots_buf.is_contiguous() or dots_buf.shape[0] < max(cap, 1)):
            raise ValueError("dots_buf must be a contiguous CPU int32 tensor of at least (dots_cap, 3)")
        dbuf = dots_buf.numpy().view(np.uint32)
    else:
        dbuf = np.empty((max(cap, 1), 3), dtype=np.uint32)   # the library fills the first count rows
    cnt = ctypes.c_int64()
    ld = out.stride(0) if rows > 1 else max(cols, out.shape[1])
    st = lib.ap_alignment_plot_host(ctypes.c_void_p(xt.data_ptr()), m, ctypes.c_void_p(yt.data_ptr()), n, w,
                                    ctypes.byref(sc), ctypes.c_void_p(out.data_ptr()), out.element_size(), ld,
                                    int(threshold if threshold is not None else 0),
                                    ctypes.c_void_p(dbuf.ctypes.data), cap,
                                    ctypes.byref(cnt) if threshold is not None else None,
                                    ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                    _stream_handle(stream))
    _check(st)
    if threshold is None:
        return out, None, 0
    k = min(cnt.value, cap)
    d = dbuf[:k].astype(np.int64)
    d[:, 2] &= 0xFFFF          # value, without the pad half-word
    return out, d, cnt.value


def plot_host_workspace_size(m: int, n: int, w: int, scores=LCS, out_elem_bytes: int = 1,
                             dots_cap: int = 0) -> int:
    """Bytes of device workspace alignment_plot_host needs."""
    need = ctypes.c_int64()
    sc = _scores(scores)
    _check(load().ap_plot_host_workspace_size(m, n, w, ctypes.byref(sc), int(out_elem_bytes),
                                              int(dots_cap), ctypes.byref(need)))
    return need.value


def _dots_tensor(count: int, device):
    import torch
    return torch.empty((max(count, 1), 3), dtype=torch.int32, device=device)


def dots_to_numpy(dots, count: int):
    """(count, 3) int64 array of (i, j, value) from a raw ap_dot buffer."""
    import numpy as np
    raw = dots[:count].cpu().numpy().view(np.uint32)
    out = np.zeros((count, 3), dtype=np.int64)
    out[:, 0] = raw[:, 0]
    out[:, 1] = raw[:, 1]
    out[:, 2] = raw[:, 2] & 0xFFFF
    return out


def alignment_dots(x, y, w: int, threshold: int, scores=LCS, cap: int | None = None,
                   dots=None, workspace=None, stream=None):
    """Dots (i, j, value) with P[i, j] >= threshold, row-major.

    Returns (dots, count): ``dots`` is a CUDA int32 tensor of shape (cap, 3)
    holding ap_dot records (i, j, value | pad << 16); ``count`` is the total
    number of qualifying pairs.  Raises ApError(AP_E_OVERFLOW) only if
    ``cap`` was given and is too small; with cap=None the buffer is sized by a
    counting pass first."""
    import torch
    x, y = _dev_u8(x, "x"), _dev_u8(y, "y")
    lib = load()
    sc = _scores(scores)
    need = ctypes.c_int64()
    _check(lib.ap_dots_workspace_size(x.numel(), y.numel(), w, ctypes.byref(sc), ctypes.byref(need)))
    if workspace is None:
        workspace = torch.empty(max(need.value, 1), dtype=torch.uint8, device=x.device)
    cnt = ctypes.c_int64()
    st = _stream_handle(stream)

    def run(buf, capacity, allow):
        return _check(lib.ap_alignment_dots(
            ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(y.data_ptr()), y.numel(), w,
            ctypes.byref(sc), int(threshold),
            ctypes.c_void_p(buf.data_ptr() if buf is not None else 0), capacity,
            ctypes.byref(cnt), ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st), allow)

    if cap is None and dots is None:
        run(None, 0, (AP_E_OVERFLOW,))
        dots = _dots_tensor(cnt.value, x.device)
        run(dots, cnt.value, ())
        return dots, cnt.value
    if dots is None:
        dots = _dots_tensor(cap, x.device)
    run(dots, dots.shape[0] if cap is None else cap, ())
    return dots, cnt.value


def plot_dots_workspace_size(rows: int) -> int:
    need = ctypes.c_int64()
    _check(load().ap_plot_dots_workspace_size(rows, ctypes.byref(need)))
    return need.value


def plot_dots(plot, threshold: int, cap: int | None = None, dots=None, workspace=None,
              stream=None):
    """Dots of an existing device plot (same order and overflow rule as
    alignment_dots).  Returns (dots, count)."""
    import torch
    lib = load()
    rows, cols = plot.shape
    if workspace is None:
        workspace = torch.empty(max(plot_dots_workspace_size(rows), 1), dtype=torch.uint8,
                                device=plot.device)
    cnt = ctypes.c_int64()
    st = _stream_handle(stream)

    def run(buf, capacity, allow):
        return _check(lib.ap_plot_dots(ctypes.c_void_p(plot.data_ptr()), plot.element_size(), rows,
                                       cols, plot.stride(0) if rows > 1 else cols, int(threshold),
                                       ctypes.c_void_p(buf.data_ptr() if buf is not None else 0),
                                       capacity, ctypes.byref(cnt),
                                       ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st),
                      allow)

    if dots is None:
        if cap is None:
            run(None, 0, (AP_E_OVERFLOW,))
            cap = cnt.value
        dots = _dots_tensor(cap, plot.device)
    run(dots, dots.shape[0] if cap is None else cap, ())
    return dots, cnt.value


PLOT_DOTS_NOALLOC_MAX_ROWS = 262144


def plot_dots_noalloc(plot, threshold: int, dots, cap: int | None = None, stream=None):
    """Dots of a device plot through ap_plot_dots_noalloc, which takes no
    workspace and allocates no device memory (its scratch is a fixed array in
    the library, for plots of at most PLOT_DOTS_NOALLOC_MAX_ROWS rows).

    ``dots`` is the caller's output buffer (CUDA int32 tensor of shape
    (capacity, 3)).  Returns (dots, count); raises ApError(AP_E_OVERFLOW) if
    the buffer is too small (the count is still reported on the error)."""
    import torch
    if plot.dim() != 2 or not plot.is_cuda or plot.element_size() not in (1, 2):
        raise ValueError("plot must be a 2-D CUDA tensor of 8- or 16-bit elements")
    rows, cols = plot.shape
    if cols > 1 and plot.stride(1) != 1:
        raise ValueError("plot rows must be contiguous (stride(1) == 1)")
    if (not isinstance(dots, torch.Tensor) or dots.dtype != torch.int32 or dots.dim() != 2
            or dots.shape[1] != 3 or not dots.is_contiguous() or dots.device != plot.device):
        raise ValueError("dots must be a contiguous (N, 3) int32 CUDA tensor on the plot's device")
    capacity = dots.shape[0] if cap is None else int(cap)
    if not 0 <= capacity <= dots.shape[0]:
        raise ValueError("cap = %d outside 0..%d (the dot buffer's rows)" % (capacity, dots.shape[0]))
    cnt = ctypes.c_int64()
    status = load().ap_plot_dots_noalloc(ctypes.c_void_p(plot.data_ptr()), plot.element_size(), rows,
                                         cols, plot.stride(0) if rows > 1 else cols, int(threshold),
                                         ctypes.c_void_p(dots.data_ptr()), capacity,
                                         ctypes.byref(cnt), _stream_handle(stream))
    if status != AP_OK:
        err = ApError(status, load().ap_last_error().decode())
        err.count = cnt.value
        raise err
    return dots, cnt.value


def debug_bounds() -> int:
    """Bounds-check violation bits since the last call (debug builds only;
    raises ApError(AP_E_UNSUPPORTED) in other builds)."""
    f = ctypes.c_uint32()
    _check(load().ap_debug_bounds(ctypes.byref(f)))
    return f.value


def int_issue_probe(kind: int, iters: int) -> float:
    """32-bit lane operations per second of the integer issue probe (kind 0:
    three-input logic, 1: multiply-add, 2: both alternately) on the current
    device; see ap_int_issue_probe."""
    r = ctypes.c_double()
    _check(load().ap_int_issue_probe(int(kind), int(iters), ctypes.byref(r)))
    return r.value


def plot_checksum(plot, nbins: int, stream=None):
    """(checksum, histogram[nbins]) of a device plot, computed on the GPU."""
    import torch
    rows, cols = plot.shape
    res = torch.zeros(1 + nbins, dtype=torch.int64, device=plot.device)
    _check(load().ap_plot_checksum(ctypes.c_void_p(plot.data_ptr()), plot.element_size(), rows, cols,
                                   plot.stride(0) if rows > 1 else cols, nbins,
                                   ctypes.cast(ctypes.c_void_p(res.data_ptr()), ctypes.POINTER(ctypes.c_uint64)),
                                   _stream_handle(stream)))
    r = res.cpu().numpy().view("uint64")
    return int(r[0]), r[1:].astype("int64")


class Batch:
    """Many plot jobs run as one CUDA graph of persistent comb kernels
    (ap_batch_create / ap_batch_run / ap_batch_destroy).

    ``jobs``: list of (x, y, w, scores, out) with x, y 1-D uint8 CUDA tensors
    and ``out`` a row-major 8- or 16-bit CUDA tensor of at least (m-w, n-w).
    The tensors must stay alive and in place while the batch is used."""

    def __init__(self, jobs, autotune: bool = False, chunk: int = 0, lanes_per_strip: int = 0):
        lib = load()
        self._keep = []
        arr = (ap_job * max(1, len(jobs)))()
        for k, (x, y, w, scores, out) in enumerate(jobs):
            x, y = _dev_u8(x, "x"), _dev_u8(y, "y")
            rows = out.shape[0]
            arr[k] = ap_job(x.data_ptr(), x.numel(), y.data_ptr(), y.numel(), int(w), _scores(scores),
                            out.data_ptr(), out.element_size(),
                            out.stride(0) if rows > 1 else max(out.shape[1], 1))
            self._keep.append((x, y, out))
        opt = ap_batch_options(1 if autotune else 0, int(chunk), int(lanes_per_strip))
        h = ctypes.c_void_p()
        _check(lib.ap_batch_create(arr, len(jobs), ctypes.byref(opt), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(load().ap_batch_run(self._h, _stream_handle(stream)))

    def info(self) -> dict:
        inf = ap_batch_info()
        _check(load().ap_batch_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in ap_batch_info._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().ap_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Dot-plot server (ap_server_*): requests carry host sequences; results
    come back as (k, 3) int64 arrays of (i, j, value), row-major."""

    def __init__(self, mem_budget: int, max_slots: int = 8):
        h = ctypes.c_void_p()
        _check(load().ap_server_create(int(mem_budget), int(max_slots), ctypes.byref(h)))
        self._h = h
        self._max_dots = {}

    def submit(self, x, y, w: int, threshold: int, scores=LCS, max_dots: int = 1 << 22) -> int:
        import numpy as np
        x = np.ascontiguousarray(x, dtype=np.uint8)
        y = np.ascontiguousarray(y, dtype=np.uint8)
        req = ap_request(x.ctypes.data, len(x), y.ctypes.data, len(y), int(w), _scores(scores),
                         int(threshold), int(max_dots))
        t = ctypes.c_uint64()
        _check(load().ap_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._max_dots[t.value] = int(max_dots)
        return t.value

    def poll(self, ticket: int) -> int:
        st = ctypes.c_int()
        _check(load().ap_server_poll(self._h, ticket, ctypes.byref(st)))
        return st.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        """The job's final status (AP_OK, AP_E_OVERFLOW, ...) or AP_E_TIMEOUT."""
        return load().ap_server_wait(self._h, ticket, int(timeout_ms))

    def fetch(self, ticket: int, cap: int | None = None):
        """(status, count, dots) for a finished job; dots is an (k, 3) int64
        array with k = min(count, the job's max_dots, cap)."""
        import numpy as np
        lib = load()
        cnt = ctypes.c_int64()
        held = self._max_dots.get(ticket, 1 << 22)
        cap = held if cap is None else min(cap, held)
        buf = np.empty((max(cap, 1), 3), dtype=np.uint32)
        st = lib.ap_server_fetch(self._h, ticket, buf.ctypes.data, cap, ctypes.byref(cnt))
        if st not in (AP_OK, AP_E_OVERFLOW, AP_E_CANCELLED, AP_E_CUDA):
            raise ApError(st, lib.ap_last_error().decode())
        self._max_dots.pop(ticket, None)
        k = min(cnt.value, cap)
        out = buf[:k].astype(np.int64)
        out[:, 2] &= 0xFFFF        # value, without the pad half-word
        return st, cnt.value, out

    def cancel(self, ticket: int) -> None:
        _check(load().ap_server_cancel(self._h, ticket))

    def stats(self) -> dict:
        st = ap_server_stats()
        _check(load().ap_server_get_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ap_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().ap_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
