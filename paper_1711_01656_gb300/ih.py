"""Python binding of the C ABI in include/ih.h (ctypes; argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers
are torch CUDA tensors; streams default to torch's current stream.  Every
step of the integral-histogram path runs in the CUDA library ``libih.so``:
this module computes nothing, and it raises if the library is missing
rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libih.so")

IH_OK, IH_EINVAL, IH_ENOMEM, IH_EBUDGET, IH_ECUDA, IH_ETIMEOUT, IH_ENOTBUILT, IH_ETOOBIG, IH_ECANCELLED = range(9)
IH_BIN_UNIFORM8, IH_BIN_INDEX = 0, 1
IH_INPUT_PLANES, IH_INPUT_RGB_FEATURES = 0, 1
IH_LAYOUT_BIN_MAJOR, IH_LAYOUT_SLAB, IH_LAYOUT_RECORD = 0, 1, 2
IH_K_EPANECHNIKOV, IH_K_MANHATTAN, IH_K_WEDDING_CAKE = 0, 1, 2
IH_NORMALIZE = 1


def IH_LAYERS(n):
    """flags field of ih_query_weighted: wedding-cake layers (1..64; 0 means 4)."""
    return (int(n) & 0xFF) << 8

STATUS_NAMES = {0: "IH_OK", 1: "IH_EINVAL", 2: "IH_ENOMEM", 3: "IH_EBUDGET", 4: "IH_ECUDA",
                5: "IH_ETIMEOUT", 6: "IH_ENOTBUILT", 7: "IH_ETOOBIG", 8: "IH_ECANCELLED"}

# The exported C symbols (include/ih.h), checked by the test suite.
C_SYMBOLS = ("ih_create", "ih_build", "ih_query_rects", "ih_query_weighted", "ih_destroy",
             "ih_release", "ih_sync", "ih_info", "ih_export", "ih_export_moments", "ih_features",
             "ih_profile_read", "ih_launch_count", "ih_last_error", "ih_batch_create", "ih_batch_run",
             "ih_batch_destroy", "ih_autotune", "ih_server_create", "ih_server_submit", "ih_server_poll",
             "ih_server_drain", "ih_server_clock", "ih_server_destroy", "ih_build_counts_static",
             "ih_match_window", "ih_accumulate", "ih_local_median", "ih_phog_build", "ih_phog_descriptors",
             "ih_phog_match", "ih_profile_select", "ih_query", "ih_canny_edges", "ih_server_cancel", "ih_memory_used", "ih_build_mma", "ih_tune_set", "ih_wait_selftest")
IH_BATCH_GRAPH, IH_BATCH_AUTOTUNE, IH_BATCH_PERSISTENT = 1, 2, 4
IH_CFG_PROFILE = 1


class IHError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ih_channel(ctypes.Structure):
    _fields_ = [("bins", ctypes.c_int32), ("mode", ctypes.c_int32)]


class ih_frame(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int32), ("width", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("input", ctypes.c_int32), ("chan", ctypes.POINTER(ih_channel)),
                ("d_pixels", ctypes.c_void_p), ("pitch_bytes", ctypes.c_int64),
                ("weighted_channel", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("moment_bits", ctypes.c_int32)]


class ih_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64),
                ("flags", ctypes.c_uint32)]


class ih_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class ih_frame_info(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int32), ("width", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("total_bins", ctypes.c_int32), ("weighted_channel", ctypes.c_int32),
                ("weighted_bins", ctypes.c_int32), ("pitch_elems", ctypes.c_int64),
                ("count_bytes", ctypes.c_int64), ("moment_bytes", ctypes.c_int64),
                ("tile_rows", ctypes.c_int32), ("tile_cols", ctypes.c_int32)]


class ih_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("max_inflight", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class ih_request(ctypes.Structure):
    _fields_ = [("tracker", ctypes.c_int32), ("frame", ih_frame), ("chan", ih_channel * 16),
                ("d_rects", ctypes.c_void_p), ("n_rects", ctypes.c_int64), ("d_rect_out", ctypes.c_void_p),
                ("d_windows", ctypes.c_void_p), ("n_windows", ctypes.c_int64), ("d_weighted_out", ctypes.c_void_p),
                ("weighted_flags", ctypes.c_uint32), ("user", ctypes.c_uint64)]


class ih_completion(ctypes.Structure):
    _fields_ = [("user", ctypes.c_uint64), ("status", ctypes.c_int32), ("handle", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ih_batch_queries(ctypes.Structure):
    _fields_ = [("d_rects", ctypes.c_void_p), ("rects", ctypes.POINTER(ctypes.c_int64)),
                ("d_rect_out", ctypes.c_void_p), ("d_windows", ctypes.c_void_p),
                ("windows", ctypes.POINTER(ctypes.c_int64)), ("d_weighted_out", ctypes.c_void_p),
                ("kernel", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libih.so (built by __graft_entry__.build()); raise if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("libih.so not found at %s: build it with __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "ih_create": ([ctypes.POINTER(ih_config), ctypes.POINTER(p)], i32),
            "ih_build": ([p, ctypes.POINTER(ih_frame), i32, ctypes.POINTER(i32), p], i32),
            "ih_query_rects": ([p, i32, p, i64, p, p], i32),
            "ih_query_weighted": ([p, i32, p, i64, u32, u32, p, p], i32),
            "ih_query": ([p, i32, p, i64, p, p, i64, u32, u32, p, p], i32),
            "ih_match_window": ([p, i32, i32, i32, p, i32, i32, p, p, p], i32),
            "ih_accumulate": ([p, i32, i32, i32, p], i32),
            "ih_profile_select": ([p, p, i32], i32),
            "ih_phog_build": ([p, p, i32, i32, i64, i32, i32, ctypes.POINTER(i32), p], i32),
            "ih_canny_edges": ([p, p, i32, i32, i64, i32, i32, p, i64, p], i32),
            "ih_phog_descriptors": ([p, i32, i32, p, i64, p, p], i32),
            "ih_phog_match": ([p, i32, i32, p, i32, i32, p, p, p], i32),
            "ih_local_median": ([p, i32, i32, i32, i32, i32, p, p], i32),
            "ih_destroy": ([p], i32),
            "ih_release": ([p, i32, p], i32),
            "ih_sync": ([p, p], i32),
            "ih_info": ([p, i32, ctypes.POINTER(ih_frame_info)], i32),
            "ih_export": ([p, i32, p, p], i32),
            "ih_export_moments": ([p, i32, i32, p, p], i32),
            "ih_features": ([p, p, i32, i32, i64, p, p], i32),
            "ih_profile_read": ([p, ctypes.POINTER(ih_kernel_stat), i32, ctypes.POINTER(i32), i32], i32),
            "ih_launch_count": ([p], i64),
            "ih_memory_used": ([p], ctypes.c_uint64),
            "ih_build_mma": ([p, p, ctypes.POINTER(i32), p], i32),
            "ih_tune_set": ([p, p, i32, i32], i32),
            "ih_wait_selftest": ([p, i32, p], i32),
            "ih_last_error": ([p], ctypes.c_char_p),
            "ih_build_counts_static": ([p, i32, i32, i64, i32, i32, p, i64, p], i32),
            "ih_batch_create": ([p, ctypes.POINTER(ih_frame), i32, ctypes.POINTER(ih_batch_queries), u32,
                                 ctypes.POINTER(p), ctypes.POINTER(i32)], i32),
            "ih_batch_run": ([p, p], i32),
            "ih_batch_destroy": ([p], i32),
            "ih_autotune": ([p, ctypes.POINTER(ih_frame), p], i32),
            "ih_server_create": ([p, ctypes.POINTER(ih_server_config), ctypes.POINTER(p)], i32),
            "ih_server_submit": ([p, ctypes.POINTER(ih_request)], i32),
            "ih_server_poll": ([p, ctypes.POINTER(ih_completion), i32, i32], i32),
            "ih_server_drain": ([p], i32),
            "ih_server_cancel": ([p, ctypes.c_uint64], i32),
            "ih_server_clock": ([p], ctypes.c_double),
            "ih_server_destroy": ([p], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(ctx, status):
    if status != IH_OK:
        msg = load_library().ih_last_error(ctx).decode() if ctx else ""
        raise IHError(status, msg)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


# ---------------------------------------------------------------- contexts

def ih_create(device: int = 0, hbm_budget_bytes: int = 0, flags: int = 0):
    lib = load_library()
    cfg = ih_config(int(device), int(hbm_budget_bytes), int(flags))
    out = ctypes.c_void_p()
    st = lib.ih_create(ctypes.byref(cfg), ctypes.byref(out))
    if st != IH_OK:
        raise IHError(st, "ih_create(device=%d)" % device)
    return out


def ih_destroy(ctx):
    _check(None, load_library().ih_destroy(ctx))


class Frame:
    """One frame to build: `pixels` is a uint8 CUDA tensor of shape (P, H, W)
    (P planes; rows may be padded: stride(1) is the row pitch); `channels` a
    list of (bins, mode) pairs, one per binned channel."""

    def __init__(self, pixels, channels, input=IH_INPUT_PLANES, weighted_channel=-1,
                 layout=IH_LAYOUT_BIN_MAJOR, moment_bits=64):
        if pixels.dtype.itemsize != 1 or pixels.dim() != 3 or not pixels.is_cuda:
            raise ValueError("pixels must be a (planes, H, W) uint8 CUDA tensor")
        planes, h, w = pixels.shape
        pitch = pixels.stride(1) if h > 1 else w
        ok = (pixels.stride(2) == 1 or w == 1) and pitch >= w and (planes == 1 or pixels.stride(0) == h * pitch)
        if not ok:
            pixels = pixels.contiguous()
            pitch = w
        self.pixels = pixels
        self.pitch = pitch
        self.channels = [(int(b), int(m)) for b, m in channels]
        self.input = int(input)
        self.weighted_channel = int(weighted_channel)
        self.layout = int(layout)
        self.moment_bits = int(moment_bits)

    def _c(self):
        arr = (ih_channel * len(self.channels))(*[ih_channel(b, m) for b, m in self.channels])
        f = ih_frame(self.pixels.shape[1], self.pixels.shape[2], len(self.channels), self.input,
                     ctypes.cast(arr, ctypes.POINTER(ih_channel)), self.pixels.data_ptr(),
                     self.pitch, self.weighted_channel, self.layout, self.moment_bits)
        return f, arr


def ih_build(ctx, frames, stream=None):
    """Build each Frame; returns the list of handles."""
    if isinstance(frames, Frame):
        frames = [frames]
    cs = [f._c() for f in frames]
    arr = (ih_frame * len(cs))(*[c[0] for c in cs])
    handles = (ctypes.c_int32 * len(cs))()
    _check(ctx, load_library().ih_build(ctx, arr, len(cs), handles, _stream(stream)))
    return list(handles)


def ih_build_mma(ctx, frame, stream=None):
    """The count build with tensor-core tiles (bin-major planes, no moment
    planes): returns the frame's handle."""
    cf, _keep = frame._c()
    out = ctypes.c_int32(-1)
    _check(ctx, load_library().ih_build_mma(ctx, ctypes.byref(cf), ctypes.byref(out), _stream(stream)))
    return out.value


def ih_query_rects(ctx, handle, rects, out, stream=None):
    """rects: (n, 4) int32 CUDA tensor; out: (n, B) int32 CUDA tensor."""
    n = 0 if rects is None else rects.shape[0]
    _check(ctx, load_library().ih_query_rects(ctx, int(handle), _ptr(rects), n, _ptr(out), _stream(stream)))
    return out


def ih_match_window(ctx, handle, bin0, nbins, target, win_h, win_w, search, out, stream=None):
    """City-block distance map (Eq. 2.22, p = 1) of every win_h x win_w window
    with its top-left pixel in search = (sr0, sc0, sr1, sc1) against `target`
    (nbins int32 CUDA tensor) over bins bin0..bin0+nbins-1; out: int32 CUDA
    tensor of (sr1-sr0+1) x (sc1-sc0+1)."""
    s = (ctypes.c_int32 * 4)(*[int(x) for x in search])
    _check(ctx, load_library().ih_match_window(ctx, int(handle), int(bin0), int(nbins), _ptr(target), int(win_h),
                                               int(win_w), s, _ptr(out), _stream(stream)))
    return out


PHOG_BINS = 9


def phog_descriptor_len(levels):
    return PHOG_BINS * sum(4 ** l for l in range(int(levels) + 1))


def _rows(gray):
    """(tensor, row pitch) of an (H, W) uint8 CUDA tensor whose rows may be strided."""
    h, w = gray.shape
    if gray.stride(1) == 1:
        return gray, gray.stride(0)
    return gray.contiguous(), w


IH_CANNY_MAX_THRESHOLD = 1024


def ih_canny_edges(ctx, gray, tau_low, tau_high, out, stream=None):
    """Algorithm 2 step 1, Canny's detector, on a (H, W) uint8 CUDA tensor:
    writes 1 on edge pixels and 0 elsewhere into out ((H, W) uint8 CUDA
    tensor, rows may be strided)."""
    h, w = gray.shape
    gray, pitch = _rows(gray)
    if out.element_size() != 1 or tuple(out.shape) != (h, w) or out.stride(1) != 1:
        raise ValueError("out must be an (H, W) uint8 tensor with unit column stride")
    _check(ctx, load_library().ih_canny_edges(ctx, _ptr(gray), int(h), int(w), int(pitch), int(tau_low),
                                              int(tau_high), _ptr(out), int(out.stride(0)), _stream(stream)))
    return out


def ih_phog_build(ctx, gray, tau_low, tau_high, stream=None):
    """Algorithm 2 steps 1-4 on a (H, W) uint8 CUDA tensor (rows may be
    strided), with Canny thresholds tau_low <= tau_high: returns the handle of
    the 9-bin magnitude-weighted orientation integral histogram."""
    h, w = gray.shape
    gray, pitch = _rows(gray)
    out = ctypes.c_int32(-1)
    _check(ctx, load_library().ih_phog_build(ctx, _ptr(gray), int(h), int(w), int(pitch), int(tau_low),
                                             int(tau_high), ctypes.byref(out), _stream(stream)))
    return out.value


def ih_phog_descriptors(ctx, handle, levels, windows, out, stream=None):
    """windows: (n, 4) int32 CUDA tensor; out: (n, 9 * sum 4^l) int64 CUDA tensor."""
    n = 0 if windows is None else windows.shape[0]
    _check(ctx, load_library().ih_phog_descriptors(ctx, int(handle), int(levels), _ptr(windows), n, _ptr(out),
                                                   _stream(stream)))
    return out


def ih_phog_match(ctx, handle, levels, target, win_h, win_w, search, out, stream=None):
    """Pyramid match kernel map (Eq. 2.24) of `target` (int64 descriptor,
    CUDA) against every win_h x win_w window with top-left pixel in search."""
    sr = (ctypes.c_int32 * 4)(*[int(x) for x in search])
    _check(ctx, load_library().ih_phog_match(ctx, int(handle), int(levels), _ptr(target), int(win_h), int(win_w),
                                             sr, _ptr(out), _stream(stream)))
    return out


def ih_accumulate(ctx, dst, add=-1, sub=-1, stream=None):
    """Joint integral histogram update (Algorithm 4): counts of dst += add - sub."""
    _check(ctx, load_library().ih_accumulate(ctx, int(dst), int(add), int(sub), _stream(stream)))


def ih_local_median(ctx, handle, bin0, nbins, m, n, out, stream=None):
    """Lower-median bin of every pixel's m x n box over bins bin0..bin0+nbins-1;
    out: (H, W) int32 CUDA tensor (-1 where the box holds no count)."""
    _check(ctx, load_library().ih_local_median(ctx, int(handle), int(bin0), int(nbins), int(m), int(n), _ptr(out),
                                               _stream(stream)))
    return out


def ih_query_weighted(ctx, handle, windows, out, kernel=IH_K_EPANECHNIKOV, flags=0, stream=None):
    """windows: (n, 4) int32 CUDA tensor; out: (n, B_w) float32 CUDA tensor."""
    n = 0 if windows is None else windows.shape[0]
    _check(ctx, load_library().ih_query_weighted(ctx, int(handle), _ptr(windows), n, int(kernel),
                                                 int(flags), _ptr(out), _stream(stream)))
    return out


def ih_query(ctx, handle, rects=None, rect_out=None, windows=None, weighted_out=None, kernel=IH_K_EPANECHNIKOV,
             flags=0, stream=None):
    """ih_query_rects and ih_query_weighted of one frame in one call and one
    launch; either part may be None."""
    nr = 0 if rects is None else rects.shape[0]
    nw = 0 if windows is None else windows.shape[0]
    _check(ctx, load_library().ih_query(ctx, int(handle), _ptr(rects), nr, _ptr(rect_out), _ptr(windows), nw,
                                        int(kernel), int(flags), _ptr(weighted_out), _stream(stream)))
    return rect_out, weighted_out


def ih_release(ctx, handle, stream=None):
    _check(ctx, load_library().ih_release(ctx, int(handle), _stream(stream)))


def ih_sync(ctx, stream=None):
    _check(ctx, load_library().ih_sync(ctx, _stream(stream)))


def ih_info(ctx, handle):
    info = ih_frame_info()
    _check(ctx, load_library().ih_info(ctx, int(handle), ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in ih_frame_info._fields_}


def ih_export(ctx, handle, out, stream=None):
    """out: (B, H, W) int32 CUDA tensor."""
    _check(ctx, load_library().ih_export(ctx, int(handle), _ptr(out), _stream(stream)))
    return out


def ih_export_moments(ctx, handle, plane, out, stream=None):
    """out: (B_w, H, W) int64 CUDA tensor; plane 0..3 = weights c, r, c^2, r^2."""
    _check(ctx, load_library().ih_export_moments(ctx, int(handle), int(plane), _ptr(out), _stream(stream)))
    return out


def ih_features(ctx, rgb, out, stream=None):
    """rgb: (3, H, W) uint8 CUDA tensor; out: (7, H, W) uint8 CUDA tensor."""
    rgb = rgb.contiguous()
    _check(ctx, load_library().ih_features(ctx, _ptr(rgb), rgb.shape[1], rgb.shape[2], rgb.shape[2],
                                           _ptr(out), _stream(stream)))
    return out


def ih_profile_read(ctx, reset=True):
    """{kernel name: (launches, total_ms)} of a context created with IH_CFG_PROFILE."""
    arr = (ih_kernel_stat * 64)()
    n = ctypes.c_int32()
    _check(ctx, load_library().ih_profile_read(ctx, arr, 64, ctypes.byref(n), int(bool(reset))))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def ih_profile_select(ctx, names=()):
    """Time only the named kernels (ih_profile_read names); () = all."""
    arr = (ctypes.c_char_p * max(1, len(names)))(*[n.encode() for n in names])
    _check(ctx, load_library().ih_profile_select(ctx, ctypes.cast(arr, ctypes.c_void_p), len(names)))


def ih_batch_create(ctx, frames, rects=None, rect_counts=None, rect_out=None, windows=None, window_counts=None,
                    weighted_out=None, kernel=IH_K_EPANECHNIKOV, flags=0, batch_flags=IH_BATCH_GRAPH):
    """Plan a batch of Frames (see include/ih.h).  rects / windows: (sum, 4)
    int32 CUDA tensors with per-frame counts; outputs: flat CUDA tensors
    holding each frame's block in frame order.  Returns (batch, handles)."""
    cs = [f._c() for f in frames]
    arr = (ih_frame * len(cs))(*[c[0] for c in cs])
    handles = (ctypes.c_int32 * len(cs))()
    q = None
    keep = []
    if rects is not None or windows is not None:
        rc = (ctypes.c_int64 * len(cs))(*(rect_counts or [0] * len(cs)))
        wc = (ctypes.c_int64 * len(cs))(*(window_counts or [0] * len(cs)))
        keep += [rc, wc]
        q = ih_batch_queries(_ptr(rects).value if rects is not None else None, rc,
                             _ptr(rect_out).value if rect_out is not None else None,
                             _ptr(windows).value if windows is not None else None, wc,
                             _ptr(weighted_out).value if weighted_out is not None else None, int(kernel), int(flags))
    out = ctypes.c_void_p()
    _check(ctx, load_library().ih_batch_create(ctx, arr, len(cs), ctypes.byref(q) if q is not None else None,
                                               int(batch_flags), ctypes.byref(out), handles))
    return out, list(handles)


def ih_batch_run(ctx, batch, stream=None):
    _check(ctx, load_library().ih_batch_run(batch, _stream(stream)))


def ih_batch_destroy(batch):
    _check(None, load_library().ih_batch_destroy(batch))


def ih_tune_set(ctx, frame, band_rows, strip_cols):
    """Later frames of this frame's shape are built on band_rows x strip_cols tiles."""
    cf, _keep = frame._c()
    _check(ctx, load_library().ih_tune_set(ctx, ctypes.byref(cf), int(band_rows), int(strip_cols)))


def ih_autotune(ctx, frame, stream=None):
    f, arr = frame._c()
    _check(ctx, load_library().ih_autotune(ctx, ctypes.byref(f), _stream(stream)))


def ih_server_create(ctx, streams=4, max_inflight=8, max_batch=32):
    cfg = ih_server_config(int(streams), int(max_inflight), int(max_batch), 0)
    out = ctypes.c_void_p()
    _check(ctx, load_library().ih_server_create(ctx, ctypes.byref(cfg), ctypes.byref(out)))
    return out


def ih_server_submit(ctx, srv, tracker, frame, rects=None, rect_out=None, windows=None, weighted_out=None,
                     weighted_flags=0, user=0):
    """Queue a request; the caller keeps `frame.pixels`, the query tensors and
    the outputs alive until its completion is polled."""
    f, arr = frame._c()
    q = ih_request()
    q.tracker = int(tracker)
    q.frame = f
    q.d_rects = _ptr(rects).value if rects is not None else None
    q.n_rects = 0 if rects is None else rects.shape[0]
    q.d_rect_out = _ptr(rect_out).value if rect_out is not None else None
    q.d_windows = _ptr(windows).value if windows is not None else None
    q.n_windows = 0 if windows is None else windows.shape[0]
    q.d_weighted_out = _ptr(weighted_out).value if weighted_out is not None else None
    q.weighted_flags = int(weighted_flags)
    q.user = int(user)
    _check(ctx, load_library().ih_server_submit(srv, ctypes.byref(q)))


def ih_server_poll(srv, max=1024, wait_ms=0):
    arr = (ih_completion * max)()
    n = load_library().ih_server_poll(srv, arr, max, int(wait_ms))
    return [{k: getattr(arr[i], k) for k, _ in ih_completion._fields_} for i in range(n)]


def ih_server_cancel(srv, user):
    """Cancels the uncompleted request tagged `user`; its completion carries
    IH_ECANCELLED."""
    _check(None, load_library().ih_server_cancel(srv, ctypes.c_uint64(int(user))))


def ih_server_drain(srv):
    _check(None, load_library().ih_server_drain(srv))


def ih_server_clock(srv) -> float:
    return float(load_library().ih_server_clock(srv))


def ih_server_destroy(srv):
    _check(None, load_library().ih_server_destroy(srv))


def ih_wait_selftest(ctx, polls, stream=None):
    """A device-side wait on a counter nothing raises, given up after `polls`
    polls: the next ih_sync raises IHError(IH_ETIMEOUT)."""
    _check(ctx, load_library().ih_wait_selftest(ctx, int(polls), _stream(stream)))


def ih_memory_used(ctx) -> int:
    """Bytes of frames the context owns (what its HBM budget bounds)."""
    return int(load_library().ih_memory_used(ctx))


def ih_launch_count(ctx) -> int:
    return int(load_library().ih_launch_count(ctx))


def ih_last_error(ctx) -> str:
    return load_library().ih_last_error(ctx).decode()


def ih_build_counts_static(pixels, bins, mode, out, stream=None):
    """Allocation-free count build of one channel into `out`.

    pixels: (H, W) uint8 CUDA tensor (rows may be padded); out: (bins, H, P)
    int32 CUDA tensor, P >= W a multiple of 4.  Uses the library's static
    carry array: calls that overlap on the GPU race (see include/ih.h)."""
    h, w = pixels.shape
    pitch = pixels.stride(0) if h > 1 else w
    st = load_library().ih_build_counts_static(_ptr(pixels), h, w, pitch, int(bins), int(mode), _ptr(out),
                                                out.shape[2], _stream(stream))
    if st != IH_OK:
        raise IHError(st, "ih_build_counts_static(%dx%d, %d bins)" % (h, w, bins))
    return out
