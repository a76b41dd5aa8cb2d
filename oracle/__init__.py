"""CPU oracle for the integral-histogram path (Poostchi 2017, arXiv 1711.01656).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never does.

The arithmetic lives in plain C (``ih_oracle.c``, FP64 where values are not
integers); this module only compiles it with gcc and marshals numpy arrays.
Each wrapper names the passage of the thesis it follows:

* :func:`integral_histogram`  -- Algorithm 5 (sequential recurrence), Eq. 2.15
* :func:`weighted_integral_histogram` -- Eq. 3.4 with w in {1, c, r, c^2, r^2}
* :func:`rect_hist`   -- Eq. 2.16's quantity by enumeration of the region
* :func:`weighted_hist` -- Eq. 3.1 by direct FP64 summation (Sec. 3.1.1)
* :func:`features`  -- Eq. 2.33 intensity + gradient orientation (Fig. 2.3)

Multi-channel frames concatenate the channels' bins in channel order, so the
tensor is (sum of bins) x H x W, bin-major (Fig. 5.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ih_oracle.c")
_LIB = os.path.join(_HERE, "libih_oracle.so")

BIN_UNIFORM8 = 0
BIN_INDEX = 1
W_ONE, W_COL, W_ROW, W_COL2, W_ROW2 = 0, 1, 2, 3, 4
MOMENT_WEIGHTS = (W_COL, W_ROW, W_COL2, W_ROW2)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libih_oracle.so`` with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    lib.oracle_bin_of.argtypes = [i32, i32, i32]
    lib.oracle_bin_of.restype = i32
    lib.oracle_weighted_ih.argtypes = [p, i64, i32, i32, i32, i32, i32, p, i32]
    lib.oracle_weighted_ih.restype = i32
    lib.oracle_ih.argtypes = [p, i64, i32, i32, i32, i32, p, i32]
    lib.oracle_ih.restype = i32
    lib.oracle_rect_hist.argtypes = [p, i64, i32, i32, i32, i32, p, i64, p]
    lib.oracle_rect_hist.restype = i64
    lib.oracle_weighted_hist.argtypes = [p, i64, i32, i32, i32, i32, p, i64, i32, p]
    lib.oracle_weighted_hist.restype = i64
    lib.oracle_kernel_weight.argtypes = [p, i32, i32]
    lib.oracle_kernel_weight.restype = ctypes.c_double
    lib.oracle_weighted_hist_k.argtypes = [p, i64, i32, i32, i32, i32, p, i64, i32, i32, i32, p]
    lib.oracle_weighted_hist_k.restype = i64
    lib.oracle_manhattan_weight.argtypes = [p, i32, i32]
    lib.oracle_manhattan_weight.restype = ctypes.c_double
    lib.oracle_wedding_weight.argtypes = [p, i32, i32, i32]
    lib.oracle_wedding_weight.restype = ctypes.c_double
    lib.oracle_match_window.argtypes = [p, i64, i32, i32, i32, i32, p, i32, i32, i32, i32, i32, i32, p]
    lib.oracle_match_window.restype = i64
    lib.oracle_local_median.argtypes = [p, i32, i32, i32, i32, i32, i32, i32, p]
    lib.oracle_local_median.restype = None
    lib.oracle_isqrt.argtypes = [i64]
    lib.oracle_isqrt.restype = i64
    lib.oracle_canny.argtypes = [p, i32, i32, i32, i32, p, p, p, p]
    lib.oracle_canny.restype = None
    lib.oracle_phog_planes.argtypes = [p, i32, i32, i32, i32, p, p]
    lib.oracle_phog_planes.restype = None
    lib.oracle_phog_ih.argtypes = [p, p, i32, i32, i32, p]
    lib.oracle_phog_ih.restype = None
    lib.oracle_phog_descriptor.argtypes = [p, p, i32, i32, i32, i32, i32, i32, i32, i32, p]
    lib.oracle_phog_descriptor.restype = None
    lib.oracle_pyramid_match.argtypes = [p, p, i32, i32]
    lib.oracle_pyramid_match.restype = ctypes.c_double
    lib.oracle_orientation_bin.argtypes = [i32, i32, i32]
    lib.oracle_orientation_bin.restype = i32
    lib.oracle_features.argtypes = [p, i32, i32, p]
    lib.oracle_features.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _plane(img) -> np.ndarray:
    a = np.ascontiguousarray(img, dtype=np.uint8)
    if a.ndim != 2:
        raise ValueError("expected an H x W uint8 plane")
    return a


def bin_of(v: int, bins: int, mode: int = BIN_UNIFORM8) -> int:
    """Eq. 2.15's binning function: the bin value v falls in (-1: none)."""
    return _load().oracle_bin_of(int(v), int(bins), int(mode))


def integral_histogram(img, bins: int, mode: int = BIN_UNIFORM8, threads: int = 1) -> np.ndarray:
    """Algorithm 5: int32 tensor bins x H x W (inclusive, Eq. 2.15)."""
    a = _plane(img)
    h, w = a.shape
    out = np.empty((bins, h, w), dtype=np.int32)
    rc = _load().oracle_ih(a.ctypes.data, w, h, w, bins, mode, out.ctypes.data, threads)
    if rc != 0:
        raise ArithmeticError("oracle_ih failed (%d)" % rc)
    return out


def weighted_integral_histogram(img, bins: int, weight: int, mode: int = BIN_UNIFORM8,
                                threads: int = 1) -> np.ndarray:
    """Eq. 3.4 with w(r,c) in {1, c, r, c^2, r^2}: int64 bins x H x W."""
    a = _plane(img)
    h, w = a.shape
    out = np.empty((bins, h, w), dtype=np.int64)
    rc = _load().oracle_weighted_ih(a.ctypes.data, w, h, w, bins, mode, weight,
                                    out.ctypes.data, threads)
    if rc != 0:
        raise ValueError("oracle_weighted_ih failed (%d)" % rc)
    return out


def _boxes(q) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.int32)
    if q.ndim != 2 or q.shape[1] != 4:
        raise ValueError("expected n x 4 int32 (r0, c0, r1, c1)")
    return q


def rect_hist(img, bins: int, rects, mode: int = BIN_UNIFORM8) -> np.ndarray:
    """Histogram of each inclusive rectangle by enumerating its pixels."""
    a, q = _plane(img), _boxes(rects)
    h, w = a.shape
    out = np.empty((q.shape[0], bins), dtype=np.int32)
    _load().oracle_rect_hist(a.ctypes.data, w, h, w, bins, mode, q.ctypes.data, q.shape[0],
                             out.ctypes.data)
    return out


# spatial kernels of weighted_hist
K_EPANECHNIKOV, K_MANHATTAN, K_WEDDING_CAKE = 0, 1, 2


def weighted_hist(img, bins: int, windows, mode: int = BIN_UNIFORM8,
                  normalize: bool = False, kernel: int = K_EPANECHNIKOV, layers: int = 4) -> np.ndarray:
    """Eq. 3.1 by direct FP64 summation with the Epanechnikov window kernel,
    the Manhattan kernel (Eq. 3.3) or the wedding-cake rings (Eq. 3.2)."""
    a, q = _plane(img), _boxes(windows)
    h, w = a.shape
    out = np.empty((q.shape[0], bins), dtype=np.float64)
    if kernel == K_EPANECHNIKOV:
        _load().oracle_weighted_hist(a.ctypes.data, w, h, w, bins, mode, q.ctypes.data,
                                     q.shape[0], int(bool(normalize)), out.ctypes.data)
    else:
        _load().oracle_weighted_hist_k(a.ctypes.data, w, h, w, bins, mode, q.ctypes.data, q.shape[0],
                                       int(kernel), int(layers), int(bool(normalize)), out.ctypes.data)
    return out


def match_window(img, bins: int, target, win_h: int, win_w: int, search, mode: int = BIN_UNIFORM8) -> np.ndarray:
    """City-block distance (Eq. 2.22, p = 1) between `target` (bins counts)
    and the histogram of every win_h x win_w window whose top-left pixel lies
    in search = (sr0, sc0, sr1, sc1); returns an int64 map of the placements."""
    a = _plane(img)
    h, w = a.shape
    t = np.ascontiguousarray(target, dtype=np.int32).reshape(bins)
    sr0, sc0, sr1, sc1 = (int(x) for x in search)
    out = np.empty((sr1 - sr0 + 1, sc1 - sc0 + 1), dtype=np.int64)
    if _load().oracle_match_window(a.ctypes.data, w, h, w, bins, mode, t.ctypes.data, int(win_h), int(win_w),
                                   sr0, sc0, sr1, sc1, out.ctypes.data) < 0:
        raise ValueError("a placement leaves the image")
    return out


def local_median(frames, bins: int, m: int, n: int, mode: int = BIN_UNIFORM8) -> np.ndarray:
    """Per-pixel lower-median bin of the m x n box (clipped at the border) over
    all frames (Algorithm 4); frames: (nf, h, w) or (h, w) uint8; int32 map."""
    a = np.ascontiguousarray(frames, dtype=np.uint8)
    if a.ndim == 2:
        a = a[None]
    nf, h, w = a.shape
    out = np.empty((h, w), dtype=np.int32)
    _load().oracle_local_median(a.ctypes.data, nf, h, w, bins, mode, int(m), int(n), out.ctypes.data)
    return out


PHOG_BINS = 9


def isqrt(n: int) -> int:
    return int(_load().oracle_isqrt(int(n)))


def canny(gray, lo: int, hi: int):
    """Algorithm 2 step 1, Canny's detector: (edges uint8 0/1, smoothed S
    int32 = 256 x the binomial-smoothed image, squared gradient magnitude of
    S int64, survivor class uint8: 0 none, 1 weak, 2 strong)."""
    a = _plane(gray)
    h, w = a.shape
    edges = np.empty((h, w), np.uint8)
    smooth = np.empty((h, w), np.int32)
    mag2 = np.empty((h, w), np.int64)
    cls = np.empty((h, w), np.uint8)
    _load().oracle_canny(a.ctypes.data, h, w, int(lo), int(hi), edges.ctypes.data, smooth.ctypes.data,
                         mag2.ctypes.data, cls.ctypes.data)
    return edges, smooth, mag2, cls


def phog_planes(gray, lo: int, hi: int):
    """Algorithm 2 steps 1-3: (bins uint8 with 255 off the Canny edges,
    int32 magnitude weights)."""
    a = _plane(gray)
    h, w = a.shape
    bins = np.empty((h, w), np.uint8)
    wt = np.empty((h, w), np.int32)
    _load().oracle_phog_planes(a.ctypes.data, h, w, int(lo), int(hi), bins.ctypes.data, wt.ctypes.data)
    return bins, wt


def phog_ih(bins, weight, b: int = PHOG_BINS) -> np.ndarray:
    """Algorithm 2 step 4: b x h x w int64 magnitude-weighted integral histogram."""
    q = np.ascontiguousarray(bins, dtype=np.uint8)
    wt = np.ascontiguousarray(weight, dtype=np.int32)
    h, w = q.shape
    out = np.empty((b, h, w), np.int64)
    _load().oracle_phog_ih(q.ctypes.data, wt.ctypes.data, h, w, b, out.ctypes.data)
    return out


def phog_descriptor_len(levels: int, b: int = PHOG_BINS) -> int:
    return b * sum(4 ** l for l in range(levels + 1))


def phog_descriptor(bins, weight, levels: int, r0: int, c0: int, wh: int, ww: int, b: int = PHOG_BINS):
    """Algorithm 2 steps 5-20 for one window: the concatenated cell histograms."""
    q = np.ascontiguousarray(bins, dtype=np.uint8)
    wt = np.ascontiguousarray(weight, dtype=np.int32)
    h, w = q.shape
    out = np.empty(phog_descriptor_len(levels, b), np.int64)
    _load().oracle_phog_descriptor(q.ctypes.data, wt.ctypes.data, h, w, b, int(levels), int(r0), int(c0), int(wh),
                                   int(ww), out.ctypes.data)
    return out


def pyramid_match(x, y, levels: int, b: int = PHOG_BINS) -> float:
    """Eq. 2.24's pyramid match kernel of two descriptors."""
    a = np.ascontiguousarray(x, dtype=np.int64)
    c = np.ascontiguousarray(y, dtype=np.int64)
    return float(_load().oracle_pyramid_match(a.ctypes.data, c.ctypes.data, b, int(levels)))


def manhattan_weight(window, r: int, c: int) -> float:
    """The Manhattan-kernel weight of one pixel inside `window`."""
    q = np.ascontiguousarray(window, dtype=np.int32).reshape(4)
    return _load().oracle_manhattan_weight(q.ctypes.data, int(r), int(c))


def wedding_weight(window, layers: int, r: int, c: int) -> float:
    """The wedding-cake weight of one pixel inside `window` (`layers` rings)."""
    q = np.ascontiguousarray(window, dtype=np.int32).reshape(4)
    return _load().oracle_wedding_weight(q.ctypes.data, int(layers), int(r), int(c))


def kernel_weight(window, r: int, c: int) -> float:
    """The spatial weight k(r, c) of one pixel inside `window` (FP64)."""
    q = np.ascontiguousarray(window, dtype=np.int32).reshape(4)
    return _load().oracle_kernel_weight(q.ctypes.data, int(r), int(c))


def orientation_bin(gx: int, gy: int, nbins: int = 9) -> int:
    """Unsigned gradient-orientation bin of the integer gradient (gx, gy)."""
    return _load().oracle_orientation_bin(int(gx), int(gy), int(nbins))


def features(rgb) -> np.ndarray:
    """7 uint8 planes (R, G, B, I, HoG s=1, s=2, s=4) from 3 x H x W RGB."""
    a = np.ascontiguousarray(rgb, dtype=np.uint8)
    if a.ndim != 3 or a.shape[0] != 3:
        raise ValueError("expected 3 x H x W uint8")
    _, h, w = a.shape
    out = np.empty((7, h, w), dtype=np.uint8)
    _load().oracle_features(a.ctypes.data, h, w, out.ctypes.data)
    return out


# ----------------------------------------------------------------------------
# multi-channel frames: channels' bins concatenated in channel order


def frame_integral_histogram(planes, chans, threads: int = 1) -> np.ndarray:
    """Algorithm 5 per channel; chans is a list of (bins, mode)."""
    return np.concatenate([integral_histogram(p, b, m, threads) for p, (b, m) in zip(planes, chans)],
                          axis=0)


def frame_rect_hist(planes, chans, rects) -> np.ndarray:
    return np.concatenate([rect_hist(p, b, rects, m) for p, (b, m) in zip(planes, chans)], axis=1)
