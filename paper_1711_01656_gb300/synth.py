"""Seeded synthetic inputs shaped like the thesis's workloads.

This module draws random frames, rectangles and windows and nothing else: it
holds none of the integral-histogram arithmetic, and both the CUDA path's
tests and the CPU oracle consume what it returns.

The thesis evaluates on full-motion video (FMV, e.g. 1920x1080 RGB) and
wide-area aerial imagery (WAMI, large 8-bit grayscale mosaics); those
datasets are not available, so frames are synthesised with the same shapes:

* ``uniform_plane``: i.i.d. uniform bytes in [0, 256);
* ``blob_plane``: 128 + a sum of 50 Gaussian blobs (amplitude U[-120, 120],
  sigma U[0.01, 0.1] * min(H, W), centre uniform, each truncated to the box
  of +-4 sigma) + N(0, 8) noise, rounded half-to-even and clipped to [0, 255];
* ``blob_rgb``: three independent blob planes (R, G, B).

Generators use numpy's PCG64 seeded with the caller's integer seed.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x1711016560


def config_seed(k: int) -> int:
    """Fixed seed of the k-th workload (k = 1..5)."""
    return SEED_BASE + int(k)


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_plane(h: int, w: int, seed) -> np.ndarray:
    return _rng(seed).integers(0, 256, size=(h, w), dtype=np.uint8)


def _blob_field(h: int, w: int, rng: np.random.Generator, nblobs: int = 50) -> np.ndarray:
    f = np.full((h, w), 128.0, dtype=np.float32)
    m = float(min(h, w))
    for _ in range(nblobs):
        a = rng.uniform(-120.0, 120.0)
        s = rng.uniform(0.01, 0.1) * m
        cy = rng.uniform(0.0, h)
        cx = rng.uniform(0.0, w)
        r0, r1 = max(0, int(cy - 4 * s)), min(h, int(cy + 4 * s) + 1)
        c0, c1 = max(0, int(cx - 4 * s)), min(w, int(cx + 4 * s) + 1)
        if r0 >= r1 or c0 >= c1:
            continue
        gy = np.exp(-((np.arange(r0, r1, dtype=np.float32) - cy) ** 2) / (2 * s * s))
        gx = np.exp(-((np.arange(c0, c1, dtype=np.float32) - cx) ** 2) / (2 * s * s))
        f[r0:r1, c0:c1] += np.float32(a) * np.outer(gy, gx)
    f += rng.normal(0.0, 8.0, size=(h, w)).astype(np.float32)
    return np.clip(np.rint(f), 0, 255).astype(np.uint8)


def blob_plane(h: int, w: int, seed) -> np.ndarray:
    return _blob_field(h, w, _rng(seed))


def blob_rgb(h: int, w: int, seed) -> np.ndarray:
    rng = _rng(seed)
    return np.stack([_blob_field(h, w, rng) for _ in range(3)], axis=0)


def rects_uniform_corners(h: int, w: int, n: int, seed) -> np.ndarray:
    """n x 4 int32 (r0, c0, r1, c1): two uniform column draws give the min and
    max column, likewise rows, so width and height range over 1..full."""
    g = _rng(seed)
    rr = g.integers(0, h, size=(n, 2))
    cc = g.integers(0, w, size=(n, 2))
    return np.stack([rr.min(1), cc.min(1), rr.max(1), cc.max(1)], axis=1).astype(np.int32)


def rects_side_range(h: int, w: int, n: int, smin: int, smax: int, seed) -> np.ndarray:
    """n x 4 int32 boxes whose height and width are independently uniform in
    [smin, smax] (clamped to the frame) and that lie fully inside it."""
    g = _rng(seed)
    hh = np.minimum(g.integers(smin, smax + 1, size=n), h)
    ww = np.minimum(g.integers(smin, smax + 1, size=n), w)
    r0 = (g.random(n) * (h - hh + 1)).astype(np.int64)
    c0 = (g.random(n) * (w - ww + 1)).astype(np.int64)
    return np.stack([r0, c0, r0 + hh - 1, c0 + ww - 1], axis=1).astype(np.int32)


# The tracker's feature channels: R, G, B and intensity with 16 uniform bins,
# three gradient-orientation index planes with 9 bins each.
FMV_CHANNELS = [(16, 0)] * 4 + [(9, 1)] * 3


def frame_sizes_batched(n: int, seed) -> list:
    """Frame sizes (h, w) drawn uniformly from the batched workload's set."""
    sizes = [(480, 640), (720, 1280), (1080, 1920), (2160, 4096)]
    g = _rng(seed)
    return [sizes[i] for i in g.integers(0, len(sizes), size=n)]
