"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Counts, indices and int64 moment planes must be bit-exact; weighted
histograms (FP32) within 1e-5 relative of the FP64 oracle and exactly 0
where the oracle is 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
WTOL = 1e-5


def _build(ih, ctx, planes, chans, weighted=-1, pitch=None, layout=0):
    planes = np.asarray(planes, dtype=np.uint8)
    if planes.ndim == 2:
        planes = planes[None]
    planes = np.ascontiguousarray(planes)
    p, h, w = planes.shape
    if pitch is not None and pitch > w:
        buf = torch.zeros((p, h, pitch), dtype=torch.uint8, device=DEV)
        buf[:, :, :w] = torch.from_numpy(planes).to(DEV)
        pix = buf[:, :, :w]
    else:
        pix = torch.from_numpy(planes).to(DEV)
    hdl, = ih.ih_build(ctx, ih.Frame(pix, chans, weighted_channel=weighted, layout=layout))
    return hdl, pix


def _export(ih, ctx, hdl):
    info = ih.ih_info(ctx, hdl)
    out = torch.empty((info["total_bins"], info["height"], info["width"]), dtype=torch.int32, device=DEV)
    ih.ih_export(ctx, hdl, out)
    ih.ih_sync(ctx)
    return out.cpu().numpy()


def _assert_weighted(got, ref):
    got = np.asarray(got, dtype=np.float64)
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero]), "non-zero where the oracle is 0"
    rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.size == 0 or rel.max() <= WTOL, "max rel err %g" % rel.max()


# ---------------------------------------------------------------- counts


SHAPES = [(1, 1), (1, 7), (7, 1), (2, 3), (37, 53), (33, 129), (64, 128), (65, 257), (130, 300),
          (200, 611), (257, 1030)]


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("h,w", SHAPES)
@pytest.mark.parametrize("bins", [1, 3, 16, 32])
def test_counts_exact(ihlib, ctx, h, w, bins, layout):
    img = synth.uniform_plane(h, w, h * 1000 + w + bins)
    hdl, _ = _build(ihlib, ctx, img, [(bins, 0)], layout=layout)
    got = _export(ihlib, ctx, hdl)
    ih_ref = oracle.integral_histogram(img, bins)
    assert np.array_equal(got, ih_ref)
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("bins", [2, 7, 9, 40, 64, 200, 256])
def test_counts_exact_bin_counts(ihlib, ctx, bins, layout):
    img = synth.blob_plane(150, 260, bins)
    hdl, _ = _build(ihlib, ctx, img, [(bins, 0)], layout=layout)
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.integral_histogram(img, bins))
    ihlib.ih_release(ctx, hdl)


def test_counts_index_mode_and_out_of_range(ihlib, ctx):
    g = np.random.Generator(np.random.PCG64(5))
    img = g.integers(0, 12, size=(90, 301)).astype(np.uint8)  # values 9..11 are in no bin
    hdl, _ = _build(ihlib, ctx, img, [(9, 1)])
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.integral_histogram(img, 9, oracle.BIN_INDEX))
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("pitch", [None, 301, 304, 512])
def test_counts_pitched_input(ihlib, ctx, pitch):
    img = synth.uniform_plane(77, 299, 3)
    hdl, _ = _build(ihlib, ctx, img, [(16, 0)], pitch=pitch)
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.integral_histogram(img, 16))
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_counts_multichannel(ihlib, ctx, layout):
    h, w = 123, 517
    planes = np.stack([synth.uniform_plane(h, w, 10 + k) for k in range(4)])
    planes[3] %= 9
    chans = [(16, 0), (5, 0), (32, 0), (9, 1)]
    hdl, _ = _build(ihlib, ctx, planes, chans, layout=layout)
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.frame_integral_histogram(planes, chans))
    ihlib.ih_release(ctx, hdl)


def test_counts_deterministic(ihlib, ctx):
    img = synth.uniform_plane(300, 700, 1)
    a, _ = _build(ihlib, ctx, img, [(16, 0)])
    b, _ = _build(ihlib, ctx, img, [(16, 0)])
    assert np.array_equal(_export(ihlib, ctx, a), _export(ihlib, ctx, b))
    ihlib.ih_release(ctx, a)
    ihlib.ih_release(ctx, b)


# ---------------------------------------------------------------- features


def _plus_pattern_rgb():
    """A gray image whose 3x3 blocks realise every integer gradient
    (gx, gy) in [-255,255]^2 at step 1 in their centre pixel."""
    n = 511
    img = np.zeros((3 * n, 3 * n), np.uint8)
    g = np.arange(-255, 256)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    cr = 3 * np.arange(n)[:, None] + 1 + np.zeros((1, n), int)
    cc = 3 * np.arange(n)[None, :] + 1 + np.zeros((n, 1), int)
    left = np.maximum(0, -gx)
    up = np.maximum(0, -gy)
    img[cr, cc - 1] = left
    img[cr, cc + 1] = left + gx
    img[cr - 1, cc] = up
    img[cr + 1, cc] = up + gy
    img[cr, cc] = 100
    return np.stack([img, img, img]), gx, gy


def test_features_exhaustive_orientations(ihlib, ctx):
    rgb, gx, gy = _plus_pattern_rgb()
    d = torch.from_numpy(rgb).to(DEV)
    out = torch.empty((7,) + rgb.shape[1:], dtype=torch.uint8, device=DEV)
    ihlib.ih_features(ctx, d, out)
    ihlib.ih_sync(ctx)
    got = out.cpu().numpy()
    ref = oracle.features(rgb)
    assert np.array_equal(got, ref)
    # every one of the 261,121 gradients occurs at a block centre
    centres = got[4][1::3, 1::3]
    exp = np.vectorize(oracle.orientation_bin)(gx, gy)
    assert np.array_equal(centres, exp)


@pytest.mark.parametrize("h,w", [(1, 1), (3, 2), (5, 9), (33, 31), (100, 257), (1080, 1920)])
def test_features_exact(ihlib, ctx, h, w):
    rgb = synth.blob_rgb(h, w, h + w)
    d = torch.from_numpy(rgb).to(DEV)
    out = torch.empty((7, h, w), dtype=torch.uint8, device=DEV)
    ihlib.ih_features(ctx, d, out)
    ihlib.ih_sync(ctx)
    assert np.array_equal(out.cpu().numpy(), oracle.features(rgb))


def test_rgb_feature_frame_build(ihlib, ctx):
    h, w = 130, 270
    rgb = synth.blob_rgb(h, w, 2)
    chans = synth.FMV_CHANNELS
    hdl, = ihlib.ih_build(ctx, ihlib.Frame(torch.from_numpy(rgb).to(DEV), chans,
                                           input=ihlib.IH_INPUT_RGB_FEATURES))
    ref = oracle.frame_integral_histogram(oracle.features(rgb), chans)
    assert np.array_equal(_export(ihlib, ctx, hdl), ref)
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- rect queries


def _rects_gpu(ihlib, ctx, hdl, rects, B):
    d_r = torch.from_numpy(np.ascontiguousarray(rects, dtype=np.int32)).to(DEV)
    out = torch.empty((len(rects), B), dtype=torch.int32, device=DEV)
    ihlib.ih_query_rects(ctx, hdl, d_r, out)
    return out


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_rects_all_of_small_frame(ihlib, ctx, layout):
    h, w, bins = 14, 19, 5
    img = synth.uniform_plane(h, w, 4)
    hdl, _ = _build(ihlib, ctx, img, [(bins, 0)], layout=layout)
    rects = np.array([(r0, c0, r1, c1) for r0 in range(h) for r1 in range(r0, h)
                      for c0 in range(w) for c1 in range(c0, w)], np.int32)
    got = _rects_gpu(ihlib, ctx, hdl, rects, bins)
    ihlib.ih_sync(ctx)
    assert np.array_equal(got.cpu().numpy(), oracle.rect_hist(img, bins, rects))
    ihlib.ih_release(ctx, hdl)


def test_rects_invalid_rows_and_status(ihlib, ctx):
    img = synth.uniform_plane(20, 30, 4)
    hdl, _ = _build(ihlib, ctx, img, [(4, 0)])
    rects = np.array([[0, 0, 19, 29], [-1, 0, 3, 3], [0, 0, 20, 3], [5, 0, 4, 3], [0, 9, 3, 8], [0, 0, 3, 30]],
                     np.int32)
    got = _rects_gpu(ihlib, ctx, hdl, rects, 4)
    with pytest.raises(ihlib.IHError) as ei:
        ihlib.ih_sync(ctx)
    assert ei.value.status == ihlib.IH_EINVAL
    g = got.cpu().numpy()
    assert (g[1:] == -1).all() and g[0].sum() == 600
    ihlib.ih_sync(ctx)  # the error word was cleared
    ihlib.ih_release(ctx, hdl)


def test_rects_empty_query(ihlib, ctx):
    img = synth.uniform_plane(8, 8, 4)
    hdl, _ = _build(ihlib, ctx, img, [(4, 0)])
    out = torch.empty((0, 4), dtype=torch.int32, device=DEV)
    ihlib.ih_query_rects(ctx, hdl, torch.empty((0, 4), dtype=torch.int32, device=DEV), out)
    ihlib.ih_sync(ctx)
    ihlib.ih_release(ctx, hdl)


def test_plain_frame_640x480_all_rects(ihlib, ctx):
    """One 640x480 uniform frame, 16 bins, 10,000 rectangles with uniform
    corners: the full tensor and every query against the oracle."""
    h, w = 480, 640
    img = synth.uniform_plane(h, w, synth.config_seed(1))
    rects = synth.rects_uniform_corners(h, w, 10000, synth.config_seed(1) + 100)
    hdl, _ = _build(ihlib, ctx, img, [(16, 0)])
    got = _rects_gpu(ihlib, ctx, hdl, rects, 16)
    tens = _export(ihlib, ctx, hdl)
    assert np.array_equal(tens, oracle.integral_histogram(img, 16, threads=8))
    assert np.array_equal(got.cpu().numpy(), oracle.rect_hist(img, 16, rects))
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_fmv_frame_1920x1080_features(ihlib, ctx, layout):
    """One 1920x1080 RGB frame, 7 feature channels (91 bins): the full
    tensor vs Algorithm 5 and 100,000 rectangles (a seeded 2,000 by
    enumeration, all by four corners of the oracle's own tensor)."""
    h, w = 1080, 1920
    rgb = synth.blob_rgb(h, w, synth.config_seed(2))
    chans = synth.FMV_CHANNELS
    B = sum(b for b, _ in chans)
    hdl, = ihlib.ih_build(ctx, ihlib.Frame(torch.from_numpy(rgb).to(DEV), chans,
                                           input=ihlib.IH_INPUT_RGB_FEATURES, layout=layout))
    rects = synth.rects_uniform_corners(h, w, 100000, synth.config_seed(2) + 100)
    got = _rects_gpu(ihlib, ctx, hdl, rects, B).cpu().numpy()
    tens = _export(ihlib, ctx, hdl)
    feats = oracle.features(rgb)
    ref = oracle.frame_integral_histogram(feats, chans, threads=8)
    assert np.array_equal(tens, ref)
    P = np.pad(ref.astype(np.int64), ((0, 0), (1, 0), (1, 0)))
    r0, c0, r1, c1 = (rects[:, i] for i in range(4))
    four = (P[:, r1 + 1, c1 + 1] - P[:, r0, c1 + 1] - P[:, r1 + 1, c0] + P[:, r0, c0]).T
    assert np.array_equal(got, four)
    sub = np.random.Generator(np.random.PCG64(9)).choice(len(rects), 2000, replace=False)
    assert np.array_equal(got[sub], oracle.frame_rect_hist(feats, chans, rects[sub]))
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- moments + weighted


@pytest.mark.parametrize("h,w,bins", [(1, 1, 2), (5, 7, 3), (64, 128, 16), (131, 389, 16), (260, 520, 8),
                                      (300, 1500, 32), (1100, 300, 5)])
def test_moment_planes_exact(ihlib, ctx, h, w, bins):
    img = synth.blob_plane(h, w, h + w)
    hdl, _ = _build(ihlib, ctx, img, [(bins, 0)], weighted=0)
    for plane, wk in enumerate(oracle.MOMENT_WEIGHTS):
        out = torch.empty((bins, h, w), dtype=torch.int64, device=DEV)
        ihlib.ih_export_moments(ctx, hdl, plane, out)
        ihlib.ih_sync(ctx)
        ref = oracle.weighted_integral_histogram(img, bins, wk)
        assert np.array_equal(out.cpu().numpy(), ref), "moment plane %d" % plane
    ihlib.ih_release(ctx, hdl)


def _weighted_gpu(ihlib, ctx, hdl, wins, Bw, normalize=False, kernel=0, layers=0):
    d = torch.from_numpy(np.ascontiguousarray(wins, dtype=np.int32)).to(DEV)
    out = torch.empty((len(wins), Bw), dtype=torch.float32, device=DEV)
    flags = (ihlib.IH_NORMALIZE if normalize else 0) | ihlib.IH_LAYERS(layers)
    ihlib.ih_query_weighted(ctx, hdl, d, out, kernel=kernel, flags=flags)
    ihlib.ih_sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("normalize", [False, True])
def test_weighted_vs_direct_sum(ihlib, ctx, normalize, layout):
    h, w = 300, 400
    img = synth.blob_plane(h, w, 12)
    hdl, _ = _build(ihlib, ctx, img, [(16, 0)], weighted=0, layout=layout)
    wins = np.concatenate([synth.rects_side_range(h, w, 1500, 1, 64, 3),
                           synth.rects_side_range(h, w, 100, 32, 256, 4),
                           np.array([[0, 0, h - 1, w - 1], [0, 0, 0, 0], [h - 1, w - 1, h - 1, w - 1]])])
    got = _weighted_gpu(ihlib, ctx, hdl, wins, 16, normalize)
    ref = oracle.weighted_hist(img, 16, wins, normalize=normalize)
    _assert_weighted(got, ref)
    ihlib.ih_release(ctx, hdl)


def test_weighted_hand_example(ihlib, ctx):
    img = np.array([[0, 200, 100], [255, 50, 130]], np.uint8)
    hdl, _ = _build(ihlib, ctx, img, [(2, 0)], weighted=0)
    got = _weighted_gpu(ihlib, ctx, hdl, [[0, 0, 1, 2]], 2)
    assert np.allclose(got[0], [157 / 72, 157 / 72], rtol=1e-6, atol=0)
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_weighted_on_feature_channel(ihlib, ctx, layout):
    h, w = 200, 330
    rgb = synth.blob_rgb(h, w, 8)
    chans = synth.FMV_CHANNELS
    hdl, = ihlib.ih_build(ctx, ihlib.Frame(torch.from_numpy(rgb).to(DEV), chans,
                                           input=ihlib.IH_INPUT_RGB_FEATURES, weighted_channel=3,
                                           layout=layout))
    wins = synth.rects_side_range(h, w, 500, 2, 150, 5)
    got = _weighted_gpu(ihlib, ctx, hdl, wins, 16)
    ref = oracle.weighted_hist(oracle.features(rgb)[3], 16, wins)
    _assert_weighted(got, ref)
    ihlib.ih_release(ctx, hdl)


def test_weighted_requires_moments(ihlib, ctx):
    img = synth.uniform_plane(10, 10, 1)
    hdl, _ = _build(ihlib, ctx, img, [(4, 0)])
    with pytest.raises(ihlib.IHError):
        _weighted_gpu(ihlib, ctx, hdl, [[0, 0, 3, 3]], 4)
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- host-side errors


def test_budget_refuses_and_builds_nothing(ihlib):
    c = ihlib.ih_create(0, hbm_budget_bytes=1 << 20)
    try:
        img = torch.zeros((1, 512, 512), dtype=torch.uint8, device=DEV)
        with pytest.raises(ihlib.IHError) as ei:
            ihlib.ih_build(c, ihlib.Frame(img, [(16, 0)]))
        assert ei.value.status == ihlib.IH_EBUDGET
        small = torch.zeros((1, 64, 64), dtype=torch.uint8, device=DEV)
        h, = ihlib.ih_build(c, ihlib.Frame(small, [(16, 0)]))
        ihlib.ih_release(c, h)
    finally:
        ihlib.ih_destroy(c)


def test_invalid_descriptors(ihlib, ctx):
    img = torch.zeros((1, 8, 8), dtype=torch.uint8, device=DEV)
    for chans in ([(0, 0)], [(257, 0)], [(4, 2)]):
        with pytest.raises(ihlib.IHError) as ei:
            ihlib.ih_build(ctx, ihlib.Frame(img, chans))
        assert ei.value.status == ihlib.IH_EINVAL
    with pytest.raises(ihlib.IHError) as ei:
        ihlib.ih_build(ctx, ihlib.Frame(img, [(4, 0)], weighted_channel=1))
    assert ei.value.status == ihlib.IH_EINVAL
    with pytest.raises(ihlib.IHError) as ei:
        ihlib.ih_query_rects(ctx, 12345, None, torch.empty(0, device=DEV))
    assert ei.value.status == ihlib.IH_ENOTBUILT


@pytest.mark.parametrize("wch", [0, 2])
def test_moments_on_multichannel_frame(ihlib, ctx, wch):
    """The moment planes of one channel of a multi-channel frame, with the
    counts of all channels, on a frame that spans many tiles."""
    h, w = 333, 1100
    planes = np.stack([synth.blob_plane(h, w, 30 + k) for k in range(3)])
    chans = [(16, 0), (9, 0), (12, 0)]
    hdl, _ = _build(ihlib, ctx, planes, chans, weighted=wch, layout=1)
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.frame_integral_histogram(planes, chans))
    bw = chans[wch][0]
    for plane, wk in enumerate(oracle.MOMENT_WEIGHTS):
        out = torch.empty((bw, h, w), dtype=torch.int64, device=DEV)
        ihlib.ih_export_moments(ctx, hdl, plane, out)
        ihlib.ih_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), oracle.weighted_integral_histogram(planes[wch], bw, wk))
    wins = synth.rects_side_range(h, w, 300, 1, 200, 6)
    got = _weighted_gpu(ihlib, ctx, hdl, wins, bw)
    _assert_weighted(got, oracle.weighted_hist(planes[wch], bw, wins))
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("bins", [16, 5])
def test_moment_planes_u32_and_weighted(ihlib, ctx, bins):
    """32-bit moment planes hold the int64 planes modulo 2^32 and still give
    the exact weighted histograms of windows with sides up to 256."""
    h, w = 700, 900
    img = synth.blob_plane(h, w, 44)
    pix = torch.from_numpy(img).to(DEV)[None]
    hdl, = ihlib.ih_build(ctx, ihlib.Frame(pix, [(bins, 0)], weighted_channel=0, layout=1, moment_bits=32))
    info = ihlib.ih_info(ctx, hdl)
    assert info["moment_bytes"] == 4 * bins * h * ((w + 3) // 4 * 4) * 4
    for plane, wk in enumerate(oracle.MOMENT_WEIGHTS):
        out = torch.empty((bins, h, w), dtype=torch.int64, device=DEV)
        ihlib.ih_export_moments(ctx, hdl, plane, out)
        ihlib.ih_sync(ctx)
        ref = oracle.weighted_integral_histogram(img, bins, wk) % (1 << 32)
        assert np.array_equal(out.cpu().numpy(), ref), "plane %d" % plane
    wins = np.concatenate([synth.rects_side_range(h, w, 800, 1, 256, 7),
                           np.array([[0, 0, 255, 255], [h - 256, w - 256, h - 1, w - 1]], np.int32)])
    got = _weighted_gpu(ihlib, ctx, hdl, wins, bins)
    _assert_weighted(got, oracle.weighted_hist(img, bins, wins))
    # a window wider than 256 is refused on the device
    with pytest.raises(ihlib.IHError):
        _weighted_gpu(ihlib, ctx, hdl, [[0, 0, 10, 256]], bins)
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- Manhattan kernel (Eq. 3.3), wedding cake (Eq. 3.2)

def _edge_windows(h, w):
    return np.array([[0, 0, h - 1, w - 1], [0, 0, 0, 0], [h - 1, w - 1, h - 1, w - 1], [0, 5, 0, 60],
                     [3, 0, 90, 0], [1, 2, 2, 3]], np.int32)


@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("normalize", [False, True])
def test_manhattan_vs_direct_sum(ihlib, ctx, normalize, layout):
    h, w = 300, 400
    img = synth.blob_plane(h, w, 14)
    hdl, _ = _build(ihlib, ctx, img, [(16, 0)], weighted=0, layout=layout)
    wins = np.concatenate([synth.rects_side_range(h, w, 1500, 1, 64, 5),
                           synth.rects_side_range(h, w, 100, 32, 256, 6), _edge_windows(h, w)])
    got = _weighted_gpu(ihlib, ctx, hdl, wins, 16, normalize, kernel=ihlib.IH_K_MANHATTAN)
    ref = oracle.weighted_hist(img, 16, wins, normalize=normalize, kernel=oracle.K_MANHATTAN)
    _assert_weighted(got, ref)
    ihlib.ih_release(ctx, hdl)


def test_manhattan_32bit_moment_planes(ihlib, ctx):
    h, w = 600, 700
    img = synth.blob_plane(h, w, 15)
    pix = torch.from_numpy(img).to(DEV)[None]
    hdl, = ihlib.ih_build(ctx, ihlib.Frame(pix, [(16, 0)], weighted_channel=0, layout=1, moment_bits=32))
    wins = np.concatenate([synth.rects_side_range(h, w, 800, 1, 256, 16),
                           np.array([[0, 0, 255, 255], [h - 256, w - 256, h - 1, w - 1]], np.int32)])
    got = _weighted_gpu(ihlib, ctx, hdl, wins, 16, kernel=ihlib.IH_K_MANHATTAN)
    _assert_weighted(got, oracle.weighted_hist(img, 16, wins, kernel=oracle.K_MANHATTAN))
    # a side above 256 is refused with 32-bit planes
    bad = torch.empty((1, 16), dtype=torch.float32, device=DEV)
    ihlib.ih_query_weighted(ctx, hdl, torch.tensor([[0, 0, 300, 10]], dtype=torch.int32, device=DEV), bad,
                            kernel=ihlib.IH_K_MANHATTAN)
    with pytest.raises(ihlib.IHError):
        ihlib.ih_sync(ctx)
    assert (bad == -1).all().item()
    ihlib.ih_release(ctx, hdl)


@pytest.mark.parametrize("layers", [0, 1, 3, 9])
@pytest.mark.parametrize("normalize", [False, True])
def test_wedding_cake_vs_direct_sum(ihlib, ctx, layers, normalize):
    h, w = 257, 333
    planes = np.stack([synth.blob_plane(h, w, 40 + k) for k in range(2)])
    hdl, _ = _build(ihlib, ctx, planes, [(5, 0), (12, 0)], weighted=1, layout=2)
    wins = np.concatenate([synth.rects_side_range(h, w, 600, 1, 64, 7),
                           synth.rects_side_range(h, w, 60, 32, 256, 8), _edge_windows(h, w)])
    got = _weighted_gpu(ihlib, ctx, hdl, wins, 12, normalize, kernel=ihlib.IH_K_WEDDING_CAKE, layers=layers)
    ref = oracle.weighted_hist(planes[1], 12, wins, normalize=normalize, kernel=oracle.K_WEDDING_CAKE,
                               layers=layers or 4)
    _assert_weighted(got, ref)
    ihlib.ih_release(ctx, hdl)


def test_weighted_kernel_arguments_refused(ihlib, ctx):
    img = synth.blob_plane(20, 30, 1)
    hdl, _ = _build(ihlib, ctx, img, [(8, 0)], weighted=0)
    d = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
    out = torch.empty((1, 8), device=DEV)
    for kernel, flags in [(3, 0), (0, 2), (2, ihlib.IH_LAYERS(65))]:
        with pytest.raises(ihlib.IHError):
            ihlib.ih_query_weighted(ctx, hdl, d, out, kernel=kernel, flags=flags)
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- sliding-window matching (Eq. 2.22)

@pytest.mark.parametrize("layout", [0, 1, 2])
def test_match_window_vs_oracle(ihlib, ctx, layout):
    h, w = 120, 170
    planes = np.stack([synth.blob_plane(h, w, 80), synth.blob_plane(h, w, 81)])
    chans = [(16, 0), (9, 0)]
    hdl, _ = _build(ihlib, ctx, planes, chans, layout=layout)
    wh, ww = 17, 23
    search = (5, 7, 5 + 60, 7 + 90)
    g = np.random.Generator(np.random.PCG64(9))
    t = g.integers(0, 30, size=25).astype(np.int32)
    ref0 = oracle.match_window(planes[0], 16, t[:16], wh, ww, search)
    ref1 = oracle.match_window(planes[1], 9, t[16:], wh, ww, search)
    for bin0, nbins, ref in ((0, 16, ref0), (16, 9, ref1), (0, 25, ref0 + ref1)):
        out = torch.full(ref.shape, -3, dtype=torch.int32, device=DEV)
        ihlib.ih_match_window(ctx, hdl, bin0, nbins, torch.from_numpy(t[bin0:bin0 + nbins].copy()).to(DEV), wh, ww,
                              search, out)
        ihlib.ih_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), ref), (bin0, nbins)
    # one placement covering the whole frame; a target equal to the window's
    # own histogram gives 0
    own = oracle.rect_hist(planes[0], 16, [[30, 40, 30 + wh - 1, 40 + ww - 1]])[0]
    one = torch.empty((1, 1), dtype=torch.int32, device=DEV)
    ihlib.ih_match_window(ctx, hdl, 0, 16, torch.from_numpy(own).to(DEV), wh, ww, (30, 40, 30, 40), one)
    full = torch.empty((1, 1), dtype=torch.int32, device=DEV)
    ihlib.ih_match_window(ctx, hdl, 0, 16, torch.from_numpy(t[:16].copy()).to(DEV), h, w, (0, 0, 0, 0), full)
    ihlib.ih_sync(ctx)
    assert one.item() == 0
    assert full.item() == int(oracle.match_window(planes[0], 16, t[:16], h, w, (0, 0, 0, 0))[0, 0])
    for bad in ((0, 0, h - wh + 1, 0), (0, -1, 0, 0)):
        with pytest.raises(ihlib.IHError):
            ihlib.ih_match_window(ctx, hdl, 0, 16, torch.from_numpy(t[:16].copy()).to(DEV), wh, ww, bad, out)
    with pytest.raises(ihlib.IHError):
        ihlib.ih_match_window(ctx, hdl, 20, 6, torch.from_numpy(t[:6].copy()).to(DEV), wh, ww, search, out)
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- Algorithm 4: joint IH and local median

@pytest.mark.parametrize("layout", [0, 1, 2])
def test_joint_ih_sliding_median(ihlib, ctx, layout):
    """Algorithm 4 over 9 frames with a temporal window of 5: the joint
    histogram is built from the first 5 integral histograms, then slid by
    adding the head frame and subtracting the tail; each step's local median
    matches the oracle's sort-based spatio-temporal median."""
    h, w, B, nf, T1 = 70, 90, 16, 9, 5
    frames = np.stack([synth.blob_plane(h, w, 90 + k) for k in range(nf)])
    pix = [torch.from_numpy(f).to(DEV)[None] for f in frames]
    hs = [ihlib.ih_build(ctx, ihlib.Frame(p, [(B, 0)], layout=layout))[0] for p in pix]
    jih, = ihlib.ih_build(ctx, ihlib.Frame(pix[0], [(B, 0)], layout=layout))
    for k in range(1, T1):
        ihlib.ih_accumulate(ctx, jih, add=hs[k])
    out = torch.empty((h, w), dtype=torch.int32, device=DEV)
    for start in range(0, nf - T1 + 1):
        if start:
            ihlib.ih_accumulate(ctx, jih, add=hs[start + T1 - 1], sub=hs[start - 1])
        for (m, n) in ((3, 5), (4, 2)):
            ihlib.ih_local_median(ctx, jih, 0, B, m, n, out)
            ihlib.ih_sync(ctx)
            ref = oracle.local_median(frames[start:start + T1], B, m, n)
            assert np.array_equal(out.cpu().numpy(), ref), (start, m, n)
    # the joint histogram's tensor is the sum of the window's tensors
    full = _export(ihlib, ctx, jih)
    ref = sum(oracle.integral_histogram(f, B).astype(np.int64) for f in frames[nf - T1:])
    assert np.array_equal(full, ref)
    # a single frame: the 2-D median filter; a bin range of another channel
    ihlib.ih_local_median(ctx, hs[0], 0, B, 7, 7, out)
    ihlib.ih_sync(ctx)
    assert np.array_equal(out.cpu().numpy(), oracle.local_median(frames[0], B, 7, 7))
    for hd in hs + [jih]:
        ihlib.ih_release(ctx, hd)


def test_accumulate_refuses_mismatched_frames(ihlib, ctx):
    a = torch.from_numpy(synth.blob_plane(20, 30, 1)).to(DEV)[None]
    b = torch.from_numpy(synth.blob_plane(20, 31, 2)).to(DEV)[None]
    ha, = ihlib.ih_build(ctx, ihlib.Frame(a, [(8, 0)]))
    hb, = ihlib.ih_build(ctx, ihlib.Frame(b, [(8, 0)]))
    hc, = ihlib.ih_build(ctx, ihlib.Frame(a, [(8, 0)], layout=1))
    hm, = ihlib.ih_build(ctx, ihlib.Frame(a, [(8, 0)], weighted_channel=0))
    for add in (hb, hc, hm):
        with pytest.raises(ihlib.IHError):
            ihlib.ih_accumulate(ctx, ha, add=add)
    with pytest.raises(ihlib.IHError):
        ihlib.ih_local_median(ctx, ha, 4, 5, 3, 3, torch.empty((20, 30), dtype=torch.int32, device=DEV))
    for hd in (ha, hb, hc, hm):
        ihlib.ih_release(ctx, hd)


# ---------------------------------------------------------------- Algorithm 2: spatial pyramid of orientations

def _canny_images():
    """Windows whose edges exercise every part of Canny's detector: blob
    content, uniform noise (many short weak runs), a bright block (long
    straight edges and corners), a constant window (no edges), single rows,
    columns and pixels, and a window that spans several 32 x 32 tiles with a
    ragged last tile."""
    g = synth.blob_plane(131, 203, 130)
    g[40:90, 60:150] = 235
    return [synth.blob_plane(64, 64, 131), synth.uniform_plane(45, 77, 132), g, np.full((20, 30), 77, np.uint8),
            synth.uniform_plane(1, 50, 133), synth.uniform_plane(50, 1, 134), np.zeros((1, 1), np.uint8),
            synth.blob_plane(257, 300, 135)]


@pytest.mark.parametrize("lo,hi", [(0, 0), (2, 6), (6, 24), (30, 90)])
def test_canny_edges_vs_oracle(ihlib, ctx, lo, hi):
    """Algorithm 2 step 1 on the GPU (tiled smoothing, gradient, suppression,
    union-find hysteresis) equals the oracle's sequential detector bit for
    bit, on whole windows and on a window with a row pitch."""
    for k, g in enumerate(_canny_images()):
        h, w = g.shape
        ref, _, _, _ = oracle.canny(g, lo, hi)
        out = torch.full((h, w), 7, dtype=torch.uint8, device=DEV)
        ihlib.ih_canny_edges(ctx, torch.from_numpy(g).to(DEV), lo, hi, out)
        ihlib.ih_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), ref), (k, lo, hi)
    g = _canny_images()[2]
    buf = torch.zeros((g.shape[0], g.shape[1] + 13), dtype=torch.uint8, device=DEV)
    buf[:, 5:5 + g.shape[1]] = torch.from_numpy(g).to(DEV)
    eb = torch.full((g.shape[0], g.shape[1] + 9), 7, dtype=torch.uint8, device=DEV)
    ihlib.ih_canny_edges(ctx, buf[:, 5:5 + g.shape[1]], lo, hi, eb[:, 3:3 + g.shape[1]])
    ihlib.ih_sync(ctx)
    e = eb.cpu().numpy()
    assert np.array_equal(e[:, 3:3 + g.shape[1]], oracle.canny(g, lo, hi)[0])
    assert (e[:, :3] == 7).all() and (e[:, 3 + g.shape[1]:] == 7).all()


def test_canny_edges_refusals(ihlib, ctx):
    g = torch.zeros((10, 10), dtype=torch.uint8, device=DEV)
    out = torch.empty((10, 10), dtype=torch.uint8, device=DEV)
    for lo, hi in ((-1, 4), (5, 4), (0, ihlib.IH_CANNY_MAX_THRESHOLD + 1)):
        with pytest.raises(ihlib.IHError):
            ihlib.ih_canny_edges(ctx, g, lo, hi, out)


@pytest.mark.parametrize("lo,hi", [(0, 0), (2, 6), (8, 40)])
def test_phog_descriptors_vs_oracle(ihlib, ctx, lo, hi):
    h, w = 130, 171
    g = synth.blob_plane(h, w, 120)
    hdl = ihlib.ih_phog_build(ctx, torch.from_numpy(g).to(DEV), lo, hi)
    info = ihlib.ih_info(ctx, hdl)
    assert info["total_bins"] == 9 and info["count_bytes"] == 0
    assert info["moment_bytes"] == 9 * h * ((w + 3) // 4 * 4) * 8
    bins, wt = oracle.phog_planes(g, lo, hi)
    assert (bins < 9).any()
    wins = np.concatenate([synth.rects_side_range(h, w, 40, 1, 100, 121),
                           np.array([[0, 0, h - 1, w - 1], [5, 6, 5, 6], [3, 4, 66, 131]], np.int32)])
    for L in (0, 2, 3):
        D = ihlib.phog_descriptor_len(L)
        out = torch.full((len(wins), D), -7, dtype=torch.int64, device=DEV)
        ihlib.ih_phog_descriptors(ctx, hdl, L, torch.from_numpy(wins).to(DEV), out)
        ihlib.ih_sync(ctx)
        got = out.cpu().numpy()
        for k, (r0, c0, r1, c1) in enumerate(wins):
            ref = oracle.phog_descriptor(bins, wt, L, r0, c0, r1 - r0 + 1, c1 - c0 + 1)
            assert np.array_equal(got[k], ref), (L, k)
    ihlib.ih_release(ctx, hdl)


def test_phog_match_map_vs_oracle(ihlib, ctx):
    h, w = 96, 128
    g = synth.blob_plane(h, w, 122)
    hdl = ihlib.ih_phog_build(ctx, torch.from_numpy(g).to(DEV), 2, 8)
    bins, wt = oracle.phog_planes(g, 2, 8)
    L, wh, ww = 2, 32, 40
    target = oracle.phog_descriptor(bins, wt, L, 30, 50, wh, ww)
    search = (20, 40, 20 + 23, 40 + 30)
    out = torch.empty((24, 31), dtype=torch.float32, device=DEV)
    ihlib.ih_phog_match(ctx, hdl, L, torch.from_numpy(target).to(DEV), wh, ww, search, out)
    ihlib.ih_sync(ctx)
    got = out.cpu().numpy().astype(np.float64)
    for i in range(24):
        for j in range(31):
            d = oracle.phog_descriptor(bins, wt, L, 20 + i, 40 + j, wh, ww)
            ref = oracle.pyramid_match(d, target, L)
            assert abs(got[i, j] - ref) <= 1e-6 * max(ref, 1.0), (i, j)
    # the best match is the target window itself (kappa(X, X) = its total)
    assert got[10, 10] == pytest.approx(float(target[:9].sum()), rel=1e-6)
    assert got.max() == pytest.approx(got[10, 10], rel=1e-6)
    with pytest.raises(ihlib.IHError):
        ihlib.ih_phog_match(ctx, hdl, L, torch.from_numpy(target).to(DEV), wh, ww, (0, 0, h - wh + 1, 0), out)
    with pytest.raises(ihlib.IHError):  # count-tensor calls refuse a pyramid frame
        ihlib.ih_query_rects(ctx, hdl, torch.zeros((1, 4), dtype=torch.int32, device=DEV),
                             torch.empty((1, 9), dtype=torch.int32, device=DEV))
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- record layout


def _record_words(bins):
    """Words per pixel of IH_LAYOUT_RECORD, from the rules stated in ih.h:
    groups of up to 8 consecutive bins from at most two channels, each taking
    8 words, packed into planes of at most 16 words."""
    groups = []  # [bins, channels] per group
    for nb in bins:
        left, first = nb, True
        while left:
            if not groups or groups[-1][0] == 8 or (first and groups[-1][1] == 2):
                groups.append([0, 0])
            g = groups[-1]
            if first or g[0] == 0:
                g[1] += 1
            take = min(8 - g[0], left)
            g[0] += take
            left -= take
            first = False
    planes, w = [], 0
    for n, _ in groups:
        wk = 8
        if w + wk > 16:
            planes.append(w)
            w = 0
        w += wk
    planes.append(w)
    return sum(planes), len(groups)


@pytest.mark.parametrize("bins", [[1], [3], [8], [9], [16, 9, 9, 9], [1, 1, 1, 1, 1], [5, 2, 1, 7, 20, 3],
                                  [13, 14, 15], [7, 1], [2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2]])
def test_record_layout_exact(ihlib, ctx, bins):
    """Record layout with groups that span two channels, cuts where a third
    channel would start, and zero padding: the tensor, its size, rectangle
    queries and the moment planes of a channel inside a shared group."""
    h, w = 75, 300
    chans = [(b, 0) for b in bins]
    planes = np.stack([synth.blob_plane(h, w, 70 + k) for k in range(len(bins))])
    wch = len(bins) // 2
    hdl, _ = _build(ihlib, ctx, planes, chans, weighted=wch, layout=2)
    info = ihlib.ih_info(ctx, hdl)
    words, _ = _record_words(bins)
    assert info["count_bytes"] == words * h * ((w + 3) // 4 * 4) * 4
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.frame_integral_histogram(planes, chans))
    rects = synth.rects_uniform_corners(h, w, 500, 91)
    d_r = torch.from_numpy(rects).to(DEV)
    out = torch.full((len(rects), sum(bins)), -5, dtype=torch.int32, device=DEV)
    ihlib.ih_query_rects(ctx, hdl, d_r, out)
    ihlib.ih_sync(ctx)
    assert np.array_equal(out.cpu().numpy(), oracle.frame_rect_hist(planes, chans, rects))
    bw = bins[wch]
    wins = synth.rects_side_range(h, w, 200, 1, 60, 92)
    _assert_weighted(_weighted_gpu(ihlib, ctx, hdl, wins, bw), oracle.weighted_hist(planes[wch], bw, wins))
    ihlib.ih_release(ctx, hdl)


# ---------------------------------------------------------------- both query kinds in one launch

@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_query_both_equals_separate_calls(ihlib, ctx, layout, kernel):
    """ih_query (one launch) returns exactly what ih_query_rects and
    ih_query_weighted return; the rectangles match the oracle exactly and the
    weighted windows the FP64 direct sum within 1e-5."""
    ih = ihlib
    h, w = 200, 611
    planes = np.stack([synth.blob_plane(h, w, 70 + k) for k in range(3)])
    chans = [(16, 0), (9, 0), (12, 0)]
    hdl, _ = _build(ih, ctx, planes, chans, weighted=0, layout=layout)
    rects = synth.rects_uniform_corners(h, w, 3000, 81)
    wins = synth.rects_side_range(h, w, 700, 1, 120, 82)
    d_r, d_w = (torch.from_numpy(x).to(DEV) for x in (rects, wins))
    r1 = torch.full((len(rects), 37), -7, dtype=torch.int32, device=DEV)
    w1 = torch.full((len(wins), 16), -7.0, dtype=torch.float32, device=DEV)
    r2, w2 = torch.full_like(r1, -9), torch.full_like(w1, -9.0)
    flags = ih.IH_NORMALIZE | ih.IH_LAYERS(3)
    ih.ih_query_rects(ctx, hdl, d_r, r1)
    ih.ih_query_weighted(ctx, hdl, d_w, w1, kernel=kernel, flags=flags)
    ih.ih_query(ctx, hdl, d_r, r2, d_w, w2, kernel=kernel, flags=flags)
    ih.ih_sync(ctx)
    assert torch.equal(r1, r2) and torch.equal(w1, w2)
    assert np.array_equal(r2.cpu().numpy(), oracle.frame_rect_hist(planes, chans, rects))
    _assert_weighted(w2.cpu().numpy(), oracle.weighted_hist(planes[0], 16, wins, normalize=True, kernel=kernel,
                                                            layers=3))
    ih.ih_release(ctx, hdl)


def test_query_both_partial_and_refusals(ihlib, ctx):
    ih = ihlib
    h, w = 90, 130
    img = synth.blob_plane(h, w, 5)
    hdl, _ = _build(ih, ctx, img, [(8, 0)])  # no moment planes
    rects = torch.from_numpy(synth.rects_uniform_corners(h, w, 50, 6)).to(DEV)
    out = torch.empty((50, 8), dtype=torch.int32, device=DEV)
    ih.ih_query(ctx, hdl, rects, out)  # rectangles only: accepted without moment planes
    ih.ih_sync(ctx)
    assert np.array_equal(out.cpu().numpy(), oracle.rect_hist(img, 8, rects.cpu().numpy()))
    wins = torch.zeros((3, 4), dtype=torch.int32, device=DEV)
    with pytest.raises(ih.IHError):  # windows need moment planes
        ih.ih_query(ctx, hdl, rects, out, wins, torch.empty((3, 8), device=DEV))
    ih.ih_release(ctx, hdl)
    # a rectangle outside the frame: its row is -1 and the call's sync fails
    hdl, _ = _build(ih, ctx, img, [(8, 0)], weighted=0)
    bad = torch.tensor([[0, 0, 5, 5], [0, 0, h, 3]], dtype=torch.int32, device=DEV)
    o = torch.zeros((2, 8), dtype=torch.int32, device=DEV)
    wo = torch.zeros((1, 8), dtype=torch.float32, device=DEV)
    ih.ih_query(ctx, hdl, bad, o, bad[:1], wo)
    with pytest.raises(ih.IHError):
        ih.ih_sync(ctx)
    assert (o[1] == -1).all().item() and np.array_equal(o[0].cpu().numpy(), oracle.rect_hist(img, 8, bad[:1].cpu().numpy())[0])
    ih.ih_release(ctx, hdl)


def test_plain_stream_order_gives_the_same_results(ihlib, ctx, tmp_path):
    """IH_PDL=0 (every launch in plain stream order, read once per process)
    builds and queries the same bits as the default programmatic launches."""
    import os
    import subprocess
    import sys
    h, w = 300, 700
    rgb = synth.blob_rgb(h, w, 91)
    rects = synth.rects_uniform_corners(h, w, 500, 92)
    wins = synth.rects_side_range(h, w, 200, 1, 100, 93)
    np.save(tmp_path / "rgb.npy", rgb)
    np.save(tmp_path / "rects.npy", rects)
    np.save(tmp_path / "wins.npy", wins)
    script = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_01656_gb300 import ih, synth
d = sys.argv[2]
rgb, rects, wins = (np.load(d + "/" + n + ".npy") for n in ("rgb", "rects", "wins"))
dev = torch.device("cuda:0")
c = ih.ih_create(0)
f = ih.Frame(torch.from_numpy(rgb).to(dev), synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES,
             weighted_channel=3, layout=ih.IH_LAYOUT_RECORD)
hd, = ih.ih_build(c, f)
full = torch.empty((91,) + rgb.shape[1:], dtype=torch.int32, device=dev)
ih.ih_export(c, hd, full)
r = torch.empty((len(rects), 91), dtype=torch.int32, device=dev)
wo = torch.empty((len(wins), 16), dtype=torch.float32, device=dev)
ih.ih_query(c, hd, torch.from_numpy(rects).to(dev), r, torch.from_numpy(wins).to(dev), wo)
ih.ih_sync(c)
np.save(d + "/out_" + sys.argv[3] + ".npy", np.concatenate([full.cpu().numpy().ravel().view(np.uint32),
        r.cpu().numpy().ravel().view(np.uint32), wo.cpu().numpy().ravel().view(np.uint32)]))
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for tag, pdl in (("pdl", "1"), ("plain", "0")):
        env = dict(os.environ, IH_PDL=pdl)
        subprocess.run([sys.executable, "-c", script, root, str(tmp_path), tag], env=env, check=True, timeout=600)
    a, b = np.load(tmp_path / "out_pdl.npy"), np.load(tmp_path / "out_plain.npy")
    assert np.array_equal(a, b)
    feats = oracle.features(rgb)
    full = a[:91 * h * w].view(np.int32).reshape(91, h, w)
    assert np.array_equal(full, oracle.frame_integral_histogram(feats, synth.FMV_CHANNELS))


# ---------------------------------------------------------------- tensor-core count tiles

@pytest.mark.parametrize("h,w,bins", [(1, 1, 4), (37, 53, 16), (128, 128, 8), (129, 257, 32), (300, 700, 16),
                                      (513, 385, 5)])
def test_build_mma_exact(ihlib, ctx, h, w, bins):
    """ih_build_mma (tiles as two chained tcgen05 products per bin) gives
    Algorithm 5's tensor bit for bit: single tiles, ragged tiles, several
    bands and strips of carries; its frame answers rectangle queries."""
    img = synth.blob_plane(h, w, 300 + h)
    hdl = ihlib.ih_build_mma(ctx, ihlib.Frame(torch.from_numpy(img).to(DEV)[None], [(bins, 0)]))
    assert np.array_equal(_export(ihlib, ctx, hdl), oracle.integral_histogram(img, bins))
    rects = synth.rects_uniform_corners(h, w, 300, 301)
    assert np.array_equal(_rects_gpu(ihlib, ctx, hdl, rects, bins).cpu().numpy(), oracle.rect_hist(img, bins, rects))
    ihlib.ih_release(ctx, hdl)


def test_build_mma_multichannel_and_refusals(ihlib, ctx):
    h, w = 200, 333
    planes = np.stack([synth.uniform_plane(h, w, 310), synth.blob_plane(h, w, 311)])
    planes[1] %= 9
    chans = [(24, 0), (9, 1)]
    hdl = ihlib.ih_build_mma(ctx, ihlib.Frame(torch.from_numpy(planes).to(DEV), chans))
    ref = oracle.frame_integral_histogram(planes, chans)
    assert np.array_equal(_export(ihlib, ctx, hdl), ref)
    ihlib.ih_release(ctx, hdl)
    pix = torch.from_numpy(planes).to(DEV)
    for bad in (ihlib.Frame(pix, chans, layout=ihlib.IH_LAYOUT_SLAB), ihlib.Frame(pix, chans, weighted_channel=0)):
        with pytest.raises(ihlib.IHError):
            ihlib.ih_build_mma(ctx, bad)


# ---------------------------------------------------------------- one-pass build of small frames

_ONEPASS_CASES = [
    (480, 640, [(16, 0)], 0),            # the plain 640 x 480 frame
    (9, 130, [(8, 0)], 0),               # one band, two strips, ragged
    (257, 2048, [(5, 0), (12, 1)], 1),   # 16 strips, slab layout, index channel
    (33, 129, [(40, 0)], 0),             # 5 groups of 8 bins
    (700, 300, [(3, 0)], 1),             # many bands: long look-back chains
]

_ONEPASS_SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_01656_gb300 import ih
d, n = sys.argv[2], int(sys.argv[4])
dev = torch.device("cuda:0")
c = ih.ih_create(0)
for k in range(n):
    z = np.load(d + "/case%d.npz" % k)
    planes, bins, modes, layout, rects = z["planes"], z["bins"], z["modes"], int(z["layout"]), z["rects"]
    chans = [(int(b), int(m)) for b, m in zip(bins, modes)]
    hd, = ih.ih_build(c, ih.Frame(torch.from_numpy(planes).to(dev), chans, layout=layout))
    B = int(bins.sum())
    t = torch.empty((B,) + planes.shape[1:], dtype=torch.int32, device=dev)
    ih.ih_export(c, hd, t)
    r = torch.empty((len(rects), B), dtype=torch.int32, device=dev)
    ih.ih_query_rects(c, hd, torch.from_numpy(rects).to(dev), r)
    ih.ih_sync(c)
    np.savez(d + "/out%d_%s.npz" % (k, sys.argv[3]), t=t.cpu().numpy(), r=r.cpu().numpy())
    ih.ih_release(c, hd)
ih.ih_destroy(c)
'''


def test_onepass_build_exact_and_equal_to_three_kernels(ihlib, tmp_path):
    """IH_ONEPASS=1 (read once per process) builds small frames without
    moment planes in one launch (column carries by decoupled look-back over
    bands): the tensors equal Algorithm 5, the rectangles the enumeration,
    and both equal the three-kernel build (IH_ONEPASS=0) bit for bit."""
    import os
    import subprocess
    import sys
    cases = []
    for k, (h, w, chans, layout) in enumerate(_ONEPASS_CASES):
        planes = np.stack([synth.blob_plane(h, w, 400 + 10 * k + c) for c in range(len(chans))])
        for c, (b, m) in enumerate(chans):
            if m == 1:
                planes[c] %= b + 2  # some values fall in no bin
        rects = synth.rects_uniform_corners(h, w, 300, 401 + k)
        np.savez(tmp_path / ("case%d.npz" % k), planes=planes, bins=np.array([b for b, _ in chans]),
                 modes=np.array([m for _, m in chans]), layout=layout, rects=rects)
        cases.append((planes, chans, rects))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for tag, one in (("one", "1"), ("three", "0")):
        env = dict(os.environ, IH_ONEPASS=one, IH_SMALL="0")
        subprocess.run([sys.executable, "-c", _ONEPASS_SCRIPT, root, str(tmp_path), tag, str(len(cases))], env=env,
                       check=True, timeout=600)
    for k, (planes, chans, rects) in enumerate(cases):
        one = np.load(tmp_path / ("out%d_one.npz" % k))
        three = np.load(tmp_path / ("out%d_three.npz" % k))
        assert np.array_equal(one["t"], three["t"]) and np.array_equal(one["r"], three["r"]), k
        assert np.array_equal(one["t"], oracle.frame_integral_histogram(planes, chans)), k
        assert np.array_equal(one["r"], oracle.frame_rect_hist(planes, chans, rects)), k


# ---------------------------------------------------------------- small-frame build (one cooperative launch)

_SMALL_CASES = [
    (480, 640, [(16, 0)], 0),            # the plain 640 x 480 frame
    (9, 130, [(8, 0)], 0),               # one band, two strips, the second 2 columns wide
    (257, 2048, [(5, 0), (12, 1)], 1),   # 16 strips, slab layout, index channel, groups of 5 and 6 bins
    (33, 129, [(40, 0)], 0),             # 5 groups of 8 bins
    (700, 300, [(3, 0)], 1),             # many bands
    (1, 1, [(4, 0)], 0),                 # one pixel
    (2, 3, [(2, 0)], 1),                 # the hand-worked frame's shape
    (1023, 1001, [(16, 0)], 0),          # ragged bands and strips, more rows per warp
    (720, 1280, [(16, 0)], 1),           # slab, eight rows per warp
]

_SMALL_SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1711_01656_gb300 import ih
d, n = sys.argv[2], int(sys.argv[4])
dev = torch.device("cuda:0")
c = ih.ih_create(0, flags=ih.IH_CFG_PROFILE)
for k in range(n):
    z = np.load(d + "/case%d.npz" % k)
    planes, bins, modes, layout, rects = z["planes"], z["bins"], z["modes"], int(z["layout"]), z["rects"]
    chans = [(int(b), int(m)) for b, m in zip(bins, modes)]
    ih.ih_profile_read(c, reset=True)
    hd, = ih.ih_build(c, ih.Frame(torch.from_numpy(planes).to(dev), chans, layout=layout))
    B = int(bins.sum())
    t = torch.empty((B,) + planes.shape[1:], dtype=torch.int32, device=dev)
    ih.ih_export(c, hd, t)
    r = torch.empty((len(rects), B), dtype=torch.int32, device=dev)
    ih.ih_query_rects(c, hd, torch.from_numpy(rects).to(dev), r)
    ih.ih_sync(c)
    kern = sorted(ih.ih_profile_read(c, reset=True))
    np.savez(d + "/out%d_%s.npz" % (k, sys.argv[3]), t=t.cpu().numpy(), r=r.cpu().numpy(),
             small=int("small_build" in kern))
    ih.ih_release(c, hd)
ih.ih_destroy(c)
'''


def test_small_build_exact_and_equal_to_three_kernels(ihlib, tmp_path):
    """Count-only frames that fit the GPU at once are built by one
    cooperative launch (tile sums, a bounded grid barrier, carries summed
    from the published sums, tiles): the tensors equal Algorithm 5, the
    rectangles the enumeration, and both equal the three-kernel build
    (IH_SMALL=0, read once per process) bit for bit."""
    import os
    import subprocess
    import sys
    cases = []
    for k, (h, w, chans, layout) in enumerate(_SMALL_CASES):
        planes = np.stack([synth.blob_plane(h, w, 500 + 10 * k + c) for c in range(len(chans))])
        for c, (b, m) in enumerate(chans):
            if m == 1:
                planes[c] %= b + 2  # some values fall in no bin
        rects = synth.rects_uniform_corners(h, w, 300, 501 + k)
        np.savez(tmp_path / ("case%d.npz" % k), planes=planes, bins=np.array([b for b, _ in chans]),
                 modes=np.array([m for _, m in chans]), layout=layout, rects=rects)
        cases.append((planes, chans, rects))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for tag, on in (("small", "1"), ("three", "0")):
        env = dict(os.environ, IH_SMALL=on, IH_ONEPASS="0")
        subprocess.run([sys.executable, "-c", _SMALL_SCRIPT, root, str(tmp_path), tag, str(len(cases))], env=env,
                       check=True, timeout=600)
    for k, (planes, chans, rects) in enumerate(cases):
        small = np.load(tmp_path / ("out%d_small.npz" % k))
        three = np.load(tmp_path / ("out%d_three.npz" % k))
        assert int(small["small"]) == 1 and int(three["small"]) == 0, k
        assert np.array_equal(small["t"], oracle.frame_integral_histogram(planes, chans)), k
        assert np.array_equal(small["r"], oracle.frame_rect_hist(planes, chans, rects)), k
        assert np.array_equal(small["t"], three["t"]) and np.array_equal(small["r"], three["r"]), k


@pytest.mark.parametrize("layout", [0, 1])
def test_small_build_repeated_and_graphed(ihlib, ctx, layout):
    """The grid barriers' counters are left zero by every launch: repeated
    builds, and a one-frame batch replayed as a CUDA graph (build and
    rectangles in one launch), give the same tensor and queries each time;
    an invalid rectangle's row is -1 and the status IH_EINVAL."""
    h, w = 480, 640
    img = synth.uniform_plane(h, w, synth.config_seed(1) + 7)
    rects = synth.rects_uniform_corners(h, w, 2000, 77)
    ref = oracle.integral_histogram(img, 16, threads=8)
    rref = oracle.rect_hist(img, 16, rects)
    pix = torch.from_numpy(img).to(DEV)[None]
    for _ in range(3):
        hdl, = ihlib.ih_build(ctx, ihlib.Frame(pix, [(16, 0)], layout=layout))
        assert np.array_equal(_export(ihlib, ctx, hdl), ref)
        ihlib.ih_release(ctx, hdl)
    bad = rects.copy()
    bad[5] = [10, 10, 9, 20]    # r0 > r1
    bad[1999] = [0, 0, h, 3]    # past the last row
    for rr, want in ((rects, rref), (bad, None)):
        d_rects = torch.from_numpy(rr).to(DEV)
        r_out = torch.full((len(rr), 16), -7, dtype=torch.int32, device=DEV)
        batch, handles = ihlib.ih_batch_create(ctx, [ihlib.Frame(pix, [(16, 0)], layout=layout)], rects=d_rects,
                                               rect_counts=[len(rr)], rect_out=r_out.view(-1),
                                               batch_flags=ihlib.IH_BATCH_GRAPH)
        try:
            for _ in range(5):
                r_out.fill_(-7)
                ihlib.ih_batch_run(ctx, batch)
                if want is not None:
                    ihlib.ih_sync(ctx)
                    assert np.array_equal(r_out.cpu().numpy(), want)
                else:
                    with pytest.raises(ihlib.IHError) as ei:
                        ihlib.ih_sync(ctx)
                    assert ei.value.status == ihlib.IH_EINVAL
                    g = r_out.cpu().numpy()
                    assert (g[5] == -1).all() and (g[1999] == -1).all()
                    keep = np.ones(len(rr), bool)
                    keep[[5, 1999]] = False
                    assert np.array_equal(g[keep], rref[keep])
            assert np.array_equal(_export(ihlib, ctx, handles[0]), ref)
        finally:
            ihlib.ih_batch_destroy(batch)
            for hd in handles:
                ihlib.ih_release(ctx, hd)
