"""Batched builds (one launch per kernel over many frames, CUDA graph
replay, autotuned tile grids) give exactly what per-frame builds give, and
per-frame builds match the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _frames(ih, seed):
    """Uneven frames: sizes, channel sets, bin counts, layouts and weighted
    channels all differ."""
    g = np.random.Generator(np.random.PCG64(seed))
    specs = []
    sizes = [(48, 64), (130, 300), (77, 1030), (257, 129), (1, 9), (200, 200)]
    for k, (h, w) in enumerate(sizes):
        layout = k % 3
        if k % 3 == 0:
            rgb = synth.blob_rgb(h, w, seed + k)
            pix = torch.from_numpy(rgb).to(DEV)
            chans = synth.FMV_CHANNELS
            f = ih.Frame(pix, chans, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=3 if k % 2 == 0 else -1,
                         layout=layout)
            planes = oracle.features(rgb)
        else:
            nch = 1 + k % 3
            chans = [(int(g.integers(1, 40)), 0) for _ in range(nch)]
            planes = np.stack([synth.blob_plane(h, w, seed + 10 * k + c) for c in range(nch)])
            pix = torch.from_numpy(planes).to(DEV)
            f = ih.Frame(pix, chans, weighted_channel=(nch - 1) if k % 2 else -1, layout=layout)
        specs.append((f, planes, chans))
    return specs


def _export(ih, ctx, h):
    info = ih.ih_info(ctx, h)
    out = torch.empty((info["total_bins"], info["height"], info["width"]), dtype=torch.int32, device=DEV)
    ih.ih_export(ctx, h, out)
    return out


def _moments(ih, ctx, h):
    info = ih.ih_info(ctx, h)
    if info["weighted_bins"] == 0:
        return None
    outs = []
    for p in range(4):
        o = torch.empty((info["weighted_bins"], info["height"], info["width"]), dtype=torch.int64, device=DEV)
        ih.ih_export_moments(ctx, h, p, o)
        outs.append(o)
    return torch.stack(outs)


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_single_and_oracle(ihlib, ctx, graph, persistent):
    """Every frame of a batch -- one launch per kernel, or the whole build in
    one persistent launch (IH_BATCH_PERSISTENT) -- equals its single build,
    which equals the oracle; so do its queries; twice in a row."""
    ih = ihlib
    specs = _frames(ih, 11)
    frames = [s[0] for s in specs]
    # queries: rectangles for every frame, weighted windows for weighted frames
    rc, wc, rects, wins, win_of = [], [], [], [], {}
    for k, (f, planes, chans) in enumerate(specs):
        h, w = f.pixels.shape[1], f.pixels.shape[2]
        r = synth.rects_uniform_corners(h, w, 37, h + w)
        rects.append(r)
        rc.append(len(r))
        if f.weighted_channel >= 0:
            q = synth.rects_side_range(h, w, 23, 1, 64, h * w)
            wins.append(q)
            win_of[k] = q
            wc.append(len(q))
        else:
            wc.append(0)
    B = [sum(b for b, _ in s[2]) for s in specs]
    Bw = [s[2][s[0].weighted_channel][0] if s[0].weighted_channel >= 0 else 0 for s in specs]
    d_rects = torch.from_numpy(np.concatenate(rects)).to(DEV)
    d_wins = torch.from_numpy(np.concatenate(wins)).to(DEV)
    rect_out = torch.full((sum(n * b for n, b in zip(rc, B)),), -7, dtype=torch.int32, device=DEV)
    w_out = torch.full((sum(n * b for n, b in zip(wc, Bw)),), -7.0, dtype=torch.float32, device=DEV)
    batch, handles = ih.ih_batch_create(ctx, frames, rects=d_rects, rect_counts=rc, rect_out=rect_out,
                                        windows=d_wins, window_counts=wc, weighted_out=w_out,
                                        batch_flags=(ih.IH_BATCH_GRAPH if graph else 0) |
                                        (ih.IH_BATCH_PERSISTENT if persistent else 0))
    try:
        for run in range(2):  # a second run (graph replay) gives the same results
            if run:
                rect_out.fill_(-7)
                w_out.fill_(-7.0)
            ih.ih_batch_run(ctx, batch)
            ih.ih_sync(ctx)
            ro, wo = 0, 0
            for k, (f, planes, chans) in enumerate(specs):
                got = _export(ih, ctx, handles[k])
                single, = ih.ih_build(ctx, f)
                ref = _export(ih, ctx, single)
                ih.ih_sync(ctx)
                assert torch.equal(got, ref), "frame %d counts" % k
                if run == 0:
                    assert np.array_equal(got.cpu().numpy(), oracle.frame_integral_histogram(planes, chans))
                gm, sm = _moments(ih, ctx, handles[k]), _moments(ih, ctx, single)
                assert (gm is None) == (sm is None)
                if gm is not None:
                    assert torch.equal(gm, sm), "frame %d moments" % k
                # queries against the single frame's own queries
                d_r = torch.from_numpy(rects[k]).to(DEV)
                sr = torch.empty((rc[k], B[k]), dtype=torch.int32, device=DEV)
                ih.ih_query_rects(ctx, single, d_r, sr)
                assert torch.equal(rect_out[ro:ro + rc[k] * B[k]].view(rc[k], B[k]), sr), "frame %d rects" % k
                ro += rc[k] * B[k]
                if wc[k]:
                    wi = win_of[k]
                    sw = torch.empty((wc[k], Bw[k]), dtype=torch.float32, device=DEV)
                    ih.ih_query_weighted(ctx, single, torch.from_numpy(wi).to(DEV), sw)
                    assert torch.equal(w_out[wo:wo + wc[k] * Bw[k]].view(wc[k], Bw[k]), sw), "frame %d weighted" % k
                    wo += wc[k] * Bw[k]
                ih.ih_sync(ctx)
                ih.ih_release(ctx, single)
    finally:
        ih.ih_batch_destroy(batch)
        for h in handles:
            ih.ih_release(ctx, h)


def test_autotune_then_build_exact(ihlib, ctx):
    ih = ihlib
    h, w = 300, 1100
    rgb = synth.blob_rgb(h, w, 5)
    f = ih.Frame(torch.from_numpy(rgb).to(DEV), synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES,
                 weighted_channel=3, layout=ih.IH_LAYOUT_SLAB)
    ih.ih_autotune(ctx, f)
    hdl, = ih.ih_build(ctx, f)
    info = ih.ih_info(ctx, hdl)
    assert info["tile_rows"] in (8, 16, 32, 64, 128) and info["tile_cols"] in (128, 256, 512, 1024, 1152)
    got = _export(ih, ctx, hdl).cpu().numpy()
    assert np.array_equal(got, oracle.frame_integral_histogram(oracle.features(rgb), synth.FMV_CHANNELS))
    ih.ih_release(ctx, hdl)


def test_batch_autotune_flag(ihlib, ctx):
    ih = ihlib
    imgs = [synth.blob_plane(100 + 37 * k, 150 + 91 * k, k) for k in range(3)]
    frames = [ih.Frame(torch.from_numpy(im).to(DEV)[None], [(16, 0)], weighted_channel=0) for im in imgs]
    batch, handles = ih.ih_batch_create(ctx, frames, batch_flags=ih.IH_BATCH_AUTOTUNE | ih.IH_BATCH_GRAPH)
    try:
        ih.ih_batch_run(ctx, batch)
        ih.ih_sync(ctx)
        for im, hdl in zip(imgs, handles):
            assert np.array_equal(_export(ih, ctx, hdl).cpu().numpy(), oracle.integral_histogram(im, 16))
            mo = _moments(ih, ctx, hdl).cpu().numpy()
            for p, wk in enumerate(oracle.MOMENT_WEIGHTS):
                assert np.array_equal(mo[p], oracle.weighted_integral_histogram(im, 16, wk))
    finally:
        ih.ih_batch_destroy(batch)
        for hdl in handles:
            ih.ih_release(ctx, hdl)


@pytest.mark.parametrize("kernel,layers", [(1, 0), (2, 5)])
def test_batch_other_kernels_equal_single(ihlib, ctx, kernel, layers):
    """Batched weighted queries with the Manhattan kernel or the wedding cake
    give exactly the single-frame queries, which match the oracle."""
    ih = ihlib
    sizes = [(90, 130), (33, 517), (200, 200)]
    imgs = [synth.blob_plane(h, w, 60 + k) for k, (h, w) in enumerate(sizes)]
    frames = [ih.Frame(torch.from_numpy(im).to(DEV)[None], [(16, 0)], weighted_channel=0, layout=k % 3)
              for k, im in enumerate(imgs)]
    wins = [synth.rects_side_range(h, w, 50, 1, 80, 70 + k) for k, (h, w) in enumerate(sizes)]
    d_w = torch.from_numpy(np.concatenate(wins)).to(DEV)
    w_out = torch.full((sum(len(x) for x in wins) * 16,), -9.0, dtype=torch.float32, device=DEV)
    flags = ih.IH_LAYERS(layers)
    batch, handles = ih.ih_batch_create(ctx, frames, windows=d_w, window_counts=[len(x) for x in wins],
                                        weighted_out=w_out, kernel=kernel, flags=flags)
    try:
        ih.ih_batch_run(ctx, batch)
        ih.ih_sync(ctx)
        off = 0
        for k, (im, hdl) in enumerate(zip(imgs, handles)):
            n = len(wins[k])
            single = torch.empty((n, 16), dtype=torch.float32, device=DEV)
            ih.ih_query_weighted(ctx, hdl, torch.from_numpy(wins[k]).to(DEV), single, kernel=kernel, flags=flags)
            ih.ih_sync(ctx)
            assert torch.equal(w_out[off:off + n * 16].view(n, 16), single)
            off += n * 16
            ref = oracle.weighted_hist(im, 16, wins[k], kernel=kernel, layers=layers or 4)
            got = single.cpu().numpy().astype(np.float64)
            nz = ref != 0
            assert np.array_equal(got[~nz], ref[~nz])
            assert (np.abs(got[nz] - ref[nz]) <= 1e-5 * np.abs(ref[nz])).all()
    finally:
        ih.ih_batch_destroy(batch)
        for hdl in handles:
            ih.ih_release(ctx, hdl)


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("layout", [0, 2])
def test_one_frame_batch(ihlib, ctx, graph, layout, persistent):
    """A batch of one frame (run with the single-frame kernels) gives the
    same tensor, rectangles and weighted windows as ih_build + ih_query."""
    ih = ihlib
    h, w = 333, 517
    rgb = torch.from_numpy(synth.blob_rgb(h, w, 61)).to(DEV)
    f = ih.Frame(rgb, synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=3, layout=layout)
    rects = torch.from_numpy(synth.rects_uniform_corners(h, w, 300, 62)).to(DEV)
    wins = torch.from_numpy(synth.rects_side_range(h, w, 120, 1, 90, 63)).to(DEV)
    r_out = torch.full((300 * 91,), -7, dtype=torch.int32, device=DEV)
    w_out = torch.full((120 * 16,), -7.0, dtype=torch.float32, device=DEV)
    batch, handles = ih.ih_batch_create(ctx, [f], rects=rects, rect_counts=[300], rect_out=r_out, windows=wins,
                                        window_counts=[120], weighted_out=w_out,
                                        batch_flags=(ih.IH_BATCH_GRAPH if graph else 0) |
                                        (ih.IH_BATCH_PERSISTENT if persistent else 0))
    try:
        ih.ih_batch_run(ctx, batch)
        ih.ih_sync(ctx)
        single, = ih.ih_build(ctx, f)
        sr = torch.empty((300, 91), dtype=torch.int32, device=DEV)
        sw = torch.empty((120, 16), dtype=torch.float32, device=DEV)
        ih.ih_query(ctx, single, rects, sr, wins, sw)
        ih.ih_sync(ctx)
        assert torch.equal(_export(ih, ctx, handles[0]), _export(ih, ctx, single))
        assert torch.equal(r_out.view(300, 91), sr) and torch.equal(w_out.view(120, 16), sw)
        feats = oracle.features(rgb.cpu().numpy())
        assert np.array_equal(sr.cpu().numpy(), oracle.frame_rect_hist(feats, synth.FMV_CHANNELS, rects.cpu().numpy()))
        ih.ih_release(ctx, single)
    finally:
        ih.ih_batch_destroy(batch)
        for hd in handles:
            ih.ih_release(ctx, hd)


def test_persistent_batch_of_many_frames(ihlib, ctx):
    """A persistent batch of 24 frames of mixed sizes (several waves of CTAs
    over the work items, frames of one tile and of many) equals per-frame
    builds, and ih_sync reports no device-side timeout."""
    ih = ihlib
    g = np.random.Generator(np.random.PCG64(77))
    sizes = [(int(g.integers(1, 700)), int(g.integers(1, 900))) for _ in range(24)]
    imgs = [synth.blob_plane(h, w, 900 + k) for k, (h, w) in enumerate(sizes)]
    pix = [torch.from_numpy(x).to(DEV)[None] for x in imgs]
    frames = [ih.Frame(p, [(int(g.integers(1, 64)), 0)], weighted_channel=0 if k % 3 == 0 else -1, layout=k % 3)
              for k, p in enumerate(pix)]
    batch, handles = ih.ih_batch_create(ctx, frames, batch_flags=ih.IH_BATCH_PERSISTENT | ih.IH_BATCH_GRAPH)
    try:
        for _ in range(3):
            ih.ih_batch_run(ctx, batch)
        ih.ih_sync(ctx)
        for k, f in enumerate(frames):
            single, = ih.ih_build(ctx, f)
            assert torch.equal(_export(ih, ctx, handles[k]), _export(ih, ctx, single)), "frame %d" % k
            gm, sm = _moments(ih, ctx, handles[k]), _moments(ih, ctx, single)
            assert (gm is None) == (sm is None) and (gm is None or torch.equal(gm, sm))
            ih.ih_release(ctx, single)
        ih.ih_sync(ctx)
        k = int(np.argmax([h * w for h, w in sizes]))
        assert np.array_equal(_export(ih, ctx, handles[k]).cpu().numpy(),
                              oracle.integral_histogram(imgs[k], frames[k].channels[0][0]))
    finally:
        ih.ih_batch_destroy(batch)
        for hd in handles:
            ih.ih_release(ctx, hd)


def test_bounded_wait_gives_up_and_context_stays_usable(ihlib, ctx):
    """The device-side wait of the persistent build gives up after its poll
    limit when its producer never finishes (here: a counter nothing raises):
    ih_sync reports IH_ETIMEOUT once, and the context then builds exactly."""
    ih = ihlib
    ih.ih_wait_selftest(ctx, 20000)
    with pytest.raises(ih.IHError) as e:
        ih.ih_sync(ctx)
    assert e.value.status == ih.IH_ETIMEOUT
    ih.ih_sync(ctx)  # the error word was cleared
    img = synth.blob_plane(70, 90, 5)
    h, = ih.ih_build(ctx, ih.Frame(torch.from_numpy(img).to(DEV)[None], [(8, 0)]))
    assert np.array_equal(_export(ih, ctx, h).cpu().numpy(), oracle.integral_histogram(img, 8))
    ih.ih_release(ctx, h)
    with pytest.raises(ih.IHError):
        ih.ih_wait_selftest(ctx, 0)
