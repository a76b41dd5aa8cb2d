"""Full-size workloads, in the configuration bench.py and the batch use,
checked on outputs the oracle can compute one by one and on properties that
hold at any size.

* WAMI: one 8192 x 8192 blob frame, 32 bins, slab layout, int64 moment
  planes (77 GB on the device); 1,000,000 rectangles of side 16..256 and
  100,000 weighted windows of side 32..256.
* Batched: 64 uneven FMV frames (sizes drawn from {640x480, 1280x720,
  1920x1080, 4096x2160}) with intensity moments and 4,096 weighted windows
  each, one graph-replayed batch.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
WTOL = 1e-5


def _assert_weighted(got, ref):
    got = np.asarray(got, dtype=np.float64)
    z = ref == 0
    assert np.array_equal(got[z], ref[z])
    assert (np.abs(got[~z] - ref[~z]) <= WTOL * np.abs(ref[~z])).all()


def test_wami_8192_full_size(ihlib):
    ih = ihlib
    H = W = 8192
    B = 32
    img = synth.blob_plane(H, W, synth.config_seed(3))
    c = ih.ih_create(0)
    try:
        pix = torch.from_numpy(img).to(DEV)[None]
        h, = ih.ih_build(c, ih.Frame(pix, [(B, 0)], weighted_channel=0, layout=ih.IH_LAYOUT_SLAB))
        rects = synth.rects_side_range(H, W, 1_000_000, 16, 256, synth.config_seed(3) + 100)
        wins = synth.rects_side_range(H, W, 100_000, 32, 256, synth.config_seed(3) + 200)
        d_r = torch.from_numpy(rects).to(DEV)
        d_w = torch.from_numpy(wins).to(DEV)
        r_out = torch.empty((len(rects), B), dtype=torch.int32, device=DEV)
        w_out = torch.empty((len(wins), B), dtype=torch.float32, device=DEV)
        ih.ih_query_rects(c, h, d_r, r_out)
        ih.ih_query_weighted(c, h, d_w, w_out)
        ih.ih_sync(c)
        g = np.random.Generator(np.random.PCG64(31))
        sr = g.choice(len(rects), 3000, replace=False)
        assert np.array_equal(r_out[torch.from_numpy(sr).to(DEV)].cpu().numpy(), oracle.rect_hist(img, B, rects[sr]))
        sw = g.choice(len(wins), 1000, replace=False)
        _assert_weighted(w_out[torch.from_numpy(sw).to(DEV)].cpu().numpy(), oracle.weighted_hist(img, B, wins[sw]))
        # the Manhattan kernel (Eq. 3.3) and the wedding cake (Eq. 3.2) on the same windows
        for kernel in (ih.IH_K_MANHATTAN, ih.IH_K_WEDDING_CAKE):
            ih.ih_query_weighted(c, h, d_w, w_out, kernel=kernel)
            ih.ih_sync(c)
            s2 = sw[:300]
            _assert_weighted(w_out[torch.from_numpy(s2).to(DEV)].cpu().numpy(),
                             oracle.weighted_hist(img, B, wins[s2], kernel=kernel, layers=4))
        del r_out, w_out
        # the tensor: exact on a top-left crop (the integral histogram of a
        # top-left crop is the crop of the integral histogram), invariants on
        # sampled full rows and columns
        full = torch.empty((B, H, W), dtype=torch.int32, device=DEV)
        ih.ih_export(c, h, full)
        ih.ih_sync(c)
        cr, cc = 640, 704
        assert np.array_equal(full[:, :cr, :cc].cpu().numpy(), oracle.integral_histogram(img[:cr, :cc], B))
        for r in (0, 4095, 8191):
            tot = full[:, r, :].sum(dim=0).cpu().numpy().astype(np.int64)
            assert np.array_equal(tot, (r + 1) * np.arange(1, W + 1, dtype=np.int64))
        col = full[:, :, W - 1].sum(dim=0).cpu().numpy().astype(np.int64)
        assert np.array_equal(col, W * np.arange(1, H + 1, dtype=np.int64))
        assert (full[:, 1:, 5000] >= full[:, :-1, 5000]).all().item()
        last = full[:, H - 1, W - 1].cpu().numpy()
        assert np.array_equal(last, np.bincount((img.astype(np.int64) * B // 256).ravel(), minlength=B))
        del full
        # moment planes on the crop
        plane = torch.empty((B, H, W), dtype=torch.int64, device=DEV)
        for p, wk in enumerate(oracle.MOMENT_WEIGHTS):
            ih.ih_export_moments(c, h, p, plane)
            ih.ih_sync(c)
            assert np.array_equal(plane[:, :cr, :cc].cpu().numpy(),
                                  oracle.weighted_integral_histogram(img[:cr, :cc], B, wk)), "plane %d" % p
        del plane
        ih.ih_release(c, h)
    finally:
        ih.ih_destroy(c)
        torch.cuda.empty_cache()


def test_batched_64_uneven_frames(ihlib):
    ih = ihlib
    sizes = synth.frame_sizes_batched(64, synth.config_seed(4))
    base = {s: synth.blob_rgb(s[0], s[1], 1000 + s[0]) for s in set(sizes)}
    rgbs = [np.roll(base[s], 37 * k, axis=2) for k, s in enumerate(sizes)]
    c = ih.ih_create(0)
    try:
        pix = [torch.from_numpy(x).to(DEV) for x in rgbs]
        frames = [ih.Frame(p, synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=3,
                           layout=ih.IH_LAYOUT_SLAB) for p in pix]
        nw = 4096
        wins = [synth.rects_side_range(h, w, nw, 32, 256, 77 + k) for k, (h, w) in enumerate(sizes)]
        d_w = torch.from_numpy(np.concatenate(wins)).to(DEV)
        w_out = torch.empty(64 * nw * 16, dtype=torch.float32, device=DEV)
        batch, handles = ih.ih_batch_create(c, frames, windows=d_w, window_counts=[nw] * 64, weighted_out=w_out,
                                            batch_flags=ih.IH_BATCH_GRAPH)
        try:
            ih.ih_batch_run(c, batch)
            ih.ih_batch_run(c, batch)
            ih.ih_sync(c)
            g = np.random.Generator(np.random.PCG64(4))
            picks = [int(np.argmin([h * w for h, w in sizes])), int(np.argmax([h * w for h, w in sizes]))]
            picks += [int(k) for k in g.choice(64, 2, replace=False)]
            for k in picks:
                h, w = sizes[k]
                feats = oracle.features(rgbs[k])
                out = torch.empty((91, h, w), dtype=torch.int32, device=DEV)
                ih.ih_export(c, handles[k], out)
                ih.ih_sync(c)
                cr, cc = min(h, 300), min(w, 520)
                ref = oracle.frame_integral_histogram(feats[:, :cr, :cc], synth.FMV_CHANNELS)
                assert np.array_equal(out[:, :cr, :cc].cpu().numpy(), ref), "frame %d" % k
                tot = out[:, h - 1, :].sum(dim=0).cpu().numpy().astype(np.int64)
                assert np.array_equal(tot, 7 * h * np.arange(1, w + 1, dtype=np.int64))
                got = w_out[k * nw * 16:(k + 1) * nw * 16].view(nw, 16).cpu().numpy()
                s = g.choice(nw, 200, replace=False)
                _assert_weighted(got[s], oracle.weighted_hist(feats[3], 16, wins[k][s]))
        finally:
            ih.ih_batch_destroy(batch)
            for hd in handles:
                ih.ih_release(c, hd)
    finally:
        ih.ih_destroy(c)
        torch.cuda.empty_cache()
