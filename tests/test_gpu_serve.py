"""The serving loop: continuous batching of requests from many tracker
streams under an HBM budget.  Each request's results are the same alone and
in a mix (exactly: the arithmetic of a work item reads only its own frame),
admission respects the budget, and a tracker's previous frame is released
once its next one completes."""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _requests(ih, seed, n=14):
    g = np.random.Generator(np.random.PCG64(seed))
    sizes = [(120, 160), (72, 128), (200, 300), (33, 517), (256, 256)]
    out = []
    for k in range(n):
        h, w = sizes[int(g.integers(0, len(sizes)))]
        if k % 4 == 3:  # gray frame, 32 bins, 32-bit moment planes
            img = synth.blob_plane(h, w, seed + k)
            frame = ih.Frame(torch.from_numpy(img).to(DEV)[None], [(32, 0)], weighted_channel=0, layout=1,
                             moment_bits=32)
            B, Bw = 32, 32
        else:
            rgb = synth.blob_rgb(h, w, seed + k)
            frame = ih.Frame(torch.from_numpy(rgb).to(DEV), synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES,
                             weighted_channel=3, layout=k % 3)
            B, Bw = 91, 16
        rects = torch.from_numpy(synth.rects_uniform_corners(h, w, 200, seed * 7 + k)).to(DEV)
        wins = torch.from_numpy(synth.rects_side_range(h, w, 150, 1, 64, seed * 11 + k)).to(DEV)
        out.append(dict(tracker=k % 5, frame=frame, rects=rects, windows=wins,
                        rect_out=torch.full((200, B), -9, dtype=torch.int32, device=DEV),
                        weighted_out=torch.full((150, Bw), -9.0, dtype=torch.float32, device=DEV)))
    return out


def _serve(ih, ctx, reqs, streams, inflight, batch):
    srv = ih.ih_server_create(ctx, streams=streams, max_inflight=inflight, max_batch=batch)
    try:
        for k, r in enumerate(reqs):
            ih.ih_server_submit(ctx, srv, r["tracker"], r["frame"], rects=r["rects"], rect_out=r["rect_out"],
                                windows=r["windows"], weighted_out=r["weighted_out"], user=k)
        ih.ih_server_drain(srv)
        done = ih.ih_server_poll(srv, max=len(reqs) + 8)
    finally:
        ih.ih_server_destroy(srv)
    ih.ih_sync(ctx)
    return done


def test_results_same_alone_and_in_mix(ihlib, ctx):
    ih = ihlib
    alone = _requests(ih, 3)
    mixed = _requests(ih, 3)
    # alone: one request per tick, one tick at a time
    for r in alone:
        d = _serve(ih, ctx, [r], streams=1, inflight=1, batch=1)
        assert len(d) == 1 and d[0]["status"] == 0
    # mixed: all submitted at once, merged into ticks that overlap on 3 streams
    d = _serve(ih, ctx, mixed, streams=3, inflight=4, batch=6)
    assert sorted(c["user"] for c in d) == list(range(len(mixed)))
    assert all(c["status"] == 0 for c in d)
    assert all(c["t_submit"] <= c["t_admit"] <= c["t_done"] for c in d)
    for a, m in zip(alone, mixed):
        assert torch.equal(a["rect_out"], m["rect_out"])
        assert torch.equal(a["weighted_out"], m["weighted_out"])
    # and both against the oracle for a few requests
    for r in mixed[:4]:
        f = r["frame"]
        planes = f.pixels.cpu().numpy()
        if f.input == ih.IH_INPUT_RGB_FEATURES:
            planes, chans, wplane, bw = oracle.features(planes), synth.FMV_CHANNELS, 3, 16
        else:
            chans, wplane, bw = [(32, 0)], 0, 32
        rects, wins = r["rects"].cpu().numpy(), r["windows"].cpu().numpy()
        assert np.array_equal(r["rect_out"].cpu().numpy(), oracle.frame_rect_hist(planes, chans, rects))
        ref = oracle.weighted_hist(planes[wplane], bw, wins)
        got = r["weighted_out"].cpu().numpy().astype(np.float64)
        nz = ref != 0
        assert np.array_equal(got[~nz], ref[~nz])
        assert (np.abs(got[nz] - ref[nz]) <= 1e-5 * np.abs(ref[nz])).all()


def test_budget_admission_and_refusal(ihlib):
    ih = ihlib
    reqs = _requests(ih, 5, n=6)
    big = max(r["frame"].pixels.shape[1] * r["frame"].pixels.shape[2] for r in reqs)
    c = ih.ih_create(0, hbm_budget_bytes=int(big * (91 * 4 + 16 * 32) * 1.2))
    try:
        d = _serve(ih, c, reqs, streams=2, inflight=4, batch=4)
        assert all(x["status"] == 0 for x in d)
        # a frame larger than the whole budget completes with IH_EBUDGET
        img = torch.zeros((1, 2048, 2048), dtype=torch.uint8, device=DEV)
        huge = [dict(tracker=0, frame=ih.Frame(img, [(64, 0)]), rects=None, windows=None, rect_out=None,
                     weighted_out=None)]
        srv = ih.ih_server_create(c, streams=1, max_inflight=1, max_batch=1)
        ih.ih_server_submit(c, srv, 0, huge[0]["frame"])
        ih.ih_server_drain(srv)
        done = ih.ih_server_poll(srv)
        ih.ih_server_destroy(srv)
        assert len(done) == 1 and done[0]["status"] == ih.IH_EBUDGET
    finally:
        ih.ih_destroy(c)


def test_tracker_frames_stay_resident_until_superseded(ihlib, ctx):
    ih = ihlib
    img = synth.blob_plane(64, 96, 1)
    f = ih.Frame(torch.from_numpy(img).to(DEV)[None], [(8, 0)])
    srv = ih.ih_server_create(ctx, streams=1, max_inflight=1, max_batch=1)
    try:
        ih.ih_server_submit(ctx, srv, 7, f, user=1)
        ih.ih_server_drain(srv)
        first = ih.ih_server_poll(srv)[0]
        info = ih.ih_info(ctx, first["handle"])  # resident
        assert info["height"] == 64
        out = torch.empty((8, 64, 96), dtype=torch.int32, device=DEV)
        ih.ih_export(ctx, first["handle"], out)
        ih.ih_sync(ctx)
        assert np.array_equal(out.cpu().numpy(), oracle.integral_histogram(img, 8))
        ih.ih_server_submit(ctx, srv, 7, f, user=2)
        ih.ih_server_drain(srv)
        second = ih.ih_server_poll(srv)[0]
        assert first["handle"] != second["handle"]
        with pytest.raises(ih.IHError):
            ih.ih_info(ctx, first["handle"])
        assert ih.ih_info(ctx, second["handle"])["height"] == 64
    finally:
        ih.ih_server_destroy(srv)


def test_invalid_request_rejected_at_submit(ihlib, ctx):
    ih = ihlib
    srv = ih.ih_server_create(ctx, streams=1, max_inflight=1, max_batch=1)
    try:
        img = torch.zeros((1, 8, 8), dtype=torch.uint8, device=DEV)
        with pytest.raises(ih.IHError):
            ih.ih_server_submit(ctx, srv, 0, ih.Frame(img, [(0, 0)]))
        with pytest.raises(ih.IHError):  # windows without a weighted channel
            w = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
            ih.ih_server_submit(ctx, srv, 0, ih.Frame(img, [(4, 0)]), windows=w,
                                weighted_out=torch.empty((1, 4), device=DEV))
    finally:
        ih.ih_server_destroy(srv)


def test_cancel_queued_and_inflight_requests(ihlib):
    """ih_server_cancel: a queued request leaves the queue and completes with
    IH_ECANCELLED; a request already on the device completes with
    IH_ECANCELLED when its tick finishes and is not kept resident, so its
    bytes return to the budget (a later request of the same size is admitted
    and completes); the other requests complete with their results; an
    unknown tag is refused."""
    ih = ihlib
    big = torch.from_numpy(synth.blob_plane(4096, 4096, 41)).to(DEV)[None]
    fbig = ih.Frame(big, [(32, 0)], weighted_channel=0)
    big_bytes = 4096 * 4096 * (32 * 4 + 4 * 32 * 8)
    c = ih.ih_create(0, hbm_budget_bytes=int(big_bytes * 1.3))
    small = [synth.blob_plane(96, 128, 50 + k) for k in range(3)]
    outs = [torch.full((40, 8), -9, dtype=torch.int32, device=DEV) for _ in small]
    rects = torch.from_numpy(synth.rects_uniform_corners(96, 128, 40, 51)).to(DEV)
    srv = ih.ih_server_create(c, streams=1, max_inflight=1, max_batch=1)
    try:
        ih.ih_server_submit(c, srv, 0, fbig, user=100)
        keep = [torch.from_numpy(img).to(DEV)[None] for img in small]  # valid until the requests complete
        for k in range(len(small)):
            ih.ih_server_submit(c, srv, 1 + k, ih.Frame(keep[k], [(8, 0)]), rects=rects, rect_out=outs[k],
                                user=200 + k)
        ih.ih_server_cancel(srv, 201)  # queued behind the 4096 x 4096 frame
        ih.ih_server_cancel(srv, 100)  # on the device, or about to be
        with pytest.raises(ih.IHError):
            ih.ih_server_cancel(srv, 999)
        ih.ih_server_drain(srv)
        done = {d["user"]: d for d in ih.ih_server_poll(srv, max=16)}
        assert sorted(done) == [100, 200, 201, 202]
        assert done[100]["status"] == ih.IH_ECANCELLED and done[100]["handle"] == -1
        assert done[201]["status"] == ih.IH_ECANCELLED and done[201]["handle"] == -1
        assert (outs[1] == -9).all()  # the cancelled request's queries never ran
        for k in (0, 2):
            assert done[200 + k]["status"] == 0
            assert np.array_equal(outs[k].cpu().numpy(), oracle.rect_hist(small[k], 8, rects.cpu().numpy()))
        with pytest.raises(ih.IHError):  # completed requests cannot be cancelled
            ih.ih_server_cancel(srv, 200)
        # only the two small frames stay resident: the cancelled frame is released
        assert ih.ih_memory_used(c) == 2 * 8 * 96 * 128 * 4
        # the cancelled frame's bytes are back in the budget: another frame of
        # the same size fits (nothing resident is large enough to evict for it)
        ih.ih_server_submit(c, srv, 5, fbig, user=300)
        ih.ih_server_drain(srv)
        last = ih.ih_server_poll(srv, max=4)
        assert len(last) == 1 and last[0]["user"] == 300 and last[0]["status"] == 0
    finally:
        ih.ih_server_destroy(srv)
        ih.ih_destroy(c)
        torch.cuda.empty_cache()
