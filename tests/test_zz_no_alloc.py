"""The allocation-free count build (ih_build_counts_static).

Some callers cannot allocate device memory while they run -- a real-time
tracking loop whose memory is reserved up front by its own arena, where a
cudaMalloc would synchronise the device, or an application whose allocator
owns all device memory.  For them the library keeps the tile carries in one
static device array instead of allocating them.  This file checks, through
the C ABI, that the static variant produces exactly the tensor that ih_build
produces, on two calls in a row (the array keeps the previous call's
contents), and that a frame too large for the array is refused.  It runs
last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _reference(ihlib, ctx, img, bins, mode):
    pix = torch.from_numpy(np.ascontiguousarray(img)).to(DEV)[None]
    h, = ihlib.ih_build(ctx, ihlib.Frame(pix, [(bins, mode)]))
    out = torch.empty((bins,) + img.shape, dtype=torch.int32, device=DEV)
    ihlib.ih_export(ctx, h, out)
    ihlib.ih_sync(ctx)
    ihlib.ih_release(ctx, h)
    return out.cpu().numpy()


CASES = [((480, 640), 16, 0, 1), ((1080, 1920), 16, 0, 2), ((301, 517), 9, 1, 3), ((1, 5), 3, 0, 4),
         ((77, 1030), 32, 0, 5)]


@pytest.mark.parametrize("shape,bins,mode,seed", CASES)
def test_static_matches_ih_build_twice(ihlib, ctx, shape, bins, mode, seed):
    h, w = shape
    pitch = (w + 3) // 4 * 4 + 4
    results = []
    for call in range(2):  # two calls in a row, different frames
        img = synth.blob_plane(h, w, seed * 10 + call)
        if mode == 1:
            img = (img % 12).astype(np.uint8)
        ref = _reference(ihlib, ctx, img, bins, mode)
        out = torch.full((bins, h, pitch), -7, dtype=torch.int32, device=DEV)
        ihlib.ih_build_counts_static(torch.from_numpy(img).to(DEV), bins, mode, out)
        torch.cuda.synchronize()
        got = out[:, :, :w].cpu().numpy()
        assert np.array_equal(got, ref), "call %d differs from ih_build" % call
        results.append(got)
    if h * w > 100:  # the two frames differ, so a stale result would show
        assert not np.array_equal(results[0], results[1])
    # and the first case against the oracle itself
    if shape == (480, 640):
        assert np.array_equal(results[1], oracle.integral_histogram(synth.blob_plane(h, w, seed * 10 + 1), bins))


def test_static_refuses_too_large(ihlib):
    img = torch.zeros((1080, 1920), dtype=torch.uint8, device=DEV)
    # a (200, 1080, 1920) view of 16 bytes: the call refuses before touching it
    out = torch.zeros(4, dtype=torch.int32, device=DEV).as_strided((200, 1080, 1920), (0, 0, 0))
    with pytest.raises(ihlib.IHError) as ei:
        ihlib.ih_build_counts_static(img, 200, 0, out)
    assert ei.value.status == ihlib.IH_ETOOBIG
    with pytest.raises(ihlib.IHError) as ei:
        ihlib.ih_build_counts_static(img, 16, 0, torch.empty((16, 1080, 1922), dtype=torch.int32, device=DEV))
    assert ei.value.status == ihlib.IH_EINVAL  # pitch not a multiple of 4
