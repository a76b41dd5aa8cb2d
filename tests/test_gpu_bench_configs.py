"""The bench's own workloads at full size, through the calls and layouts the
bench times, compared with the oracle.

* FMV step: one 1920 x 1080 RGB frame -> 7 feature channels (91 bins) in
  the record layout with the intensity channel's four int64 moment planes
  (the merged count + moment tiles kernel), then one ih_query call with
  100,000 rectangles and 4,096 Epanechnikov windows.  Whole count tensor
  and all four moment planes bit-exact against Algorithm 5 / Eq. 3.4; every
  rectangle by four corners of the (verified) tensor and 2,000 by
  enumeration; every window against the FP64 direct sum (Eq. 3.1).
* WAMI frame: one 8192 x 8192 blob plane, 32 bins, record layout, int64
  moment planes (77 GB on the device), one ih_query call with 1,000,000
  rectangles and 100,000 windows.  The whole count tensor and all four
  moment planes are compared band by band (each band's oracle tensor plus
  the running last row of the bands above it: Eq. 2.15 split at a row), so
  every cell is checked, the 64-bit offsets at the bottom-right included;
  every rectangle by enumeration and every window by direct summation,
  spread over the host's cores.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1711_01656_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
WTOL = 1e-5
NCPU = max(1, min(32, os.cpu_count() or 1))


def _assert_weighted(got, ref):
    got = np.asarray(got, dtype=np.float64)
    zero = ref == 0
    assert np.array_equal(got[zero], ref[zero]), "non-zero where the oracle is 0"
    rel = np.abs(got[~zero] - ref[~zero]) / np.abs(ref[~zero])
    assert rel.size == 0 or rel.max() <= WTOL, "max rel err %g" % rel.max()


def _split(fn, q, parts=NCPU):
    """fn over row chunks of q on host threads (the oracle's C calls release
    the GIL), results concatenated in order."""
    chunks = np.array_split(q, parts)
    with cf.ThreadPoolExecutor(max_workers=parts) as ex:
        return np.concatenate(list(ex.map(fn, chunks)), axis=0)


def _four_corners(t, rects):
    """Rectangle histograms from four corners of a b x h x w tensor t (int64,
    on the device): Eq. 2.16 with H(-1, .) = H(., -1) = 0."""
    P = torch.nn.functional.pad(t, (1, 0, 1, 0))
    r0, c0, r1, c1 = (rects[:, i].long() for i in range(4))
    return (P[:, r1 + 1, c1 + 1] - P[:, r0, c1 + 1] - P[:, r1 + 1, c0] + P[:, r0, c0]).T


def test_fmv_bench_step_full_size(ihlib):
    ih = ihlib
    rgb, rects, wins = bench.make_inputs(synth.config_seed(2))
    chans = synth.FMV_CHANNELS
    B, Bw = bench.total_bins(), 16
    h, w = rgb.shape[1:]
    c = ih.ih_create(0, flags=ih.IH_CFG_PROFILE)
    try:
        hdl, = ih.ih_build(c, ih.Frame(torch.from_numpy(rgb).to(DEV), chans, input=ih.IH_INPUT_RGB_FEATURES,
                                       weighted_channel=bench.WEIGHTED_CH, layout=ih.IH_LAYOUT_RECORD))
        d_r, d_w = torch.from_numpy(rects).to(DEV), torch.from_numpy(wins).to(DEV)
        r_out = torch.full((len(rects), B), -5, dtype=torch.int32, device=DEV)
        w_out = torch.full((len(wins), Bw), -5.0, dtype=torch.float32, device=DEV)
        ih.ih_query(c, hdl, d_r, r_out, d_w, w_out)
        full = torch.empty((B, h, w), dtype=torch.int32, device=DEV)
        ih.ih_export(c, hdl, full)
        ih.ih_sync(c)
        feats = oracle.features(rgb)
        ref = oracle.frame_integral_histogram(feats, chans, threads=NCPU)
        assert np.array_equal(full.cpu().numpy(), ref), "count tensor"
        # the moment planes of the intensity channel (w = c, r, c^2, r^2)
        plane = torch.empty((Bw, h, w), dtype=torch.int64, device=DEV)
        for p, wk in enumerate(oracle.MOMENT_WEIGHTS):
            ih.ih_export_moments(c, hdl, p, plane)
            ih.ih_sync(c)
            assert np.array_equal(plane.cpu().numpy(),
                                  oracle.weighted_integral_histogram(feats[bench.WEIGHTED_CH], Bw, wk,
                                                                     threads=NCPU)), "moment plane %d" % p
        del plane
        # every rectangle by four corners of the verified tensor, 2,000 by enumeration
        got = r_out.cpu().numpy()
        assert np.array_equal(got, _four_corners(full.long(), d_r).cpu().numpy())
        sub = np.random.Generator(np.random.PCG64(11)).choice(len(rects), 2000, replace=False)
        assert np.array_equal(got[sub], _split(lambda q: oracle.frame_rect_hist(feats, chans, q), rects[sub]))
        # every window against the FP64 direct sum
        _assert_weighted(w_out.cpu().numpy(),
                         _split(lambda q: oracle.weighted_hist(feats[bench.WEIGHTED_CH], Bw, q), wins))
        ih.ih_release(c, hdl)
    finally:
        ih.ih_destroy(c)
        torch.cuda.empty_cache()


def _band_moment(wk, ra, n_loc, m_loc):
    """The moment plane w of a band [ra, rb) spanning all columns, from the
    band's own oracle planes (rows counted from ra): columns are absolute
    already; r = ra + r_loc, so sum r = sum r_loc + ra N and
    sum r^2 = sum r_loc^2 + 2 ra sum r_loc + ra^2 N (Eq. 3.4, w polynomial)."""
    if wk in (oracle.W_COL, oracle.W_COL2):
        return m_loc[wk]
    if wk == oracle.W_ROW:
        return m_loc[oracle.W_ROW] + ra * n_loc
    return m_loc[oracle.W_ROW2] + 2 * ra * m_loc[oracle.W_ROW] + ra * ra * n_loc


def test_wami_bench_frame_record_full_size(ihlib):
    ih = ihlib
    img, rects, wins = bench.make_wami_inputs(synth.config_seed(3))
    H, W = img.shape
    B = bench.WAMI_BINS
    free, _ = torch.cuda.mem_get_info(DEV)
    assert free > 110e9, "the 8192 x 8192 frame needs about 110 GB free on the device"
    c = ih.ih_create(0, flags=ih.IH_CFG_PROFILE)
    try:
        pix = torch.from_numpy(img).to(DEV)[None]
        hdl, = ih.ih_build(c, ih.Frame(pix, [(B, 0)], weighted_channel=0, layout=ih.IH_LAYOUT_RECORD))
        d_r, d_w = torch.from_numpy(rects).to(DEV), torch.from_numpy(wins).to(DEV)
        r_out = torch.full((len(rects), B), -5, dtype=torch.int32, device=DEV)
        w_out = torch.full((len(wins), B), -5.0, dtype=torch.float32, device=DEV)
        ih.ih_query(c, hdl, d_r, r_out, d_w, w_out)
        ih.ih_sync(c)
        # every rectangle by enumeration, every window by direct summation
        assert np.array_equal(r_out.cpu().numpy(), _split(lambda q: oracle.rect_hist(img, B, q), rects))
        _assert_weighted(w_out.cpu().numpy(), _split(lambda q: oracle.weighted_hist(img, B, q), wins))
        del r_out, w_out
        # the whole count tensor and the four moment planes, band by band
        full = torch.empty((B, H, W), dtype=torch.int32, device=DEV)
        ih.ih_export(c, hdl, full)
        ih.ih_sync(c)
        band = 512
        carry = np.zeros((B, W), np.int64)
        n_bands = []
        for ra in range(0, H, band):
            rb = min(H, ra + band)
            loc = oracle.integral_histogram(img[ra:rb], B, threads=NCPU)
            exp = loc.astype(np.int64) + carry[:, None, :]
            assert np.array_equal(full[:, ra:rb, :].cpu().numpy().astype(np.int64), exp), "counts, rows %d.." % ra
            carry = exp[:, -1, :]
            n_bands.append(ra)
        del full
        plane = torch.empty((B, H, W), dtype=torch.int64, device=DEV)
        for p, wk in enumerate(oracle.MOMENT_WEIGHTS):
            ih.ih_export_moments(c, hdl, p, plane)
            ih.ih_sync(c)
            carry = np.zeros((B, W), np.int64)
            for ra in n_bands:
                rb = min(H, ra + band)
                part = img[ra:rb]
                n_loc = (oracle.integral_histogram(part, B, threads=NCPU).astype(np.int64)
                         if wk in (oracle.W_ROW, oracle.W_ROW2) else None)
                need = {wk} | ({oracle.W_ROW} if wk == oracle.W_ROW2 else set())
                m_loc = {k: oracle.weighted_integral_histogram(part, B, k, threads=NCPU) for k in need}
                exp = _band_moment(wk, ra, n_loc, m_loc) + carry[:, None, :]
                assert np.array_equal(plane[:, ra:rb, :].cpu().numpy(), exp), "moment plane %d, rows %d.." % (p, ra)
                carry = exp[:, -1, :]
        del plane
        ih.ih_release(c, hdl)
    finally:
        ih.ih_destroy(c)
        torch.cuda.empty_cache()
