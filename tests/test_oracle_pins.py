"""Pins of the CPU oracle to facts other than itself.

Each test checks one oracle routine against something the thesis or the
mathematics fixes: the hand-worked example (tests/golden), closed forms,
invariants, special cases that reduce to a library routine, and brute force
on tiny inputs.  A wrong sign, index, dropped term or transposed operand in
the oracle fails at least one of them (see test_oracle_mutations.py).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1711_01656_gb300 import synth


def _bins_by_edges(img, bins):
    """Uniform binning over [0,256) by searching the bin edges 256*b/bins:
    an independent route to Eq. 2.15's Q (searchsorted, not the formula)."""
    edges = np.array([Fraction(256 * b, bins) for b in range(1, bins)], dtype=object)
    flat = np.asarray(img, dtype=np.int64).ravel()
    idx = np.array([int(np.searchsorted(edges.astype(float), v, side="right")) for v in flat])
    return idx.reshape(np.shape(img))


def _prefix_by_enumeration(q, bins):
    """H(b, r, c) = #{(r', c') : r' <= r, c' <= c, q = b}, pure Python loops."""
    h, w = q.shape
    out = np.zeros((bins, h, w), dtype=np.int64)
    for r in range(h):
        for c in range(w):
            for rr in range(r + 1):
                for cc in range(c + 1):
                    b = q[rr, cc]
                    if 0 <= b < bins:
                        out[b, r, c] += 1
    return out


# ---------------------------------------------------------------- hand example

def test_hand_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_2x3.json")))
    img = np.array(g["image"], dtype=np.uint8)
    ih = oracle.integral_histogram(img, g["bins"])
    assert ih.tolist() == g["ih"]
    rh = oracle.rect_hist(img, g["bins"], [g["rect"]["box"]])
    assert rh.tolist() == [g["rect"]["hist"]]
    wd = g["weighted"]
    wh = oracle.weighted_hist(img, g["bins"], [wd["window"]])
    for k in range(g["bins"]):
        assert wh[0, k] == pytest.approx(wd["hist_num"][k] / wd["hist_den"], rel=1e-15)
    for r in range(2):
        for c in range(3):
            assert oracle.kernel_weight(wd["window"], r, c) == pytest.approx(wd["k_rows"][r][c], rel=1e-15)
    whn = oracle.weighted_hist(img, g["bins"], [wd["window"]], normalize=True)
    assert whn[0].tolist() == pytest.approx([157 / 314, 157 / 314], rel=1e-15)


# ---------------------------------------------------------------- binning

@pytest.mark.parametrize("bins", [1, 2, 3, 7, 9, 16, 32, 40, 91, 256])
def test_uniform_binning_matches_edges(bins):
    v = np.arange(256).reshape(16, 16)
    got = np.array([[oracle.bin_of(x, bins) for x in row] for row in v])
    assert (got == _bins_by_edges(v, bins)).all()
    # every bin of a uniform binning over [0,256) holds floor or ceil of 256/bins values
    counts = np.bincount(got.ravel(), minlength=bins)
    assert counts.min() >= 256 // bins and counts.max() <= -(-256 // bins)


def test_index_binning():
    assert [oracle.bin_of(v, 9, oracle.BIN_INDEX) for v in range(12)] == list(range(9)) + [-1] * 3


# ---------------------------------------------------------------- Algorithm 5

@pytest.mark.parametrize("h,w,bins,seed", [(1, 1, 1, 0), (1, 7, 3, 1), (6, 1, 4, 2), (5, 6, 2, 3),
                                           (7, 5, 16, 4), (4, 9, 40, 5)])
def test_alg5_equals_enumeration(h, w, bins, seed):
    img = synth.uniform_plane(h, w, seed)
    got = oracle.integral_histogram(img, bins)
    ref = _prefix_by_enumeration(_bins_by_edges(img, bins), bins)
    assert (got == ref).all()


@pytest.mark.parametrize("bins", list(range(1, 41)))
def test_alg5_equals_cumsum_of_onehot(bins):
    img = synth.uniform_plane(23, 31, 100 + bins)
    q = _bins_by_edges(img, bins)
    onehot = (q[None, :, :] == np.arange(bins)[:, None, None]).astype(np.int64)
    ref = np.cumsum(np.cumsum(onehot, axis=1), axis=2)
    assert (oracle.integral_histogram(img, bins) == ref).all()


@pytest.mark.parametrize("h,w,bins", [(17, 29, 16), (64, 48, 32), (9, 64, 9)])
def test_alg5_invariants(h, w, bins):
    img = synth.blob_plane(h, w, 7)
    H = oracle.integral_histogram(img, bins).astype(np.int64)
    # the full-image histogram sums to H*W
    assert H[:, -1, -1].sum() == h * w
    # every prefix holds (r+1)(c+1) pixels in total
    rr, cc = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    assert (H.sum(axis=0) == (rr + 1) * (cc + 1)).all()
    # monotone non-decreasing along rows and columns
    assert (np.diff(H, axis=1) >= 0).all() and (np.diff(H, axis=2) >= 0).all()
    # full-image histogram equals numpy's bincount of the bins
    assert (H[:, -1, -1] == np.bincount(_bins_by_edges(img, bins).ravel(), minlength=bins)).all()


@pytest.mark.parametrize("v", [0, 1, 127, 128, 200, 255])
def test_alg5_constant_image(v):
    h, w, bins = 13, 11, 16
    H = oracle.integral_histogram(np.full((h, w), v, np.uint8), bins)
    b = v * bins // 256
    rr, cc = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    assert (H[b] == (rr + 1) * (cc + 1)).all()
    assert (np.delete(H, b, axis=0) == 0).all()


def test_alg5_bin_subsets_are_slices():
    img = synth.uniform_plane(20, 24, 11)
    full = oracle.integral_histogram(img, 16)
    # a 16-bin build is the 4-bin build of (v >> 2) refined: bins 4k..4k+3 sum to 4-bin bin k
    coarse = oracle.integral_histogram(img, 4)
    assert (full.reshape(4, 4, 20, 24).sum(axis=1) == coarse).all()


def test_alg5_index_mode_skips_out_of_range():
    img = np.array([[0, 1, 9, 2], [3, 200, 8, 8]], np.uint8)
    H = oracle.integral_histogram(img, 9, oracle.BIN_INDEX)
    assert H[:, -1, -1].sum() == 6  # 9 and 200 are in no bin
    assert H[8, -1, -1] == 2 and H[0, -1, -1] == 1


def test_alg5_threads_agree():
    img = synth.uniform_plane(40, 50, 3)
    assert (oracle.integral_histogram(img, 16, threads=1) ==
            oracle.integral_histogram(img, 16, threads=5)).all()


# ---------------------------------------------------------------- Eq. 2.16

def test_four_corner_identity_all_rects():
    h, w, bins = 10, 12, 5
    img = synth.uniform_plane(h, w, 21)
    H = np.pad(oracle.integral_histogram(img, bins).astype(np.int64), ((0, 0), (1, 0), (1, 0)))
    rects = [(r0, c0, r1, c1) for r0 in range(h) for r1 in range(r0, h)
             for c0 in range(w) for c1 in range(c0, w)]
    rects = np.array(rects, np.int32)
    brute = oracle.rect_hist(img, bins, rects)
    r0, c0, r1, c1 = (rects[:, i] for i in range(4))
    four = (H[:, r1 + 1, c1 + 1] - H[:, r0, c1 + 1] - H[:, r1 + 1, c0] + H[:, r0, c0]).T
    assert (brute == four).all()


def test_rect_hist_is_bincount_of_slice():
    img = synth.blob_plane(40, 37, 5)
    rects = synth.rects_uniform_corners(40, 37, 300, 9)
    got = oracle.rect_hist(img, 16, rects)
    q = _bins_by_edges(img, 16)
    for (r0, c0, r1, c1), row in zip(rects, got):
        assert (row == np.bincount(q[r0:r1 + 1, c0:c1 + 1].ravel(), minlength=16)).all()
        assert row.sum() == (r1 - r0 + 1) * (c1 - c0 + 1)


def test_rect_hist_invalid_rows():
    img = synth.uniform_plane(8, 8, 1)
    bad = [[-1, 0, 3, 3], [0, 0, 8, 3], [4, 0, 3, 3], [0, 5, 3, 4], [0, 0, 3, 8]]
    out = oracle.rect_hist(img, 4, bad + [[0, 0, 7, 7]])
    assert (out[:5] == -1).all() and out[5].sum() == 64


# ---------------------------------------------------------------- Eq. 3.1

def _K_closed_form(w, h):
    """sum over a w x h window of k(r,c) = 1 - d_c^2/(2w^2) - d_r^2/(2h^2),
    d = 2*offset - (span-1): sum of d^2 over an axis of length n is
    (n-1)n(n+1)/3 (sum of squares of n values spaced by 2, symmetric)."""
    sx = Fraction((w - 1) * w * (w + 1), 3)
    sy = Fraction((h - 1) * h * (h + 1), 3)
    return w * h - h * sx / (2 * w * w) - w * sy / (2 * h * h)


@pytest.mark.parametrize("wh", [(1, 1), (1, 5), (4, 1), (3, 2), (8, 8), (33, 17), (64, 100)])
def test_weighted_constant_image_closed_form(wh):
    w, h = wh
    img = np.full((h + 3, w + 2), 77, np.uint8)
    win = [[1, 2, h, w + 1]]
    out = oracle.weighted_hist(img, 16, win)
    K = float(_K_closed_form(w, h))
    assert out[0, 77 * 16 // 256] == pytest.approx(K, rel=1e-13)
    assert np.count_nonzero(out[0]) == 1


def test_weighted_sum_over_bins_is_K_and_normalized_sums_to_one():
    img = synth.blob_plane(60, 70, 3)
    wins = synth.rects_side_range(60, 70, 50, 1, 40, 4)
    out = oracle.weighted_hist(img, 16, wins)
    outn = oracle.weighted_hist(img, 16, wins, normalize=True)
    for (r0, c0, r1, c1), row, rown in zip(wins, out, outn):
        assert row.sum() == pytest.approx(float(_K_closed_form(c1 - c0 + 1, r1 - r0 + 1)), rel=1e-12)
        assert rown.sum() == pytest.approx(1.0, rel=1e-12)


def test_weighted_translation_invariance():
    """The weights depend on the position relative to the window only (Sec. 3.1.3)."""
    patch = synth.uniform_plane(9, 14, 8)
    a = synth.uniform_plane(30, 40, 1)
    b = synth.uniform_plane(30, 40, 2)
    a[3:12, 5:19] = patch
    b[20:29, 22:36] = patch
    oa = oracle.weighted_hist(a, 8, [[3, 5, 11, 18]])
    ob = oracle.weighted_hist(b, 8, [[20, 22, 28, 35]])
    assert np.array_equal(oa, ob)


def test_weighted_mirror_symmetry():
    img = synth.uniform_plane(11, 16, 5)
    win = [[0, 0, 10, 15]]
    base = oracle.weighted_hist(img, 8, win)
    assert oracle.weighted_hist(img[:, ::-1].copy(), 8, win) == pytest.approx(base, rel=1e-14)
    assert oracle.weighted_hist(img[::-1, :].copy(), 8, win) == pytest.approx(base, rel=1e-14)


def test_weighted_single_pixel_values():
    """One pixel of bin 1 in a bin-0 background isolates k at that pixel."""
    h, w = 7, 9  # odd: the centre pixel has weight exactly 1
    for (r, c) in [(3, 4), (0, 0), (6, 8), (2, 7)]:
        img = np.zeros((h, w), np.uint8)
        img[r, c] = 255
        out = oracle.weighted_hist(img, 2, [[0, 0, h - 1, w - 1]])
        k = 1 - Fraction((2 * c - (w - 1)) ** 2, 2 * w * w) - Fraction((2 * r - (h - 1)) ** 2, 2 * h * h)
        assert out[0, 1] == pytest.approx(float(k), rel=1e-15)
        if (r, c) == (3, 4):
            assert out[0, 1] == 1.0
        assert out[0, 1] > 0


def test_weighted_equals_exact_rational_sum():
    img = synth.uniform_plane(12, 10, 6)
    win = (2, 1, 10, 8)
    r0, c0, r1, c1 = win
    w, h = c1 - c0 + 1, r1 - r0 + 1
    exact = [Fraction(0)] * 4
    for r in range(r0, r1 + 1):
        for c in range(c0, c1 + 1):
            k = 1 - Fraction((2 * c - c0 - c1) ** 2, 2 * w * w) - Fraction((2 * r - r0 - r1) ** 2, 2 * h * h)
            exact[int(img[r, c]) >> 6] += k
    out = oracle.weighted_hist(img, 4, [win])
    assert out[0].tolist() == pytest.approx([float(x) for x in exact], rel=1e-14)


# ---------------------------------------------------------------- Eq. 3.3 Manhattan kernel, Eq. 3.2 wedding cake

def test_manhattan_and_wedding_hand_example(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "hand_2x3.json")))
    img = np.array(g["image"], np.uint8)
    m = g["manhattan"]
    for r in range(2):
        for c in range(3):
            assert oracle.manhattan_weight(m["window"], r, c) == m["k_rows"][r][c]
    assert oracle.weighted_hist(img, 2, [m["window"]], kernel=oracle.K_MANHATTAN)[0].tolist() == m["hist"]
    assert oracle.weighted_hist(img, 2, [m["window"]], kernel=oracle.K_MANHATTAN, normalize=True)[0].tolist() == \
        [x / m["K"] for x in m["hist"]]
    wc = g["wedding_cake"]
    assert oracle.weighted_hist(img, 2, [wc["window"]], kernel=oracle.K_WEDDING_CAKE,
                                layers=wc["layers"])[0].tolist() == wc["hist"]


def _manhattan_K(w, h):
    """sum over a w x h window of (h + w) - |2r - (r0+r1)| - |2c - (c0+c1)|:
    the |2i - (n-1)| over i = 0..n-1 sum to floor(n^2/2)."""
    return (h + w) * h * w - w * (h * h // 2) - h * (w * w // 2)


@pytest.mark.parametrize("wh", [(1, 1), (1, 5), (4, 1), (3, 2), (8, 8), (33, 17), (64, 100)])
def test_manhattan_constant_image_closed_form(wh):
    w, h = wh
    img = np.full((h + 3, w + 2), 200, np.uint8)
    out = oracle.weighted_hist(img, 8, [[1, 2, h, w + 1]], kernel=oracle.K_MANHATTAN)
    assert out[0, 200 * 8 // 256] == _manhattan_K(w, h)
    assert np.count_nonzero(out[0]) == 1


def test_manhattan_equals_quadrant_decomposition():
    """Sec. 3.1.3 / Fig. 3.4: split the window at its centre into four
    quadrants; inside each, the weight is linear in (r, c), so each quadrant's
    weighted histogram is a combination of plain, r-weighted and c-weighted
    region sums -- here taken from numpy cumulative sums, not from the
    oracle."""
    img = synth.blob_plane(50, 61, 12)
    B = 16
    q = (img.astype(np.int64) * B) >> 8
    onehot = (q[None] == np.arange(B)[:, None, None]).astype(np.int64)
    rr, cc = np.meshgrid(np.arange(50), np.arange(61), indexing="ij")
    planes = {k: np.cumsum(np.cumsum(onehot * wgt[None], axis=1), axis=2)
              for k, wgt in (("n", np.ones_like(rr)), ("r", rr), ("c", cc))}

    def box(plane, r0, c0, r1, c1):
        if r1 < r0 or c1 < c0:
            return np.zeros(B, np.int64)
        P = planes[plane]
        s = P[:, r1, c1].copy()
        if r0 > 0:
            s -= P[:, r0 - 1, c1]
        if c0 > 0:
            s -= P[:, r1, c0 - 1]
        if r0 > 0 and c0 > 0:
            s += P[:, r0 - 1, c0 - 1]
        return s

    wins = synth.rects_side_range(50, 61, 60, 1, 40, 13)
    ref = oracle.weighted_hist(img, B, wins, kernel=oracle.K_MANHATTAN)
    for (r0, c0, r1, c1), row in zip(wins, ref):
        h, w, sr, sc = r1 - r0 + 1, c1 - c0 + 1, r0 + r1, c0 + c1
        rs, cs = sr // 2, sc // 2
        tot = np.zeros(B, np.int64)
        for (a, b, er) in ((r0, rs, -1), (rs + 1, r1, 1)):       # rows: |2r - sr| = er * (2r - sr)
            for (c, d, ec) in ((c0, cs, -1), (cs + 1, c1, 1)):
                n, sr_, sc_ = box("n", a, c, b, d), box("r", a, c, b, d), box("c", a, c, b, d)
                tot += (h + w + er * sr + ec * sc) * n - 2 * er * sr_ - 2 * ec * sc_
        assert np.array_equal(row, tot.astype(np.float64))


def test_manhattan_translation_and_mirror():
    patch = synth.uniform_plane(9, 14, 8)
    a = synth.uniform_plane(30, 40, 1)
    b = synth.uniform_plane(30, 40, 2)
    a[3:12, 5:19] = patch
    b[20:29, 22:36] = patch
    oa = oracle.weighted_hist(a, 8, [[3, 5, 11, 18]], kernel=oracle.K_MANHATTAN)
    ob = oracle.weighted_hist(b, 8, [[20, 22, 28, 35]], kernel=oracle.K_MANHATTAN)
    assert np.array_equal(oa, ob)
    img = synth.uniform_plane(11, 16, 5)
    base = oracle.weighted_hist(img, 8, [[0, 0, 10, 15]], kernel=oracle.K_MANHATTAN)
    assert np.array_equal(oracle.weighted_hist(img[:, ::-1].copy(), 8, [[0, 0, 10, 15]], kernel=oracle.K_MANHATTAN),
                          base)


@pytest.mark.parametrize("layers", [1, 2, 3, 5, 8])
def test_wedding_cake_is_sum_of_nested_windows(layers):
    """Eq. 3.2 telescopes: sum_j w_j (H(R_j) - H(R_{j+1})) with equal steps
    w_j - w_{j-1} = (h+w)/L is (h+w)/L times the sum of the nested windows'
    plain histograms (np.bincount of each sub-rectangle)."""
    img = synth.blob_plane(40, 52, 21)
    B = 8
    wins = synth.rects_side_range(40, 52, 40, 1, 40, 22)
    ref = oracle.weighted_hist(img, B, wins, kernel=oracle.K_WEDDING_CAKE, layers=layers)
    for (r0, c0, r1, c1), row in zip(wins, ref):
        h, w = r1 - r0 + 1, c1 - c0 + 1
        tot = np.zeros(B, np.int64)
        for j in range(layers):
            dr, dc = j * h // (2 * layers), j * w // (2 * layers)
            sub = img[r0 + dr: r1 - dr + 1, c0 + dc: c1 - dc + 1].astype(np.int64)
            tot += np.bincount(((sub * B) >> 8).ravel(), minlength=B)
        assert row == pytest.approx(tot * (h + w) / layers, rel=1e-14)


def test_wedding_cake_one_layer_is_plain_histogram():
    img = synth.uniform_plane(20, 30, 4)
    wins = synth.rects_side_range(20, 30, 30, 1, 20, 5)
    plain = oracle.rect_hist(img, 8, wins).astype(np.float64)
    wc = oracle.weighted_hist(img, 8, wins, kernel=oracle.K_WEDDING_CAKE, layers=1)
    sides = (wins[:, 2] - wins[:, 0] + 1) + (wins[:, 3] - wins[:, 1] + 1)
    assert np.array_equal(wc, plain * sides[:, None])


def test_wedding_cake_rings_are_a_staircase():
    """Sec. 3.1.2 / Fig. 3.3: nested windows around the centre; each pixel's
    weight is (h+w)/L times the number of nested windows holding it, so the
    weights never decrease towards the centre and reach h+w there; with a
    few layers the rings approximate the Manhattan pyramid better than one
    flat window does (normalised histograms' L1 distance)."""
    win = [3, 4, 20, 30]
    r0, c0, r1, c1 = win
    h, w = r1 - r0 + 1, c1 - c0 + 1
    for L in (1, 3, 6):
        wt = np.array([[oracle.wedding_weight(win, L, r, c) for c in range(c0, c1 + 1)] for r in range(r0, r1 + 1)])
        nest = np.zeros_like(wt)
        for j in range(L):
            dr, dc = j * h // (2 * L), j * w // (2 * L)
            nest[dr: h - dr, dc: w - dc] += 1
        assert np.array_equal(wt, nest * (h + w) / L)
        mid_r, mid_c = h // 2, w // 2
        assert np.all(np.diff(wt[mid_r, : mid_c + 1]) >= 0) and np.all(np.diff(wt[: mid_r + 1, mid_c]) >= 0)
        assert wt[mid_r, mid_c] == h + w
    img = synth.blob_plane(64, 64, 30)
    wins = np.array([[0, 0, 63, 63], [5, 9, 60, 50], [10, 3, 41, 62]], np.int32)
    man = oracle.weighted_hist(img, 16, wins, kernel=oracle.K_MANHATTAN, normalize=True)
    err = {L: np.abs(oracle.weighted_hist(img, 16, wins, kernel=oracle.K_WEDDING_CAKE, layers=L, normalize=True)
                     - man).sum() for L in (1, 4)}
    assert err[4] < err[1]


# ---------------------------------------------------------------- Eq. 2.22 sliding-window matching

def _box_hist_numpy(img, bins, wh, ww):
    """Every placement's window histogram from 2-D cumulative sums of the
    one-hot (numpy, independent of the oracle): [bins, h-wh+1, w-ww+1]."""
    q = (img.astype(np.int64) * bins) >> 8
    onehot = (q[None] == np.arange(bins)[:, None, None]).astype(np.int64)
    P = np.zeros((bins, img.shape[0] + 1, img.shape[1] + 1), np.int64)
    P[:, 1:, 1:] = onehot.cumsum(1).cumsum(2)
    return P[:, wh:, ww:] - P[:, :-wh, ww:] - P[:, wh:, :-ww] + P[:, :-wh, :-ww]


@pytest.mark.parametrize("wh,ww", [(1, 1), (3, 5), (8, 8), (12, 4)])
def test_match_window_equals_cumsum_boxes(wh, ww):
    img = synth.blob_plane(30, 41, 50)
    B = 8
    target = np.array([5, 0, 3, 9, 1, 0, 2, 7], np.int32)
    search = (2, 3, 30 - wh, 41 - ww)
    got = oracle.match_window(img, B, target, wh, ww, search)
    boxes = _box_hist_numpy(img, B, wh, ww)[:, search[0]:search[2] + 1, search[1]:search[3] + 1]
    assert np.array_equal(got, np.abs(boxes - target[:, None, None]).sum(0))


def test_match_window_zero_at_own_placement_and_constant_image():
    img = synth.uniform_plane(25, 30, 51)
    B = 16
    r, c, wh, ww = 7, 11, 6, 9
    target = np.bincount((img[r:r + wh, c:c + ww].astype(np.int64) * B >> 8).ravel(), minlength=B).astype(np.int32)
    got = oracle.match_window(img, B, target, wh, ww, (0, 0, 25 - wh, 30 - ww))
    assert got[r, c] == 0 and (got >= 0).all()
    const = np.full((20, 20), 90, np.uint8)
    t = np.arange(B, dtype=np.int32)
    d = oracle.match_window(const, B, t, 4, 5, (0, 0, 16, 15))
    k = 90 * B >> 8
    assert (d == t.sum() - t[k] + abs(20 - t[k])).all()
    with pytest.raises(ValueError):
        oracle.match_window(const, B, t, 4, 5, (0, 0, 17, 15))


# ---------------------------------------------------------------- Algorithm 4 spatio-temporal median

def _median_by_counting(frames, bins, m, n):
    """Lower median bin per pixel from per-bin counts and their running sum
    (the histogram route), not by sorting."""
    nf, h, w = frames.shape
    q = (frames.astype(np.int64) * bins) >> 8
    out = np.empty((h, w), np.int32)
    for r in range(h):
        for c in range(w):
            box = q[:, max(0, r - m // 2): r + (m + 1) // 2, max(0, c - n // 2): c + (n + 1) // 2]
            cnt = np.bincount(box.ravel(), minlength=bins)
            out[r, c] = int(np.searchsorted(np.cumsum(cnt), (box.size + 1) // 2))
    return out


@pytest.mark.parametrize("nf,m,n", [(1, 1, 1), (1, 3, 3), (3, 3, 5), (5, 4, 2), (4, 6, 6)])
def test_local_median_equals_counting(nf, m, n):
    frames = np.stack([synth.blob_plane(17, 23, 60 + k) for k in range(nf)])
    assert np.array_equal(oracle.local_median(frames, 16, m, n), _median_by_counting(frames, 16, m, n))


def test_local_median_special_cases():
    img = synth.uniform_plane(12, 15, 61)
    assert np.array_equal(oracle.local_median(img, 8, 1, 1), (img.astype(np.int32) * 8) >> 8)
    const = np.full((3, 10, 10), 200, np.uint8)
    assert (oracle.local_median(const, 4, 5, 3) == 200 * 4 // 256).all()
    # nf identical frames: the 3-D median is the 2-D median of one frame
    f = synth.blob_plane(14, 16, 62)
    assert np.array_equal(oracle.local_median(np.stack([f] * 4), 16, 3, 5), oracle.local_median(f, 16, 3, 5))
    # one salt pixel in a flat 3 x 3 neighbourhood does not move the median
    g = np.full((9, 9), 10, np.uint8)
    g[4, 4] = 250
    assert (oracle.local_median(g, 16, 3, 3) == 0).all()


# ---------------------------------------------------------------- Algorithm 2 PHoG, Eq. 2.23-2.24

def test_isqrt_exhaustive_against_math_isqrt():
    import math
    vals = sorted({256 * (gx * gx + gy * gy) for gx in range(256) for gy in range(256)})
    for n in vals[::7] + vals[-50:] + [0, 1, 2, 3, 4, 15, 16, 17]:
        assert oracle.isqrt(n) == math.isqrt(n)


# Canny's detector (Algorithm 2 step 1; J. Canny 1986), pinned stage by stage
# against library routines and independent formulations, and end to end on
# images whose edges are known by construction.

def _canny_case(k):
    if k == 0:
        return synth.blob_plane(41, 57, 90)
    if k == 1:
        return synth.uniform_plane(33, 29, 91)
    g = synth.blob_plane(48, 64, 92)
    g[10:30, 20:40] = 230  # a bright block: long straight edges and corners
    return g


@pytest.mark.parametrize("k", [0, 1, 2])
def test_canny_smoothing_is_binomial_convolution(k):
    from scipy import ndimage
    g = _canny_case(k)
    _, S, _, _ = oracle.canny(g, 5, 20)
    b = np.array([1, 4, 6, 4, 1], np.int64)
    ref = ndimage.convolve(g.astype(np.int64), np.outer(b, b), mode="nearest")
    assert np.array_equal(S, ref)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_canny_gradient_of_the_smoothed_image(k):
    g = _canny_case(k)
    _, S, M, _ = oracle.canny(g, 5, 20)
    p = np.pad(S.astype(np.int64), 1, mode="edge")
    gx = p[1:-1, 2:] - p[1:-1, :-2]
    gy = p[2:, 1:-1] - p[:-2, 1:-1]
    assert np.array_equal(M, gx * gx + gy * gy)


def _nms_by_angle(S):
    """Non-maximum suppression by the gradient angle in degrees (numpy
    arctan2), an independent formulation of the oracle's exact sector test."""
    h, w = S.shape
    p = np.pad(S.astype(np.int64), 1, mode="edge")
    gx = p[1:-1, 2:] - p[1:-1, :-2]
    gy = p[2:, 1:-1] - p[:-2, 1:-1]
    m = gx * gx + gy * gy
    ang = np.degrees(np.arctan2(gy, gx)) % 180.0
    mp = np.pad(m, 1)  # neighbours outside the window count as 0
    keep = np.zeros((h, w), bool)
    for r in range(h):
        for c in range(w):
            a = ang[r, c]
            if a < 22.5 or a >= 157.5:
                lo_, hi_ = (r, c - 1), (r, c + 1)
            elif a < 67.5:
                lo_, hi_ = (r - 1, c - 1), (r + 1, c + 1)
            elif a < 112.5:
                lo_, hi_ = (r - 1, c), (r + 1, c)
            else:
                lo_, hi_ = (r + 1, c - 1), (r - 1, c + 1)
            v = m[r, c]
            keep[r, c] = v > mp[lo_[0] + 1, lo_[1] + 1] and v >= mp[hi_[0] + 1, hi_[1] + 1]
    return keep, m


@pytest.mark.parametrize("k", [0, 1, 2])
def test_canny_suppression_and_thresholds_by_angle(k):
    g = _canny_case(k)
    lo, hi = 6, 24
    _, S, _, cls = oracle.canny(g, lo, hi)
    keep, m = _nms_by_angle(S)
    ref = np.where(keep & (m >= (256 * hi) ** 2), 2, np.where(keep & (m >= (256 * lo) ** 2), 1, 0))
    assert np.array_equal(cls, ref)
    assert (cls == 1).any() and (cls == 2).any()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_canny_hysteresis_is_8_connected_components(k):
    """Edge pixels = survivors in an 8-connected component of survivors that
    holds a strong one (scipy.ndimage.label)."""
    from scipy import ndimage
    g = _canny_case(k)
    edges, _, _, cls = oracle.canny(g, 6, 24)
    lab, _ = ndimage.label(cls > 0, structure=np.ones((3, 3), int))
    strong = np.unique(lab[cls == 2])
    ref = np.isin(lab, strong[strong > 0]) & (cls > 0)
    assert np.array_equal(edges.astype(bool), ref)
    assert edges.sum() < (cls > 0).sum()  # some weak runs are dropped


def test_canny_step_edges_are_one_pixel_wide():
    v = np.zeros((12, 14), np.uint8)
    v[:, 6:] = 255
    e, _, _, _ = oracle.canny(v, 20, 60)
    ref = np.zeros_like(e)
    ref[:, 5] = 1  # the two-pixel plateau of |G| at columns 5 and 6 keeps column 5
    assert np.array_equal(e, ref)
    e, _, _, _ = oracle.canny(np.ascontiguousarray(v.T), 20, 60)
    assert np.array_equal(e, np.ascontiguousarray(ref.T))
    # a 45-degree step: the line stays on the two anti-diagonals next to it
    rr, cc = np.mgrid[0:16, 0:16]
    d = np.where(rr + cc >= 15, 255, 0).astype(np.uint8)
    e, _, _, _ = oracle.canny(d, 20, 60)
    assert e.sum() > 0 and set(np.unique((rr + cc)[e == 1])) == {14, 15}
    for r in range(1, 15):  # every interior row: both pixels, one on each anti-diagonal
        assert list(np.nonzero(e[r])[0]) == [14 - r, 15 - r]


def test_canny_hysteresis_keeps_connected_weak_runs():
    """A vertical step whose contrast falls from 200 to 40 down the rows:
    strong above, weak below, one connected line -> all rows are edges; an
    isolated weak run beside it is dropped; with a high threshold above every
    magnitude nothing is kept."""
    g = np.zeros((21, 20), np.uint8)
    for r in range(21):
        g[r, 8:] = 200 - 8 * r
    e, _, _, cls = oracle.canny(g, 10, 60)
    assert (cls[:, 8] == 2).sum() >= 5 and (cls[:, 8] == 1).sum() >= 5
    ref = np.zeros_like(e)
    ref[:, 8] = 1
    assert np.array_equal(e, ref)
    assert ((cls == 1) & (ref == 0)).any()  # the isolated weak run exists but is not an edge
    e, _, _, cls = oracle.canny(g, 10, 130)
    assert (cls == 1).sum() > 0 and (cls == 2).sum() == 0 and e.sum() == 0


def test_phog_planes_follow_the_stencil():
    """Algorithm 2 steps 2-3 on the Canny edge pixels of step 1."""
    import math
    g = synth.blob_plane(23, 31, 70)
    lo, hi = 3, 9
    bins, wt = oracle.phog_planes(g, lo, hi)
    edges, _, _, _ = oracle.canny(g, lo, hi)
    p = np.pad(g.astype(np.int64), 1, mode="edge")
    gx = p[1:-1, 2:] - p[1:-1, :-2]
    gy = p[2:, 1:-1] - p[:-2, 1:-1]
    for r in range(23):
        for c in range(31):
            m = math.isqrt(256 * int(gx[r, c] ** 2 + gy[r, c] ** 2))
            if edges[r, c]:
                assert wt[r, c] == m and bins[r, c] == oracle.orientation_bin(int(gx[r, c]), int(gy[r, c]))
            else:
                assert wt[r, c] == 0 and bins[r, c] == 255
    assert (bins < 9).any() and (bins == 255).any()


def test_phog_ih_equals_cumsum():
    g = synth.blob_plane(30, 37, 71)
    bins, wt = oracle.phog_planes(g, 2, 6)
    onehot = (bins[None] == np.arange(9)[:, None, None]) * wt[None].astype(np.int64)
    assert np.array_equal(oracle.phog_ih(bins, wt), onehot.cumsum(1).cumsum(2))


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_phog_descriptor_cells(L):
    g = synth.blob_plane(70, 90, 72)
    bins, wt = oracle.phog_planes(g, 2, 8)
    r0, c0, wh, ww = 6, 9, 48, 64
    d = oracle.phog_descriptor(bins, wt, L, r0, c0, wh, ww)
    assert d.shape == (9 * sum(4 ** l for l in range(L + 1)),)
    k = 0
    for l in range(L + 1):
        s_ = 2 ** l
        ch, cw = wh // s_, ww // s_
        lev = d[k: k + 9 * s_ * s_].reshape(s_, s_, 9)
        for i in range(s_):
            for j in range(s_):
                cb = bins[r0 + i * ch: r0 + (i + 1) * ch, c0 + j * cw: c0 + (j + 1) * cw]
                cwt = wt[r0 + i * ch: r0 + (i + 1) * ch, c0 + j * cw: c0 + (j + 1) * cw]
                assert np.array_equal(lev[i, j], [int(cwt[cb == q].sum()) for q in range(9)])
        # 48 and 64 divide by 2^l up to l = 3: every level covers the window
        assert np.array_equal(lev.sum((0, 1)), d[:9])
        k += 9 * s_ * s_


def test_pyramid_match_kernel_forms_agree():
    """Eq. 2.24: I^L + sum_{l<L} (I^l - I^{l+1}) / 2^(L-l) equals
    I^0 / 2^L + sum_{l>=1} I^l / 2^(L-l+1); the oracle computes the second
    form, numpy the first; kappa(X, X) is X's total weight."""
    g = synth.blob_plane(80, 80, 73)
    bins, wt = oracle.phog_planes(g, 2, 8)
    L = 3
    x = oracle.phog_descriptor(bins, wt, L, 4, 4, 64, 64)
    y = oracle.phog_descriptor(bins, wt, L, 10, 7, 64, 64)
    I, k = [], 0
    for l in range(L + 1):
        n = 9 * 4 ** l
        I.append(float(np.minimum(x[k:k + n], y[k:k + n]).sum()))
        k += n
    first = I[L] + sum((I[l] - I[l + 1]) / 2 ** (L - l) for l in range(L))
    assert oracle.pyramid_match(x, y, L) == pytest.approx(first, rel=1e-13)
    assert oracle.pyramid_match(x, x, L) == pytest.approx(float(x[:9].sum()), rel=1e-13)
    assert oracle.pyramid_match(x, np.zeros_like(x), L) == 0.0


# ---------------------------------------------------------------- Eq. 3.4 moment planes

@pytest.mark.parametrize("weight", [oracle.W_ONE] + list(oracle.MOMENT_WEIGHTS))
def test_weighted_ih_equals_cumsum(weight):
    h, w, bins = 19, 23, 6
    img = synth.uniform_plane(h, w, 40 + weight)
    q = _bins_by_edges(img, bins)
    rr, cc = np.meshgrid(np.arange(h, dtype=np.int64), np.arange(w, dtype=np.int64), indexing="ij")
    wt = {oracle.W_ONE: np.ones_like(rr), oracle.W_COL: cc, oracle.W_ROW: rr,
          oracle.W_COL2: cc * cc, oracle.W_ROW2: rr * rr}[weight]
    f = (q[None] == np.arange(bins)[:, None, None]) * wt[None]
    ref = np.cumsum(np.cumsum(f, axis=1), axis=2)
    assert (oracle.weighted_integral_histogram(img, bins, weight) == ref).all()


def test_weighted_ih_small_enumeration():
    img = synth.uniform_plane(4, 5, 77)
    q = _bins_by_edges(img, 3)
    got = oracle.weighted_integral_histogram(img, 3, oracle.W_COL2)
    for b in range(3):
        for r in range(4):
            for c in range(5):
                s = sum(cc * cc for rr in range(r + 1) for cc in range(c + 1) if q[rr, cc] == b)
                assert got[b, r, c] == s


# ---------------------------------------------------------------- features

def test_intensity_is_floor_mean():
    rgb = synth.blob_rgb(21, 33, 5)
    f = oracle.features(rgb)
    assert (f[:3] == rgb).all()
    assert (f[3] == rgb.astype(np.int64).sum(0) // 3).all()
    # special cases
    x = np.array([[[0, 255, 1, 2]], [[0, 255, 1, 2]], [[0, 255, 0, 1]]], np.uint8)
    assert oracle.features(x)[3].tolist() == [[0, 255, 0, 1]]


# (gx, gy) -> bin; angles: atan(84/100) = 40.03, atan(83/100) = 39.69,
# atan(36/100) = 19.80, atan(37/100) = 20.30 degrees; bins are 20 degrees wide
KNOWN_ORIENTATIONS = [((1, 0), 0), ((0, 1), 4), ((1, 1), 2), ((-1, 1), 6), ((-1, 0), 0), ((0, -1), 4),
                      ((0, 0), 0), ((-1, -1), 2), ((1, -1), 6), ((255, 1), 0), ((-255, 1), 8),
                      ((1, 255), 4), ((100, 84), 2), ((100, 83), 1), ((100, 36), 0), ((100, 37), 1)]


@pytest.mark.parametrize("g,b", KNOWN_ORIENTATIONS)
def test_orientation_known(g, b):
    assert oracle.orientation_bin(*g) == b


def _orientation_exact_table():
    """Bins of all 511^2 integer gradients by exact integer half-plane tests:
    theta >= 20j deg  <=>  cos(20j) gy - sin(20j) gx >= 0 for the folded
    vector.  The unit vectors are scaled by 2^52 and rounded from 40-digit
    values, so the integer cross products carry an error below 2^8 while the
    true ones, never zero (tan 20j deg is irrational), exceed 2^30."""
    import mpmath
    mpmath.mp.dps = 40
    U = [(int(mpmath.nint(mpmath.cos(mpmath.pi * j / 9) * 2 ** 52)),
          int(mpmath.nint(mpmath.sin(mpmath.pi * j / 9) * 2 ** 52))) for j in range(1, 9)]
    gx, gy = np.meshgrid(np.arange(-255, 256, dtype=np.int64), np.arange(-255, 256, dtype=np.int64),
                         indexing="ij")
    flip = (gy < 0) | ((gy == 0) & (gx < 0))
    fx, fy = np.where(flip, -gx, gx), np.where(flip, -gy, gy)
    b = np.zeros_like(fx)
    for ux, uy in U:
        cross = ux * fy - uy * fx
        assert (np.abs(cross[(fx != 0) | (fy != 0)]) > 2 ** 30).all()
        b += (cross >= 0)
    b[(fx == 0) & (fy == 0)] = 0
    return gx, gy, b


def test_orientation_exhaustive_vs_exact_integer_test():
    gx, gy, b = _orientation_exact_table()
    got = np.array([oracle.orientation_bin(int(x), int(y)) for x, y in zip(gx.ravel(), gy.ravel())])
    assert (got == b.ravel()).all()


def test_orientation_margin_to_bin_boundaries():
    """No integer gradient in [-255,255]^2 lies within 1e-5 rad of a bin
    boundary, so an FP64 atan2 decides every bin without ambiguity."""
    gx, gy = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256), indexing="ij")
    flip = (gy < 0) | ((gy == 0) & (gx < 0))
    fx, fy = np.where(flip, -gx, gx), np.where(flip, -gy, gy)
    nz = (fx != 0) | (fy != 0)
    th = np.arctan2(fy[nz], fx[nz])
    step = math.pi / 9
    frac = th / step - np.floor(th / step)
    gap = np.minimum(frac, 1 - frac) * step
    gap = gap[th > 1e-12]  # theta = 0 exactly (gy == 0) sits on bin 0's lower edge by definition
    assert gap.min() > 1e-5


def test_hog_stencil_replicated_borders():
    rgb = synth.blob_rgb(13, 17, 9)
    f = oracle.features(rgb)
    I = f[3].astype(np.int64)
    for li, s in enumerate((1, 2, 4)):
        P = np.pad(I, s, mode="edge")
        gx = P[s:-s, 2 * s:] - P[s:-s, :-2 * s]
        gy = P[2 * s:, s:-s] - P[:-2 * s, s:-s]
        exp = np.array([[oracle.orientation_bin(int(x), int(y)) for x, y in zip(rx, ry)]
                        for rx, ry in zip(gx, gy)])
        assert (f[4 + li] == exp).all()
