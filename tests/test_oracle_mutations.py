"""The pins bite: plant one plausible mistake at a time in a copy of the
oracle's C source (on the CPU), rebuild it, and check that the pins of
test_oracle_pins.py reject the mutant.  The oracle itself is untouched."""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ih_oracle.c")

# (name, original text, mutated text, pin tests that must fail)
MUTANTS = [
    ("alg5_diag_sign", "up + left - diag", "up + left + diag",
     [lambda: pins.test_alg5_equals_enumeration(5, 6, 2, 3)]),
    ("alg5_drop_up", "up + left - diag", "left - diag",
     [lambda: pins.test_alg5_constant_image(128)]),
    ("bin_denominator", "(v * B) / 256", "(v * B) / 255",
     [lambda: pins.test_uniform_binning_matches_edges(3)]),
    ("rect_row_exclusive", "o[k] = 0;\n        for (int r = q[0]; r <= q[2]; r++)",
     "o[k] = 0;\n        for (int r = q[0]; r < q[2]; r++)",
     [pins.test_rect_hist_is_bincount_of_slice, pins.test_four_corner_identity_all_rects]),
    ("kernel_transposed_axes", "dc * dc / (2.0 * wdt * wdt)", "dc * dc / (2.0 * hgt * hgt)",
     [pins.test_weighted_single_pixel_values]),
    ("kernel_sign", "return 1.0 - dc * dc", "return 1.0 + dc * dc",
     [lambda: pins.test_weighted_constant_image_closed_form((8, 8))]),
    ("kernel_centre_off_by_one", "double dc = 2.0 * c - (double)(q[1] + q[3]);",
     "double dc = 2.0 * c - (double)(q[1] + q[3] + 1);",
     [pins.test_weighted_mirror_symmetry]),
    ("weight_axes_swapped", "case OR_W_COL: return c;", "case OR_W_COL: return r;",
     [lambda: pins.test_weighted_ih_equals_cumsum(oracle.W_COL)]),
    ("orientation_fold", "if (gy < 0 || (gy == 0 && gx < 0)) {", "if (gy < 0) {",
     [lambda: pins.test_orientation_known((-1, 0), 0)]),
    ("orientation_step", "th / (M_PI / nb)", "th / (M_PI / (nb + 1))",
     [pins.test_orientation_exhaustive_vs_exact_integer_test]),
    ("intensity_rounding", "G[i] + B[i]) / 3)", "G[i] + B[i] + 1) / 3)",
     [pins.test_intensity_is_floor_mean]),
    ("hog_stencil_step", "clampi(c + s, 0, w - 1)", "clampi(c + 1, 0, w - 1)",
     [pins.test_hog_stencil_replicated_borders]),
    ("manhattan_centre", "int dr = 2 * r - (q[0] + q[2]), dc = 2 * c - (q[1] + q[3]);",
     "int dr = 2 * r - (q[0] + q[2]), dc = 2 * c - (q[1] + q[3] + 1);",
     [pins.test_manhattan_equals_quadrant_decomposition]),
    ("manhattan_scale", "return (double)(hgt + wdt - abs(dr) - abs(dc));",
     "return (double)(hgt + wdt - abs(dr) - 2 * abs(dc));",
     [lambda: pins.test_manhattan_constant_image_closed_form((8, 8))]),
    ("match_window_extent", "for (int x = c; x < c + ww; x++) {", "for (int x = c; x <= c + ww; x++) {",
     [lambda: pins.test_match_window_equals_cumsum_boxes(3, 5)]),
    ("median_rank", "vals[(cnt + 1) / 2 - 1]", "vals[cnt / 2]",
     [lambda: pins.test_local_median_equals_counting(5, 4, 2)]),
    ("median_box_rows", "for (int y = r - m / 2; y <=", "for (int y = r - m / 2 + 1; y <=",
     [lambda: pins.test_local_median_equals_counting(5, 4, 2)]),
    ("isqrt_round_up", "    return lo;\n}", "    return hi;\n}",
     [pins.test_isqrt_exhaustive_against_math_isqrt]),
    ("phog_cell_offset", "for (int y = r0 + i * ch; y < r0 + (i + 1) * ch; y++)",
     "for (int y = r0 + i * cw; y < r0 + (i + 1) * ch; y++)",
     [lambda: pins.test_phog_descriptor_cells(2)]),
    ("pyramid_level_weight", "il / (double)(1 << (L - l + 1))", "il / (double)(1 << (L - l))",
     [pins.test_pyramid_match_kernel_forms_agree]),
    ("canny_binomial_kernel", "or_binom5[5] = {1, 4, 6, 4, 1};", "or_binom5[5] = {1, 3, 6, 3, 1};",
     [lambda: pins.test_canny_smoothing_is_binomial_convolution(0)]),
    ("canny_gradient_axes", "int64_t gy = (int64_t)S[(int64_t)clampi(r + 1, 0, h - 1) * w + c] - S[(int64_t)clampi(r - 1, 0, h - 1) * w + c];\n            M[",
     "int64_t gy = (int64_t)S[(int64_t)r * w + clampi(c + 1, 0, w - 1)] - S[(int64_t)clampi(r - 1, 0, h - 1) * w + c];\n            M[",
     [lambda: pins.test_canny_gradient_of_the_smoothed_image(0)]),
    ("canny_nms_diagonals_swapped", "dr = 1; dc = 1;            /* near 45 deg", "dr = -1; dc = 1;           /* near 45 deg",
     [lambda: pins.test_canny_suppression_and_thresholds_by_angle(0), pins.test_canny_step_edges_are_one_pixel_wide]),
    ("canny_nms_sector_test", "if (s2 < 2 * ax * ax) {", "if (s2 < 3 * ax * ax) {",
     [lambda: pins.test_canny_suppression_and_thresholds_by_angle(0)]),
    ("canny_nms_ties_kept", "if (m > mm && m >= mp)", "if (m >= mm && m >= mp)",
     [pins.test_canny_step_edges_are_one_pixel_wide]),
    ("canny_weak_threshold", "(m >= tlo ? 1 : 0)", "(m >= thi ? 1 : 0)",
     [pins.test_canny_hysteresis_keeps_connected_weak_runs]),
    ("canny_hysteresis_4_connected", "if ((a == 0 && b == 0) || y < 0", "if ((a == 0) == (b == 0) || y < 0",
     [lambda: pins.test_canny_hysteresis_is_8_connected_components(0)]),
    ("canny_hysteresis_off", "if (K[j] != 0 && !edges[j]) {", "if (K[j] == 2 && !edges[j]) {",
     [pins.test_canny_hysteresis_keeps_connected_weak_runs]),
    ("phog_edges_ignored", "int e = edge[(int64_t)r * w + c];", "int e = m > 0;",
     [pins.test_phog_planes_follow_the_stencil]),
    ("wedding_shrink_axes", "int dr = j * hgt / (2 * layers), dc = j * wdt / (2 * layers);",
     "int dr = j * wdt / (2 * layers), dc = j * hgt / (2 * layers);",
     [lambda: pins.test_wedding_cake_is_sum_of_nested_windows(3)]),
]


@pytest.mark.parametrize("name,old,new,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, monkeypatch, name, old, new, checks):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must be unique: %r" % old
    msrc = tmp_path / "mutant.c"
    msrc.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o",
                           str(so), str(msrc), "-lm", "-lpthread"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(str(so)))
    for check in checks:
        with pytest.raises(AssertionError):
            check()
