"""The roofline numerator of bench.py: algorithmic bytes per launch of each
kernel on the FMV workload (1920x1080, 7 channels = 91 bins, 16 weighted
bins, 100,000 rectangles, 4,096 windows), counted from the sizes by hand."""
import json


def test_fmv_algorithmic_bytes():
    import bench
    hw = 1920 * 1080
    assert (bench.H, bench.W, bench.N_RECTS, bench.N_WINDOWS) == (1080, 1920, 100_000, 4096)
    B, Bw = 91, 16
    count_tiles = 7 * hw + 4 * B * hw            # 7 channel planes in, 91 int32 planes out
    moment_tiles = hw + 4 * 8 * Bw * hw          # the intensity plane in, 4 x 16 int64 planes out
    assert bench.algorithmic_bytes("tiles/count+moments", B, Bw, 100_000, 4096) == count_tiles + moment_tiles
    assert count_tiles + moment_tiles == 1_833_062_400
    rects = 100_000 * (16 + 4 * B * 4 + 4 * B)   # box in, 4 corners x 91 int32 in, 91 int32 out
    wins = 4096 * (16 + 4 * Bw * (4 + 4 * 8) + 4 * Bw)  # box, per bin 4 corners x (count + 4 moments), out
    assert bench.algorithmic_bytes("queries", B, Bw, 100_000, 4096) == rects + wins
    assert bench.algorithmic_bytes("features", B, Bw, 100_000, 4096) == 7 * hw
    assert bench.algorithmic_bytes("tile_sums", B, Bw, 100_000, 4096) == 7 * hw


def test_wami_algorithmic_bytes():
    import bench
    hw = 8192 * 8192
    B = Bw = 32
    tiles = hw + 4 * B * hw + hw + 4 * 8 * Bw * hw    # gray in (counts, moments), 32 int32 + 4 x 32 int64 out
    assert bench.algorithmic_bytes("tiles/count+moments", B, Bw, 10 ** 6, 10 ** 5, hw, 1) == tiles
    assert tiles == 77_443_629_056
    assert bench.algorithmic_bytes("queries", B, Bw, 10 ** 6, 10 ** 5, hw, 1) == (
        10 ** 6 * (16 + 16 * B + 4 * B) + 10 ** 5 * (16 + 4 * Bw * 36 + 4 * Bw))


def test_traffic_only_for_the_profiled_sources(tmp_path, monkeypatch):
    import bench
    d = {"source_digest": bench.source_digest(),
         "workloads": {"fmv": {"kernels": {"queries": {"dram_bytes_per_launch": 123.0}}}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda: d["source_digest"])
    assert bench.dram_traffic("queries") == 123.0
    assert bench.dram_traffic("queries", "wami") is None
    assert bench.dram_traffic("features") is None
    monkeypatch.setattr(bench, "source_digest", lambda: "another")
    assert bench.dram_traffic("queries") is None
