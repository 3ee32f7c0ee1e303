"""Host-side helpers of bench.py (no GPU): the comment-free source hash that
keys the committed ncu traffic figure, the figure's lookup, and the roofline
denominators."""
import pytest

import bench


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // note\n'
           '/* block\n   comment */ const char *s = "a // b /* c */";\n'
           "char q = '\"';  \n"
           '\n'
           '  int b; /* t */\n')
    assert bench.strip_comments(src) == ('int a = 1;\n'
                                         ' const char *s = "a // b /* c */";\n'
                                         "char q = '\"';\n"
                                         '  int b;')


def test_comment_edits_do_not_change_the_stripped_source():
    a = "x = f(y);  // Algorithm 1\nz = 2;\n"
    b = "// a new line of commentary\nx = f(y);  /* reworded */\n\nz = 2;\n"
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments("x = f(y);\nz = 3;\n") != bench.strip_comments(a)


def test_kernel_source_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16


def _fake_tree(tmp_path, kernel_src="int k() { return 1; }\n"):
    """A copy of the layout bench.py reads: the bin kernels' sources and
    profiles/traffic.json."""
    csrc = tmp_path / "paper_1503_04500_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.BIN_KERNEL_SOURCES:
        (csrc / name).write_text(f"// {name}\n" + kernel_src)
    (tmp_path / "profiles").mkdir()
    return tmp_path


def test_traffic_figure_follows_the_kernel_sources(tmp_path, monkeypatch):
    """The committed DRAM figure is reported only while the bin kernels' code
    (comments aside) is the code it was measured on."""
    import json

    root = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h = bench.kernel_source_hash()
    entry = {"source_hash": h, "dram_bytes_per_launch": 12345}
    (root / "profiles" / "traffic.json").write_text(json.dumps({"k_bin_warp:fp32_refine": entry}))
    assert bench.traffic_from_profiles("k_bin_warp", "fp32_refine") == 12345
    assert bench.traffic_from_profiles("k_bin_warp", "fp64") is None  # no entry for this precision
    # a comment edit keeps the figure, a code edit drops it
    col = root / "paper_1503_04500_gb300" / "csrc" / "column.cuh"
    col.write_text("/* reworded */\n" + col.read_text())
    assert bench.traffic_from_profiles("k_bin_warp", "fp32_refine") == 12345
    col.write_text(col.read_text() + "int extra;\n")
    assert bench.traffic_from_profiles("k_bin_warp", "fp32_refine") is None
    (root / "profiles" / "traffic.json").unlink()
    assert bench.traffic_from_profiles("k_bin_warp", "fp32_refine") is None


def test_roofline_denominators(tmp_path, monkeypatch):
    """FP32 unit-count rate: SMs x 128 lanes x 2 flop x clock (152 SMs at 2070 MHz:
    80.5 TFLOP/s); the HBM figure comes from MEASURED_PEAKS.json, else the
    stated fallback."""
    import json

    assert bench.fp32_units_peak(152, 2070.0) / 1e12 == pytest.approx(80.54, abs=0.01)
    assert bench.fp32_units_peak(1, 1000.0) == 128 * 2 * 1e9
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_hbm_gbs() == (bench.HBM_FALLBACK_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6781.4}))
    gbs, src = bench.measured_hbm_gbs()
    assert gbs == 6781.4 and src.startswith("measured")
