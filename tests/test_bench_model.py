"""The byte model bench.py reports its step roofline against (CPU only).

The per-height model counts the HBM bytes of the Split_T recursion (Section 3,
Algorithm 2) run one tree level per pass over subtrees of at most 64 rows:
the image read once per quadrant, each leaf subtree written once, and every
node above the leaves reading its two children and writing its own rows.  Row
widths are L + m - 1 for an m-row node with the extended boundary and L with
the cyclic one (Section 2).  The sums below are written out by hand for small
trees; the 4095 x 4095 figures are the ones the bench quotes.

Also: the bench reports a kernel's captured DRAM traffic only while the
forward kernels' sources hash as they did at the capture, takes its peak
from the measured copy bandwidth when there is one, else the fallback, and
reads the median SM clock and the throttle reasons from its clock samples.
"""
import os

import bench


def test_leaf_only_tree():
    # 64 x 64: one leaf per quadrant, no upper level
    ext = 4 * (64 * 64 * 4 + 64 * (64 + 63) * 4)
    cyc = 4 * (64 * 64 * 4 + 64 * 64 * 4)
    assert bench.per_height_model_bytes(64, 64, True) == ext
    assert bench.per_height_model_bytes(64, 64, False) == cyc


def test_one_upper_level():
    # 128 x 128: two 64-row leaves and one merge per quadrant
    leaf = 64 * (128 + 63) * 4
    merge = (2 * 64 * (128 + 63) + 128 * (128 + 127)) * 4
    assert bench.per_height_model_bytes(128, 128, True) == 4 * (128 * 128 * 4 + 2 * leaf + merge)
    leaf_c = 64 * 128 * 4
    merge_c = (2 * 64 * 128 + 128 * 128) * 4
    assert bench.per_height_model_bytes(128, 128, False) == 4 * (128 * 128 * 4 + 2 * leaf_c + merge_c)


def test_uneven_split_and_transposed_quadrants():
    # 100 x 30: quadrants 0, 1 split 100 rows (64 + 36) of length 30; quadrants 2, 3
    # are the transpose, 30 rows of length 100 (one leaf)
    ext_01 = 100 * 30 * 4 + (64 * 93 + 36 * 65) * 4 + (64 * 93 + 36 * 65 + 100 * 129) * 4
    ext_23 = 30 * 100 * 4 + 30 * 129 * 4
    assert bench.per_height_model_bytes(100, 30, True) == 2 * ext_01 + 2 * ext_23
    cyc_01 = 100 * 30 * 4 + 100 * 30 * 4 + (100 * 30 + 100 * 30) * 4
    cyc_23 = 30 * 100 * 4 + 30 * 100 * 4
    assert bench.per_height_model_bytes(100, 30, False) == 2 * cyc_01 + 2 * cyc_23


def test_headline_figures():
    assert bench.per_height_model_bytes(4095, 4095, True) == 4_551_938_688
    assert bench.per_height_model_bytes(4095, 4095, False) == 3_756_261_600


def _fake_root(tmp_path, traffic_hash=None, peaks=None):
    import json
    import shutil

    csrc = tmp_path / "paper_2411_07351_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in bench.FORWARD_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2411_07351_gb300", "csrc", fn), csrc / fn)
    (tmp_path / "profiles").mkdir()
    if traffic_hash is not None:
        (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(
            {"c2-extended": {"fused_kernel": {"source_hash": traffic_hash, "dram_bytes_per_launch": 123}}}))
    if peaks is not None:
        (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(peaks))
    return str(tmp_path)


def test_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    root = _fake_root(tmp_path / "a", traffic_hash="0" * 16)
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench._traffic("fused_kernel", "c2-extended") is None  # taken on other sources
    root = _fake_root(tmp_path / "c", traffic_hash=bench._source_hash())
    monkeypatch.setattr(bench, "ROOT", root)
    assert bench._traffic("fused_kernel", "c2-extended") == 123
    assert bench._traffic("band_kernel", "c2-extended") is None
    # any change to a forward source voids the figure
    src = os.path.join(root, "paper_2411_07351_gb300", "csrc", "fht_forward.cu")
    with open(src, "a") as f:
        f.write("\n// changed\n")
    assert bench._traffic("fused_kernel", "c2-extended") is None


def test_peak_is_measured_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _fake_root(tmp_path / "a", peaks={"hbm_gbs": 6697.2}))
    assert bench._peaks() == (6697.2, "measured")
    monkeypatch.setattr(bench, "ROOT", _fake_root(tmp_path / "b"))
    assert bench._peaks() == (6800.0, "fallback")


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_give_median_and_throttle_reasons(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits lines of the fields in bench.CLOCK_FIELDS
    path = tmp_path / "clocks.csv"
    path.write_text(
        "0, 2070, 2070, 330.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 900.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 310.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n"
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    d = bench.clocks_stop((_DoneProcess(), str(path)))
    assert d["sm_mhz"] == 2070 and d["sm_max_mhz"] == 2070 and d["samples"] == 3
    assert d["power_w_max"] == 900.0
    assert d["reasons"] == ["sw_power_cap"]  # kept and noted; not a reason to reject
    path.write_text("0, 1200, 2070, 500.0, 0x8, Active, Not Active, Active, Not Active\n")
    d = bench.clocks_stop((_DoneProcess(), str(path)))
    assert d["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and d["sm_mhz"] == 1200


def test_no_nvidia_smi_is_reported():
    d = bench.clocks_stop((None, "unused"))
    assert d["sm_mhz"] is None and d["reasons"] == ["nvidia-smi unavailable"]
