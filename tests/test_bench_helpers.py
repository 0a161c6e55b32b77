"""Host-side helpers of the benchmark: the DRAM-traffic figure is used only for the code it was measured on."""
import json
import os
import shutil

import bench

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1609_05722_gb300", "csrc")


def _copy_tree(tmp_path):
    d = tmp_path / "paper_1609_05722_gb300" / "csrc"
    d.mkdir(parents=True)
    for name in {n for names in bench.KERNEL_SOURCES.values() for n in names}:
        shutil.copy(os.path.join(CSRC, name), d / name)
    (tmp_path / "profiles").mkdir()
    return d


def test_code_only_drops_comments_and_blank_lines():
    src = "int a = 1;  // one\n\n   // a whole comment line\nint b = 2;\t\n"
    assert bench.code_only(src) == "int a = 1;\nint b = 2;"


def test_sha_ignores_comments_but_not_code(tmp_path, monkeypatch):
    d = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    before = bench.kernel_source_sha("foe_tc_step")
    p = d / "foe_tc.cu"
    p.write_text("// an added comment line\n" + p.read_text() + "\n// and another\n")
    assert bench.kernel_source_sha("foe_tc_step") == before
    p.write_text(p.read_text() + "\nstatic const int unused_marker = 0;\n")
    assert bench.kernel_source_sha("foe_tc_step") != before


def test_traffic_figure_needs_matching_code(tmp_path, monkeypatch):
    _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"source_sha": bench.kernel_source_sha("foe_tc_step"), "bytes_per_launch": 123}
    path = tmp_path / "profiles" / "traffic.json"
    path.write_text(json.dumps({"foe_tc_step": entry}))
    assert bench.ncu_traffic("foe_tc_step") == 123
    entry["source_sha"] = "0" * 16
    path.write_text(json.dumps({"foe_tc_step": entry}))
    assert bench.ncu_traffic("foe_tc_step") is None
    assert bench.ncu_traffic("foe_f32_step") is None
