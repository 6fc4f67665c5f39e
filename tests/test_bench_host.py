"""Host-side logic of bench.py that needs no GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_only():
    src = "int f(int a) {\n    return a + 1;  // add one\n}\n/* block\n comment */\n"
    same = "// header\nint f(int a) {\n\n    return a + 1;\n}\n"
    other = "int f(int a) {\n    return a + 2;\n}\n"
    assert bench.code_hash(src) == bench.code_hash(same)
    assert bench.code_hash(src) != bench.code_hash(other)


def test_kernel_traffic_requires_matching_code(tmp_path, monkeypatch):
    """A profile taken on other code is not reported (traffic = None)."""
    import json
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "enum_kernel_traffic.json").write_text(
        json.dumps({"code_sha256": "0" * 64, "bytes_per_full_launch": 1.0}))
    csrc = tmp_path / "paper_2407_20474_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "fz_enum.cu").write_text("int x;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic(6) is None
    rec = {"code_sha256": bench.code_hash("int x;\n"), "bytes_per_full_launch": 5.0}
    (prof / "enum_kernel_traffic.json").write_text(json.dumps(rec))
    assert bench.kernel_traffic(6) == 5.0
