"""CPU checks of bench.py's bookkeeping: the source hash that keys recorded ncu traffic ignores
comments but not code, and recorded traffic is reported only while its kernel's sources are
the ones it was captured from."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_strips_comments_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) {  // add one\n  return x + 1;\n}\n/* block\n comment */\n")
    b.write_text("// header\nint f(int x) {\n\n  return x + 1;   \n}\n")
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench._code_only(str(a)) == bench._code_only(str(b))
    assert bench._code_only(str(a)) != bench._code_only(str(c))


def test_recorded_traffic_is_used_only_for_unchanged_sources():
    t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, entry in t.items():
        kernel, workload = key.split("@")
        assert os.path.exists(os.path.join(ROOT, entry["capture"]))
        got = bench.recorded_traffic(kernel, workload)
        if entry["source_hash"] == bench.kernel_source_hash(kernel):
            assert got == entry["dram_bytes_per_launch"], key
        else:
            assert got is None, key
