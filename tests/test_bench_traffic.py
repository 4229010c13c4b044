"""The DRAM traffic that bench.py reports beside the roofline comes from the
committed ncu summary (profiles/traffic.json), keyed to the accumulate
kernel's own source text: the region markers must exist, the hash must be
of that text only, and a changed kernel must read as unmeasured (None)."""

import json
import os

import bench


def test_region_markers_exist_and_hash_the_region_only(tmp_path, monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for ent in d.values():
        h = bench.kernel_source_hash(ent["source"], ent.get("region"))
        assert h is not None and len(h) == 16
    # text outside the region does not change the hash, text inside does
    src = tmp_path / "paper_1303_7425_gb300" / "csrc"
    src.mkdir(parents=True)
    body = "// head\n// BEGIN x\nint k = 1;\n// END y\n// tail\n"
    (src / "k.cu").write_text(body)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    region = ["// BEGIN", "// END"]
    h0 = bench.kernel_source_hash("k.cu", region)
    assert h0 is not None
    (src / "k.cu").write_text(body.replace("// tail", "// other tail").replace("// head", "// other head"))
    assert bench.kernel_source_hash("k.cu", region) == h0
    (src / "k.cu").write_text(body.replace("int k = 1;", "int k = 2;"))
    assert bench.kernel_source_hash("k.cu", region) != h0
    assert bench.kernel_source_hash("k.cu", ["// NOPE", "// END"]) is None


def test_changed_kernel_reads_as_unmeasured(tmp_path, monkeypatch):
    src = tmp_path / "paper_1303_7425_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "k.cu").write_text("// a\n// BEGIN\nint k;\n// END\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("k.cu", ["// BEGIN", "// END"])
    ent = {"kernel": "k_x", "source": "k.cu", "region": ["// BEGIN", "// END"], "source_sha256_16": h,
           "dram_bytes_per_launch": 1234}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"w": ent}))
    assert bench.traffic_for("k_x", "w") == 1234
    assert bench.traffic_for("k_y", "w") is None
    (src / "k.cu").write_text("// a\n// BEGIN\nint k = 3;\n// END\n")
    assert bench.traffic_for("k_x", "w") is None
