"""bench.py reports a kernel's ncu DRAM traffic from profiles/ncu_traffic.json
only while the coupling kernel sources hash to the value stored with it, and
only for a launch shape (variant, chunks) the record holds; a record taken on
other source, or on other shapes, reads as null."""

import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_traffic_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_committed_record_is_consistent():
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)["coupling_fp32_L4"]
    assert len(rec["source_hash"]) == 16 and "--clock-control none" in rec["command"]
    assert rec["shapes"]
    current = rec["source_hash"] == b.kernel_source_hash()
    for key, e in rec["shapes"].items():
        assert e["dram_bytes_per_launch"] == e["dram_read"] + e["dram_write"]
        v, ch = (int(q) for q in key.split(","))
        assert 0 <= v <= 7 and ch >= 1
        assert b.ncu_traffic("coupling_fp32_L4", (v, ch)) == (e["dram_bytes_per_launch"] if current else None)
        if v & 4:  # the L2 reduction keeps the sums out of DRAM: at most 2.5x the 4.2 MB algorithmic bytes
            assert e["dram_bytes_per_launch"] < 10.5e6
    assert b.ncu_traffic("coupling_fp32_L4", (0, 100000)) is None
    assert b.ncu_traffic("coupling_fp32_L4") is None  # no shape given


def test_record_of_other_source_or_missing_key_reads_as_none(tmp_path, monkeypatch):
    b = _bench()
    (tmp_path / "profiles").mkdir()
    rec = {"coupling_fp32_L4": {"dram_bytes_per_launch": 123, "dram_read": 100, "dram_write": 23,
                                "source_hash": "0000000000000000"}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "ffffffffffffffff")
    assert b.ncu_traffic("coupling_fp32_L4") is None
    assert b.ncu_traffic("no_such_kernel") is None
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "0000000000000000")
    assert b.ncu_traffic("coupling_fp32_L4") == 123
    # a record of several launch shapes answers only for those shapes
    rec = {"coupling_fp32_L4": {"source_hash": "0000000000000000",
                                "shapes": {"5,64": {"dram_bytes_per_launch": 7, "dram_read": 7, "dram_write": 0}}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    assert b.ncu_traffic("coupling_fp32_L4", (5, 64)) == 7
    assert b.ncu_traffic("coupling_fp32_L4", (0, 64)) is None
    assert b.ncu_traffic("coupling_fp32_L4") is None
    monkeypatch.setattr(b, "kernel_source_hash", lambda: "ffffffffffffffff")
    assert b.ncu_traffic("coupling_fp32_L4", (5, 64)) is None
