"""Host-side checks of the autotuner's persisted table (no GPU)."""
import json


def test_table_roundtrip(tmp_path, monkeypatch):
    from paper_1403_0968_gb300 import autotune

    monkeypatch.setenv("SEM_AUTOTUNE_TABLE", str(tmp_path / "t.json"))
    assert autotune._load() == {}
    autotune._store({"problem/fp32/N7/2^27": {"variant": 0, "ms": {"0": 1.0}}})
    assert json.load(open(tmp_path / "t.json"))["problem/fp32/N7/2^27"]["variant"] == 0
    assert autotune._key("batch", "fp32", 5, 1 << 20) == "batch/fp32/N5/2^20"
    (tmp_path / "t.json").write_text("not json")
    assert autotune._load() == {}
