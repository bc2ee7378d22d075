"""Host logic of the benchmark's roofline bookkeeping: the DRAM traffic and L2
figures are taken from the committed ncu summary only while its source hash
matches the tracer source, and each figure carries the capture it came from."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

HEADER = """# k_trace summary

source_hash: {h}
dram_bytes_per_segment: 34.97
traffic_case: full launch, single-pass ncu
l2_hit_rate: 0.580
l2_atomic_alu_frac: 0.144
l2_atomic_input_max_slice_frac: 0.228
l2_case: 100-source launch, ncu --set full

text that follows the header
"""


def _with_profile(tmp_path, monkeypatch, h, current):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_trace_cosmic_256.md").write_text(HEADER.format(h=h))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: current)
    return bench.profiled_traffic()


def test_profile_used_while_the_hash_matches(tmp_path, monkeypatch):
    prof, h = _with_profile(tmp_path, monkeypatch, "abc123", "abc123")
    assert h == "abc123"
    assert prof["dram_bytes_per_segment"] == 34.97
    assert prof["l2_hit_rate"] == 0.58
    assert prof["l2_atomic_alu_frac"] == 0.144
    assert prof["l2_atomic_input_max_slice_frac"] == 0.228
    assert prof["traffic_case"] == "full launch, single-pass ncu"
    assert prof["l2_case"] == "100-source launch, ncu --set full"


def test_profile_dropped_once_the_tracer_changes(tmp_path, monkeypatch):
    prof, h = _with_profile(tmp_path, monkeypatch, "abc123", "def456")
    assert prof is None and h == "abc123"


def test_missing_profile_gives_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic() == (None, None)


def test_committed_profile_header_parses():
    """The committed summary's header has every key the bench reads (its hash
    may lag the source between a kernel change and the next capture)."""
    txt = open(os.path.join(ROOT, "profiles", "k_trace_cosmic_256.md")).read()
    keys = [ln.split(":", 1)[0] for ln in txt.splitlines()[:12] if ":" in ln]
    for k in ("source_hash", "dram_bytes_per_segment", "traffic_case", "l2_hit_rate",
              "l2_atomic_alu_frac", "l2_atomic_input_max_slice_frac", "l2_case"):
        assert k in keys, k
