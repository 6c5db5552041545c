"""Host-side helpers of bench.py on CPU: the algorithmic bytes per node update
the roofline divides by, and the lookup of the DRAM traffic the committed ncu
summary records (taken only while the step kernel's sources are the ones the
capture ran on)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("model,storage,scalar,want", [
    ("bgk", "fp32", "q7", (19 + 7) * 4 * 2),
    ("bgk", "fp32", "q6", (19 + 6) * 4 * 2),
    ("cumulant", "fp32", "q7", (27 + 7) * 4 * 2),
    ("cumulant", "fp32", "q27", (27 + 27) * 4 * 2),
    # 16 bits: every population read and written once in 2 bytes, the
    # scalar's rest population in an FP32 row (none on D3Q6)
    ("bgk", "fp16s", "q7", (19 + 6) * 2 * 2 + 4 * 2),
    ("bgk", "bf16s", "q6", (19 + 6) * 2 * 2),
    ("cumulant", "fp16s", "q7", (27 + 6) * 2 * 2 + 4 * 2),
    ("cumulant", "fp16s", "q27", (27 + 26) * 2 * 2 + 4 * 2),
])
def test_bytes_per_node(model, storage, scalar, want):
    assert bench.bytes_per_node(model, storage, scalar) == want


def _summary(path, h, box=1000, per_launch=207_000.0, per_node=207.0):
    path.write_text(f"# capture\n\nbox_nodes: {box}\ndram_bytes_per_launch: {per_launch}\n"
                    f"dram_bytes_per_node_update: {per_node}\nkernel_source_hash: {h}\n")


def test_traffic_of_the_captured_box(tmp_path, monkeypatch):
    p = tmp_path / "t.md"
    _summary(p, bench.kernel_hash())
    monkeypatch.setattr(bench, "PROFILE", str(p))
    b, why = bench.profiled_traffic(1000)
    assert b == 207_000.0 and "this box" in why
    b, why = bench.profiled_traffic(4000)          # another box: per node, scaled
    assert b == pytest.approx(207.0 * 4000) and "scaled" in why


def test_traffic_refused_after_a_kernel_change(tmp_path, monkeypatch):
    p = tmp_path / "t.md"
    _summary(p, "0" * 16)
    monkeypatch.setattr(bench, "PROFILE", str(p))
    assert bench.profiled_traffic(1000) == (None, "kernel changed since the capture")
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic(1000)[0] is None


def test_committed_summary_names_its_kernel_sources():
    """The committed summary carries the hash of the sources it was captured
    on and the box it ran on (it may be older than the sources: the bench
    then reports no traffic rather than a stale one)."""
    txt = open(bench.PROFILE).read()
    assert "kernel_source_hash:" in txt and "box_nodes:" in txt
    assert "--clock-control none" in txt
    assert all(os.path.exists(os.path.join(ROOT, s)) for s in bench.KERNEL_SOURCES)


def test_workload_config_names_the_scalar_lattice():
    c = bench.config_dict(1, "cumulant", "fp16s", False, "q27")
    assert "D3Q27 cumulant + D3Q27 FCM scalar, FP16S storage" in c["workload"]
    assert c["nodes"] == 2048 * 128 * 256
