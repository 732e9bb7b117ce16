"""bench.py's use of the committed ncu summary, on the CPU: the DRAM traffic of
the headline kernel is reported only while the fused-pass sources hash to the
value the summary records and the lattice runs the launch shape it was
captured with; otherwise the bench line carries null."""
import os
import pathlib
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

DEFAULT_1024 = {"kind": "tma", "warps": 15, "stages": 6, "z_chunk": 76, "tile_x": 0, "threads": 0}


def test_traffic_reported_exactly_when_summary_matches_sources_and_shape():
    txt = pathlib.Path(bench.TRAFFIC_FILE).read_text()
    current = (f"kernel source sha256[:16]: {bench.kernel_hash()}" in txt
               and f"launch shape of the capture: {bench.shape_tag(DEFAULT_1024)}" in txt)
    t = bench.measured_traffic(DEFAULT_1024)
    if current:  # about the algorithmic 34.36 GB per launch plus halo re-reads and ghost writes
        assert t is not None and 34.36e9 < t < 40e9
    else:
        assert t is None


def test_traffic_is_null_for_another_shape_or_changed_sources(monkeypatch, tmp_path):
    assert bench.measured_traffic(dict(DEFAULT_1024, z_chunk=72)) is None
    assert bench.measured_traffic(dict(DEFAULT_1024, kind="stream")) is None
    changed = tmp_path / "tl_pass_impl.cuh"
    changed.write_bytes(pathlib.Path(bench.KERNEL_SRCS[0]).read_bytes() + b"\n// edited\n")
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(changed)] + bench.KERNEL_SRCS[1:])
    assert bench.measured_traffic(DEFAULT_1024) is None
