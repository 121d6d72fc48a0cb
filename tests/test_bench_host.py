"""Host logic of bench.py that needs no GPU: the workloads it builds from its
flags, the algorithmic bytes per fluid node that the roofline divides by, and
the reading of the committed ncu summaries (DRAM bytes per launch, taken only
when the summary was made on the current kernel source)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_tube_slab_planes_and_rounding_flags():
    args = bench.parse_args(["--workload", "tube_slab", "--planes", "24", "--precision", "f16",
                             "--rounding", "nearest"])
    g, c, p, desc = bench._workload(args.workload, args.precision, args.planes, args.rounding)
    assert g["nz"] == 24 and g["nx"] == g["ny"] == 256
    assert p["precision"] == "f16" and p["rounding"] == "nearest"
    assert "nearest rounding" in desc and "256x256x24" in desc
    # FP32 carries no rounding mode
    g, c, p, desc = bench._workload("tube_slab", "f32", 20)
    assert "rounding" not in p and desc.endswith("FP32 populations")
    # the defaults: the tube, stochastic rounding
    args = bench.parse_args([])
    assert args.workload == "tube" and args.rounding == "stochastic" and args.planes == 20


def test_algorithmic_bytes_per_node():
    """Populations read and written (19 x 4 B each way in FP32, 19 x 2 B with
    16-bit storage), u written (12 B), with cells G and theta read (16 B) and
    the stress written (24 B, when the elongational torque is on), one byte
    of node flags on walled lattices."""
    tube = {"solid": object()}
    box = {"solid": None}
    f32, f16 = {"precision": "f32"}, {"precision": "f16"}
    assert bench._algorithmic_bytes_per_node(tube, f32) == 205
    assert bench._algorithmic_bytes_per_node(tube, f16) == 129
    assert bench._algorithmic_bytes_per_node(tube, f32, has_cells=False) == 165
    assert bench._algorithmic_bytes_per_node(box, f32, has_cells=False) == 164
    assert bench._algorithmic_bytes_per_node(box, f16, has_cells=False) == 88
    assert bench._algorithmic_bytes_per_node(tube, dict(f32, alpha_tt=0.0)) == 181


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    """A summary whose source hash is the current kernel source's gives its
    DRAM bytes per launch; any other hash gives None (stale counters are not
    reported)."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    cur = bench._lb_source_hash()
    (prof / "lb_pass_tube.md").write_text(f"source_sha256_16: {cur}\ndram_bytes_per_launch: 2719223808\n")
    (prof / "lb_pass_tube_f16.md").write_text("source_sha256_16: 0123456789abcdef\ndram_bytes_per_launch: 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is taken from the package sources, which stay where they are
    monkeypatch.setattr(bench, "_lb_source_hash", lambda: cur)
    assert bench._profiled_traffic("tube") == pytest.approx(2719223808.0)
    assert bench._profiled_traffic("tube", "f16") is None
    assert bench._profiled_traffic("channel") is None
    # the launch's time alone, when the summary gives it
    assert bench._profiled_lb("tube")["alone_us"] is None
    (prof / "lb_pass_channel.md").write_text(
        f"source_sha256_16: {cur}\ndram_bytes_per_launch: 171991296\nalone_us_per_launch: 37.4\n")
    got = bench._profiled_lb("channel")
    assert got["traffic"] == pytest.approx(171991296.0) and got["alone_us"] == pytest.approx(37.4)
    assert got["summary"] == os.path.join("profiles", "lb_pass_channel.md")


def test_committed_lattice_summaries_are_current():
    """Every committed summary of the lattice pass carries the hash of the
    current kernel source (else the bench line reports no traffic), its DRAM
    bytes and its time alone."""
    for w, p in (("tube", "f32"), ("tube", "f16"), ("channel", "f32"), ("channel", "f16")):
        got = bench._profiled_lb(w, p)
        assert got is not None, (w, p)
        assert got["traffic"] > 0 and got["alone_us"] > 0
