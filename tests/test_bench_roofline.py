"""CPU: the roofline bookkeeping of bench.py.  The committed DRAM-traffic record
is used only while the kernel's source is the one the counters were taken on;
the roofline object names the dominant class, its achieved rate against the
peak, and the traffic's launch and algorithmic bytes."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_record_follows_the_source_hash(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2311_00921_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    src.write_text("kernel source v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\n"
        f"kernel=k_kernel prec=f64 src=k.cu src_sha={sha} bytes_per_launch=100 "
        "algo_bytes_per_launch=110 scale=4 case=a_small_case\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("k_kernel", "f64") == (400.0, "a small case", 440.0)
    assert bench.traffic_record("k_kernel", "f32") is None      # another arithmetic
    assert bench.traffic_record("other_kernel", "f64") is None
    src.write_text("kernel source v2\n")                          # the kernel changed
    assert bench.traffic_record("k_kernel", "f64") is None


def test_committed_traffic_record_matches_the_current_source():
    """The committed record of the dominant FP64 kernel is live (its source hash
    is the current file's), so the bench line's traffic is not null."""
    rec = bench.traffic_record("gemm_n16_kernel", "f64")
    assert rec is not None
    traffic, case, algo = rec
    assert 0.9 * algo <= traffic <= 1.1 * algo, (traffic, algo)   # no re-reads


def test_roofline_of_picks_the_dominant_class():
    tr = {"gemm_skinny.f64": (23.6, 121, 24.1e9), "ql.f32": (5.8, 9, 17.9e9),
          "trsv_fwd.f32": (3.5, 27, 1.0e9)}
    peaks = {"f64": 1.1, "f32": 80.0}
    r = bench.roofline_of(tr, peaks, steps=1)
    assert r["kernel"].startswith("gemm_n16_kernel")
    assert abs(r["achieved"] - 24.1e9 / 23.6e-3 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / 1.1) < 1e-12
    assert abs(r["kernel_share"] - 23.6 / (23.6 + 5.8 + 3.5)) < 1e-12
    assert r["kernel_launches_per_step"] == 121
