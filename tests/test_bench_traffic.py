"""Host logic of bench.py's roofline `traffic`: a DRAM figure is read from a committed ncu
summary under profiles/ only while the summary's kernel-source hash equals the hash of the
current sources, so a figure never outlives the kernel it was measured on."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_matching_source_hash(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k.txt").write_text(
        "Kernel: k (one line: with a colon)\n"
        "kernel_source_sha256: " + "a" * 64 + "\n"
        "dram_bytes_per_launch: 1.5e6\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile("k.txt", "a" * 64) == 1.5e6
    assert bench.traffic_from_profile("k.txt", "b" * 64) is None
    assert bench.traffic_from_profile("missing.txt", "a" * 64) is None


def test_kernel_hash_is_a_sha256_of_the_sources():
    h = bench.kernel_hash()
    assert re.fullmatch(r"[0-9a-f]{64}", h)
    assert h == bench.kernel_hash()


def test_committed_summaries_carry_a_hash_and_a_positive_figure():
    for name in ("cgs_f64_gaussian_bumps_64.txt", "poly_stage_gaussian_bumps_64.txt"):
        vals = {}
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            for ln in fh:
                if ":" in ln:
                    k, v = ln.split(":", 1)
                    vals[k.strip()] = v.strip()
        assert re.fullmatch(r"[0-9a-f]{64}", vals["kernel_source_sha256"]), name
        assert float(vals["dram_bytes_per_launch"]) > 0, name
