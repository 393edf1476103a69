"""Host-side pieces of bench.py: the roofline's DRAM traffic is taken from a
committed ncu summary only when that summary was made on the current kernel
source, and the peak comes from the measured-peaks file."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    # a scratch tree: the real kernel source, a profiles folder of our own
    os.makedirs(tmp_path / "paper_1912_08453_gb300" / "csrc")
    src = open(os.path.join(ROOT, "paper_1912_08453_gb300", "csrc", "ccpm_kernels.cu"), "rb").read()
    (tmp_path / "paper_1912_08453_gb300" / "csrc" / "ccpm_kernels.cu").write_bytes(src)
    os.makedirs(tmp_path / "profiles")
    monkeypatch.setattr(mod, "ROOT", str(tmp_path))
    return mod, tmp_path


def test_traffic_only_for_matching_source(bench):
    mod, root = bench
    h = mod.kernel_source_hash()
    prof = root / "profiles" / "dram_wl.md"
    prof.write_text(f"kernel-source-sha256: {h}\ndram-bytes-per-launch k_lcc_round: 1234\n")
    assert mod.recorded_traffic("k_lcc_round", "wl") == 1234.0
    assert mod.recorded_traffic("k_nlcc_items", "wl") is None
    prof.write_text("kernel-source-sha256: 0000000000000000\ndram-bytes-per-launch k_lcc_round: 1234\n")
    assert mod.recorded_traffic("k_lcc_round", "wl") is None
    assert mod.recorded_traffic("k_lcc_round", "other") is None


def test_peak_from_measured_file(bench):
    mod, root = bench
    assert mod.measured_peak_hbm() == (6800.0, "fallback")
    (root / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.5}))
    assert mod.measured_peak_hbm() == (7000.5, "measured")


def test_hash_tracks_the_source(bench):
    mod, root = bench
    h = mod.kernel_source_hash()
    p = root / "paper_1912_08453_gb300" / "csrc" / "ccpm_kernels.cu"
    p.write_bytes(p.read_bytes() + b"\n")
    assert mod.kernel_source_hash() != h
