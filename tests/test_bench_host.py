"""Host-side logic of the benchmark (no GPU): the DRAM-traffic record is tied
to the transport kernel's source, the peaks come from the measured file or
the stated fallback, and the reference leg prints one JSON line with the
contract's keys."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_record_matches_the_kernel_source():
    # the committed ncu record belongs to the committed transport source, and
    # stays far below the algorithmic bytes of a launch (40 B x 4.59e9 free
    # flights): the phantom is read from L2, the source records once
    t = bench.kernel_traffic()
    assert isinstance(t, int) and 1e7 < t < 0.1 * bench.BYTES_PER_STEP_ALGO * 4.593e9


def test_traffic_record_is_dropped_for_another_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1204_6367_gb300" / "csrc").mkdir(parents=True)
    src = open(os.path.join(ROOT, "profiles", "mc_kernel_torso2mm_traffic.txt")).read()
    (tmp_path / "profiles" / "mc_kernel_torso2mm_traffic.txt").write_text(src)
    kernel = open(os.path.join(ROOT, "paper_1204_6367_gb300", "csrc", "mc_transport.cu")).read()
    (tmp_path / "paper_1204_6367_gb300" / "csrc" / "mc_transport.cu").write_text(kernel + "\n// edited\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic() is None
    (tmp_path / "paper_1204_6367_gb300" / "csrc" / "mc_transport.cu").write_text(kernel)
    assert bench.kernel_traffic() == int(dict(l.split() for l in src.splitlines()
                                              if l.strip() and not l.startswith("#"))["bytes_per_launch"])


def test_instruction_record_matches_the_kernel_source(tmp_path, monkeypatch):
    ipp = bench.kernel_inst_per_step()
    assert ipp is not None and 50.0 < ipp < 2000.0
    # the records name the macro cells they were taken with
    shift = int(bench.profile_record("mc_kernel_torso2mm_issue.txt")["cell_shift"])
    assert bench.kernel_inst_per_step(shift) == ipp and bench.kernel_inst_per_step(shift + 1) is None
    assert bench.kernel_traffic(shift) is not None and bench.kernel_traffic(shift + 1) is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))           # no record there
    assert bench.kernel_inst_per_step() is None


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak("hbm_gbs", 6800.0) == 6800.0          # no file: the stated fallback
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6790.3}))
    assert bench.measured_peak("hbm_gbs", 6800.0) == pytest.approx(6790.3)
    assert bench.measured_peak("bf16_tflops", 1900.0) == 1900.0      # missing key: the fallback


def test_reference_leg_prints_the_contract_line():
    # a tiny run of the CPU reference arm (the oracle on host cores)
    env = dict(os.environ, PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"],
                         capture_output=True, text=True, timeout=900, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_transport_roofline_entry():
    # the headline: algorithmic voxel bytes (40 B per free flight) against the HBM copy peak
    r = bench.transport_roofline(4.593e9, 0.0988, 6790.3, 51540736, 275.3, 152, 2070.0, {"l2_gather_frac": 0.74})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6790.3
    assert r["frac"] == pytest.approx(40 * 4.593e9 / 0.0988 / 1e9 / 6790.3)
    assert r["traffic"] == 51540736 and r["mc_ms"] == pytest.approx(98.8) and r["l2_gather_frac"] == 0.74
    # the issue rate rides along: 275.3 instructions per flight against 152 x 4 x 32 lanes x 2.07 GHz
    assert r["issue_peak_tinst_s"] == pytest.approx(40.28, rel=1e-3)
    assert r["issue_frac"] == pytest.approx(0.3177, rel=1e-3)
    json.dumps(r)
    # without an instruction record for this source and launch configuration
    h = bench.transport_roofline(4.593e9, 0.0988, 6790.3, None)
    assert h["bound"] == "hbm" and h["issue_frac"] is None and h["traffic"] is None


def test_instruction_record_is_keyed_to_the_launch_configuration(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1204_6367_gb300" / "csrc").mkdir(parents=True)
    kernel = open(os.path.join(ROOT, "paper_1204_6367_gb300", "csrc", "mc_transport.cu")).read()
    (tmp_path / "paper_1204_6367_gb300" / "csrc" / "mc_transport.cu").write_text(kernel)
    import hashlib
    h = hashlib.sha256(kernel.encode()).hexdigest()[:16]
    (tmp_path / "profiles" / "mc_kernel_torso2mm_issue.txt").write_text(
        f"cell_shift 2\nsource_sha256_16 {h}\nconfig 64 20 8 250.0 20.0 1000\nconfig 512 16 1 260.0 18.0 1000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    cfg = {"block_size": 64, "batch_min": 20, "hist_per_thread": 8}
    assert bench.kernel_inst_per_step(2, cfg) == 250.0
    assert bench.kernel_inst_per_step(2, dict(cfg, batch_min=16)) is None
    assert bench.kernel_inst_per_step(2, dict(cfg, block_size=128)) is None
    assert bench.kernel_inst_per_step(2, dict(cfg, block_size=512, batch_min=16, hist_per_thread=1)) == 260.0
    assert bench.kernel_inst_per_step(2, dict(cfg, hist_per_thread=64)) == 250.0     # not part of the key
    assert bench.kernel_inst_per_step(3, cfg) is None
