"""bench.py host logic that decides what the JSON line reports (CPU only):
the clock record parsed from nvidia-smi samples, the peaks and their
source, and the ncu traffic figure that is reported only while the kernel
sources still hash to the digest the counters were taken on."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(lines, monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    c = bench.Clocks(0)
    c.file.write("\n".join(lines) + "\n")
    c.proc = _Proc()
    return c.stop()


def test_clock_record(monkeypatch):
    row = "0, {sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"
    lines = [row.format(sm=s, cap="Not Active") for s in (1900, 1950, 2000)]
    lines.append(row.format(sm=1800, cap="Active"))
    lines.append("0, [N/A], 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active")
    lines.append("garbage")
    rec = _clocks_from(lines, monkeypatch)
    assert rec["sm_mhz"] == 1925.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 4
    assert rec["reasons"] == ["sw_power_cap"]       # "Not Active" is not active
    hot = "0, 1500, 2070, 1390, 0x8, Active, Not Active, Active, Not Active"
    assert _clocks_from([hot], monkeypatch)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert _clocks_from([], monkeypatch)["reasons"] == ["no samples"]


def test_clocks_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
    os.unlink(c.file.name)


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    p = bench.peaks(152)
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert p["src"] == "measured"
    # FP32 FMA peak from the device's SMs x 128 lanes x 2 FLOP x 2.07 GHz
    assert p["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.peaks(148)["fp32_tflops"] == pytest.approx(148 * 128 * 2 * 2.07e9 / 1e12)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    f = bench.peaks(152)
    assert f["src"] == "fallback" and f["hbm_gbs"] == 6800.0


def _fake_root(tmp_path):
    src = os.path.join(ROOT, "paper_2402_15641_gb300", "csrc")
    dst = tmp_path / "paper_2402_15641_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.o", "*.so"))
    (tmp_path / "profiles").mkdir()
    return dst


def test_traffic_reported_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    csrc = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.csrc_digest()
    prof = tmp_path / "profiles" / "traffic_w.txt"
    prof.write_text(f"# comment = ignored\ncsrc_sha = {digest}\n"
                    "dram_bytes_per_launch.fwd.spmm2 = 1002149120\n")
    assert bench.ncu_traffic("fwd.spmm2", "w") == 1002149120.0
    assert bench.ncu_traffic("adj.spmm1t", "w") is None       # not recorded
    assert bench.ncu_traffic("fwd.spmm2", "other") is None    # no summary
    # the measurement helper is not on the path: editing it keeps the figure
    with open(csrc / "peak.cu", "a") as fh:
        fh.write("\n// edited\n")
    assert bench.csrc_digest() == digest
    # any kernel source edit makes it stale
    with open(csrc / "spmm.cu", "a") as fh:
        fh.write("\n// edited\n")
    assert bench.csrc_digest() != digest
    assert bench.ncu_traffic("fwd.spmm2", "w") is None


@pytest.mark.parametrize("extra", [[], ["--rho-linear", "--voxel-linear"], ["--weights", "bf16"]])
def test_reference_arm_runs_on_cpu(extra):
    """`bench.py --impl reference` (the FP64 oracle on the host cores) on the
    16^3 workload prints its one JSON line, with every option of the CUDA
    arm accepted."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "srt16fd", "--steps", "1", "--warmup", "0", *extra],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
