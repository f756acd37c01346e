"""Calls made with another device current than the plan's are refused
(SRT_ERR_ARG) before any launch: tests/plan_device_check.cu marks a real
plan as made on another device index and calls every entry point that runs
work, then restores it and checks the calls succeed."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plan_device_mismatch_refused(tmp_path):
    from paper_2402_15641_gb300 import build
    lib = build.build()
    exe = tmp_path / "plan_device_check"
    subprocess.run([build.nvcc(), "-std=c++17", "-O1", *build.ARCH,
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2402_15641_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "plan_device_check.cu"), "-o", str(exe), lib,
                    f"-Xlinker=-rpath,{os.path.dirname(lib)}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout, r.stderr)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().endswith("OK")
