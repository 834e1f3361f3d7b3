"""The render server's host core (allocator, FIFO admission, latency
percentiles) compiled as a plain C++ program and run on the CPU."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_serve_core(tmp_path):
    exe = str(tmp_path / "test_serve_core")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall",
                           "-I", os.path.join(ROOT, "paper_2110_06635_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "test_serve_core.cpp"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "serve core: ok" in out.stdout
