"""The serving loop's admission queue on the host (no GPU): compiled with the system C++
compiler and run with fake work (see serve_queue_test.cpp)."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1503_03520_gb300", "csrc")


def test_admission_queue(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "serve_queue_test")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-I" + CSRC, os.path.join(HERE, "serve_queue_test.cpp"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "OK"
