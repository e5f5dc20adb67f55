"""The serving loop's first-fit device-memory allocator (host bookkeeping),
compiled with g++ and checked against a brute-force byte map."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1711_06127_b300", "csrc")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_first_fit_allocator_against_brute_force(tmp_path):
    exe = str(tmp_path / "arena_test")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "arena_test.cpp"), "-o", exe],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
