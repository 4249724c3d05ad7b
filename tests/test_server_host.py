"""Host logic of the request server that needs no GPU: the arena
bookkeeping (first fit, alignment, no overlap, coalescing) checked against a
byte-map model by a small C++ driver compiled here."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2609_15217_gb300", "csrc")


def test_arena_against_model():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "arena_check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I" + CSRC, os.path.join(HERE, "cpu_helpers", "arena_check.cpp"),
                        "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
