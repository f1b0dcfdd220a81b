"""The serving arena's budget accounting on the CPU (paper_2607_05622_gb300/csrc/arena.h):
a budget that is not a multiple of the block size is rounded down, so a
request between the usable and the raw budget is refused at submission
instead of waiting forever at the head of the first-come-first-served queue;
first-fit allocation, alignment and coalescing of freed blocks."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "_build")


def test_arena_budget_rounding_and_coalescing():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "arena_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2607_05622_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "arena ok" in r.stdout
