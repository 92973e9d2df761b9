"""Host-side logic of the library checked on the CPU, compiled from the
library's own headers: the serving loop's device-memory sub-allocator and its
watchdog over batches in flight."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_09118_gb300", "csrc")


@pytest.fixture(scope="module")
def arena_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    src = os.path.join(ROOT, "tests", "native", "arena_check.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_output_arena_invariants(arena_check, seed):
    r = subprocess.run([arena_check, str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.fixture(scope="module")
def watch_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("watch") / "watch_check")
    src = os.path.join(ROOT, "tests", "native", "watch_check.cpp")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_serve_watchdog_never_completing_batch(watch_check, seed):
    # a batch whose completion event never fires: its requests time out once,
    # after the limit; its output memory and slot stay held until it ends
    r = subprocess.run([watch_check, str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
