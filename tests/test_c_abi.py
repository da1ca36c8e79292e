"""The C ABI from plain C (tests/c/four_stream.c): compiled and linked with gcc against
include/num_pmp.h and the in-tree library only, no Python or PyTorch types involved.
Without a GPU the program runs its host-only checks; with one it solves the paper's
four-stream example and compares it with the closed form."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "four_stream.c")
LIBDIR = os.path.join(ROOT, "paper_2509_10722_b300", "lib")


@pytest.fixture(scope="module")
def exe():
    from paper_2509_10722_b300 import build
    build.build()
    outdir = os.path.join(ROOT, "tests", "c", "build")  # git-ignored
    os.makedirs(outdir, exist_ok=True)
    out = os.path.join(outdir, "four_stream")
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    SRC, "-o", out, "-L", LIBDIR, "-lnum_pmp", f"-Wl,-rpath,{LIBDIR}", "-lm"],
                   check=True)
    return out


def test_c_program_builds_and_runs_host_checks(exe):
    r = subprocess.run([exe, "--no-gpu"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_program_solves_the_four_stream_example(exe):
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "max error" in r.stdout
