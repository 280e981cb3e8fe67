"""The C ABI from plain C: tests/c/solve_example.c is compiled against
include/tw.h and linked to libtw.so (CPU test), then run on the GPU."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_09990_gb300 import native
    libdir = os.path.dirname(native.LIB_PATH)
    exe = tmp_path / "solve_example"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "solve_example.c"), "-o", str(exe),
                           "-L", libdir, "-ltw", "-Wl,-rpath," + libdir])
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert _build(tmp_path).exists()


@pytest.mark.gpu
def test_c_client_solves(tmp_path):
    out = subprocess.run([str(_build(tmp_path))], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "grid3x3: status 0 tw 3" in out.stdout
