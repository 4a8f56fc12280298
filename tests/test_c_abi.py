"""libnbody from C: the header compiles as C11 and a C program links against
the library (CPU); the program runs a force evaluation on host arrays (GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_smoke.c")


def _build(tmp_path):
    from paper_2411_18889_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2411_18889_gb300 import build
        build.build()
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    exe = str(tmp_path / "abi_smoke")
    libdir = os.path.dirname(_lib.LIB_PATH)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"), SRC,
                    "-o", exe, "-L", libdir, "-lnbody", "-Wl,-rpath," + libdir, "-lm"], check=True)
    return exe


def test_header_is_c11_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_program_runs(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "c abi ok" in r.stdout
