"""The boundary is a C ABI: a plain C99 program (tests/c/abi_check.c)
includes include/bdu.h, links against libbdu.so with gcc and runs the calls
that need no GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2509_02840_gb300 import bdu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_compiles_links_and_runs(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = bdu.library_path()
    bdu.load()  # builds the library when it is missing
    exe = tmp_path / "abi_check"
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", str(exe),
           "-L", os.path.dirname(lib), "-lbdu", "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi_check ok" in r.stdout
