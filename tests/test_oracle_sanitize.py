"""The oracle's C library under AddressSanitizer and UndefinedBehavior-
Sanitizer: tests/c/oracle_sanitize.c drives every entry point through
randomized problems with structured zeros and extreme magnitudes; any invalid
access, leak or undefined operation aborts it.  Also the rank-deficient case
that one-sided Jacobi must handle (a numerically null column)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_is_clean_under_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "oracle_sanitize"
    cmd = [gcc, "-std=c99", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-ffp-contract=off", os.path.join(ROOT, "tests", "c", "oracle_sanitize.c"),
           os.path.join(ROOT, "oracle", "bgu_oracle.c"), "-lm", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "oracle_sanitize ok" in r.stdout


def test_jacobi_on_a_singular_bidiagonal():
    d = np.array([-1.2598357859647178, 0.36848678121180339, 0.8016337373318031, -0.118686493721537, 0.0])
    e = np.array([-0.19069955598279378, 0.83491617545584251, -0.63417627565191315, 0.27142391215981232])
    X = O.bidiag_dense(d, e)
    sv = np.linalg.svd(X, compute_uv=False)
    np.testing.assert_allclose(O.jacobi_sv(X), sv, rtol=0, atol=1e-14 * sv[0])
