"""The apply autotuner (bdu_options.nb = 0): after the first update of a shape
it has not seen, every candidate tile shape is timed on scratch copies of Q and
P and the fastest is kept.  Every candidate computes the same thing, so the
tuned handle's results equal those of each forced variant bit for bit; the
choice is cached for the process and, with BDU_TUNE_FILE, across processes."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(precision, m, n, nb, ups=3):
    Q, d, e, P = I.factorization(m, n, config=0, which=53)
    with bdu.Factorization(Q, d, e, P, precision=precision, nb=nb,
                           check_every=0 if precision == bdu.MIXED else None) as F:
        for h in range(ups):
            F.update(*I.dense_update(m, n, h, config=0))
        return F.read(), F.stats()


@pytest.mark.parametrize("precision,m,n,forced", [
    (bdu.FP64, 311, 293, [2, 6, 16, 64]),
    (bdu.MIXED, 612, 533, [1, 2, 3, 4, 5]),
])
def test_tuned_equals_every_forced_variant(precision, m, n, forced):
    tuned, st = _run(precision, m, n, 0)
    assert st["tunings"] == 2
    assert all(v != 0 for v in st["apply_variant"])
    again, st2 = _run(precision, m, n, 0)  # same shape: the process cache answers
    assert st2["tunings"] == 0 and st2["apply_variant"] == st["apply_variant"]
    for nb in forced:
        got, sf = _run(precision, m, n, nb)
        assert sf["tunings"] == 0 and sf["apply_variant"] == [nb, nb]
        for a, b in zip(got, tuned):
            assert np.array_equal(a, b), nb


def test_bad_variant_is_rejected():
    Q, d, e, P = I.factorization(40, 30, config=0, which=1)
    for precision, nb in ((bdu.FP64, 3), (bdu.FP64, 66), (bdu.MIXED, 6), (bdu.MIXED, -1)):
        with pytest.raises(bdu.BduError):
            bdu.Factorization(Q, d, e, P, precision=precision, nb=nb)


def test_choices_persist_in_the_tune_file(tmp_path):
    path = str(tmp_path / "tune.json")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2509_02840_gb300 import bdu, inputs as I\n"
            "Q, d, e, P = I.factorization(257, 199, config=0, which=9)\n"
            "with bdu.Factorization(Q, d, e, P) as F:\n"
            "    F.update(*I.dense_update(257, 199, 0, config=0))\n"
            "    st = F.stats()\n"
            "print(st['tunings'], *st['apply_variant'])\n" % ROOT)
    env = dict(os.environ, BDU_TUNE_FILE=path)
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    t1, q1, p1 = map(int, first.stdout.split())
    assert t1 == 2
    table = json.load(open(path))
    assert any("|fp64|257|" in k for k in table) and any("|fp64|199|" in k for k in table)
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    t2, q2, p2 = map(int, second.stdout.split())
    assert t2 == 0 and (q2, p2) == (q1, p1)
