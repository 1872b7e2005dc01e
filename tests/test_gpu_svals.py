"""Singular values of Bd on the device (bdu_singular_values): multisection on
the Golub-Kahan matrix against the oracle (a library SVD of the dense
bidiagonal), to ~1e-15 of the largest value, for updated factorizations and for
the degenerate cases (diagonal, zero and repeated entries, graded scales)."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _check(sv, d, e, k):
    ref = O.singular_values(d, e)[:k]
    assert sv.shape == (k,)
    assert np.all(np.diff(sv) <= 1e-13 * max(ref[0], 1e-300))
    assert np.max(np.abs(sv - ref)) <= 2e-14 * ref[0]


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
@pytest.mark.parametrize("m,n", [(50, 40), (300, 300), (700, 520)])
def test_updated_factorization(precision, m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=71)
    with bdu.Factorization(Q, d, e, P, precision=precision) as F:
        for h in range(2):
            F.update(*I.dense_update(m, n, h, config=0))
        dg, eg = F.read_bidiagonal()
        for k in (1, 9, n):
            _check(F.singular_values(k), dg, eg, k)


@pytest.mark.parametrize("case", ["diagonal", "zeros", "repeated", "graded", "one"])
def test_degenerate_bidiagonals(case):
    g = np.random.default_rng(5)
    n = 1 if case == "one" else 64
    d = g.uniform(1, 10, n)
    e = g.standard_normal(n - 1)
    if case == "diagonal":
        e[:] = 0.0
    elif case == "zeros":
        d[::7] = 0.0
        e[3::11] = 0.0
    elif case == "repeated":
        d[:] = 2.5
        e[:] = 0.0
        e[::2] = 1.0
    elif case == "graded":
        d = d * np.logspace(-9, 3, n)
        e = e * np.logspace(-9, 3, n)[:-1]
    m = n + 3
    Q, P = np.eye(m), np.eye(n)
    with bdu.Factorization(Q, d, e, P) as F:
        _check(F.singular_values(), d, e, n)
        assert F.singular_values(0).shape == (0,)
        with pytest.raises(bdu.BduError):
            F.singular_values(n + 1)
