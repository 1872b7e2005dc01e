"""FP64 form against the oracle, bit for bit, on seeded random small problems
with structured exact zeros (zero entries of d and e, sparse or zero columns
of B and C, m > n spikes, m < n, ranks above 1): the cases that exercise the
schedule's zero rules (no rotation for g = 0, the signed swap for f = 0)."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _case(rng):
    n = int(rng.integers(1, 24))
    m = n + int(rng.integers(0, 12))
    r = int(rng.integers(1, 4))
    Q = I.householder_orthogonal(m, rng)
    P = I.householder_orthogonal(n, rng)
    d = rng.standard_normal(n) * (rng.random(n) > 0.3)
    e = rng.standard_normal(max(n - 1, 0)) * (rng.random(max(n - 1, 0)) > 0.3)
    B = rng.standard_normal((m, r)) * (rng.random((m, r)) > 0.5)
    C = rng.standard_normal((n, r)) * (rng.random((n, r)) > 0.5)
    if rng.random() < 0.1:
        B[:] = 0.0
    if rng.random() < 0.1:
        C[:] = 0.0
    return Q, d, e, P, np.asfortranarray(B), np.asfortranarray(C)


def test_fp64_structured_zeros_bitwise():
    rng = np.random.default_rng(20250905)
    for _ in range(60):
        Q, d, e, P, B, C = _case(rng)
        with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
            F.update(B, C)
            got = F.read()
        want = O.update(Q, d, e, P, B, C)[:4]
        for a, b in zip(got, want):
            assert np.array_equal(a, b)


def test_fp64_lower_structured_zeros_bitwise():
    rng = np.random.default_rng(20250906)
    done = 0
    while done < 30:
        Qt, d, e, Pt, Bt, Ct = _case(rng)
        if Qt.shape[0] == Pt.shape[0]:
            continue
        Q, P, B, C = Pt, Qt, np.asfortranarray(Ct), np.asfortranarray(Bt)  # m < n
        with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
            F.update(B, C)
            got = F.read()
        want = O.update_lower(Q, d, e, P, B, C)[:4]
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        done += 1
